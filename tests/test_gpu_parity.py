"""GPU parity of every hot-path entry point against the FP64 oracle.

Tolerances (from the method's arithmetic, see the design notes):
  * chain states: every site-update equals the oracle's draw given the same
    conditioning and Philox uniform, except draws whose uniform lies within
    1e-5 of a CDF boundary (FP32 vs FP64 fields); such flips are counted;
  * counts, identity counts: bit-exact;
  * weighted frequencies: 1e-6 absolute;
  * update: |dJ| <= 4 ulp(J) + 1e-7 absolute (one FP32 fma of FP32 inputs);
  * Pearson: 1e-6 absolute;
  * energies / mutant dE: FP32 sums of <= L(L-1)/2 terms, 2e-5 relative to
    the sum of absolute terms.
"""
import math

import numpy as np
import pytest
import torch

import fliplog
from fliplog import FLIP_MARGIN
from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


GIBBS_ENGINES = ["simt", "mma", "mma_pair", "mma_pair2"]


def load(bm, h, J, engine=None):
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    if engine is not None:
        bm.bm_model_set_engine(m, {"simt": bm.BM_ENGINE_SIMT, "mma": bm.BM_ENGINE_MMA,
                                   "mma_pair": bm.BM_ENGINE_MMA_PAIR,
                                   "mma_pair2": bm.BM_ENGINE_MMA_PAIR2}[engine])
    return m


def states_of(bm, c):
    out = torch.empty((c.M, c.L), dtype=torch.uint8, device=DEV)
    bm.bm_chains_get(c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def here():
    import os
    return os.environ.get("PYTEST_CURRENT_TEST", "?").split(" ")[0]


def check_sweep(orc, h, J, before, after, seed, sweep, beta=1.0, chain0=0):
    """Teacher-forced check of every site-update of one sweep; each flip is
    logged (chain, site, margin) in the run's flip record."""
    bad, worst = fliplog.verify(orc, h, J, before, after, seed, sweep, beta, chain0, here())
    assert bad == 0 or worst < FLIP_MARGIN, f"{bad} disagreeing draws, worst margin {worst}"
    assert bad <= max(2, before.size // 10000), f"too many boundary flips: {bad}"
    return bad


# ---------------------------------------------------------------- chains_init

@pytest.mark.parametrize("M,L,q", [(1024, 16, 21), (333, 37, 5), (1, 1, 1), (70, 64, 32)])
def test_chains_init_bit_exact(bm, orc, M, L, q):
    h, J = synth.planted_local_model(L, q, 1)
    m = load(bm, h, J)
    c = bm.bm_chains_init(m, M, 12345)
    assert np.array_equal(states_of(bm, c), orc.chains_init(M, L, q, 12345))
    assert bm.bm_chains_sweep_counter(c) == 0


def test_chains_init_from_states_and_symbol_check(bm):
    L, q, M = 10, 5, 20
    h, J = synth.planted_local_model(L, q, 2)
    m = load(bm, h, J)
    S = synth.random_states(M, L, q, 3)
    c = bm.bm_chains_init(m, M, 1, torch.from_numpy(S))
    assert np.array_equal(states_of(bm, c), S)
    S[3, 4] = q
    with pytest.raises(bm.BmError) as e:
        bm.bm_chains_init(m, M, 1, to_dev(S))
    assert e.value.code == bm.BM_EINVAL


# ---------------------------------------------------------------- gibbs_sweep

@pytest.mark.parametrize("M,L,q,beta", [
    (1024, 16, 21, 1.0),   # planted local model, training shape
    (333, 37, 5, 1.0),     # RNA alphabet, ragged sizes
    (70, 50, 21, 0.8),     # sampling temperature
    (129, 24, 32, 1.2),    # largest alphabet
    (45, 9, 3, 1.0),
    (17, 2, 1, 1.0),       # degenerate alphabet
    (200, 61, 4, 1.0),     # several blocks of 32 sites, ragged tail
    (150, 40, 8, 1.0),     # operand rows with 8 or 9 nonzeros per K chunk
    (90, 30, 9, 1.0),      # operand rows with exactly 8 nonzeros per K chunk
])
@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_single_sweep_teacher_forced(bm, orc, M, L, q, beta, engine):
    h, J = synth.planted_local_model(L, q, 5, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 99)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, beta)
    bm.bm_device_status(m)
    s1 = states_of(bm, c)
    check_sweep(orc, h, J, s0, s1, 99, 0, beta)
    assert bm.bm_chains_sweep_counter(c) == 1
    if q > 1:
        assert (s1 != s0).mean() > 0.05


@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_consecutive_sweeps_each_verified(bm, orc, engine):
    L, q, M = 20, 21, 300
    h, J = synth.planted_contact_model(L, q, 6, frac=0.2)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 4)
    prev = states_of(bm, c)
    for k in range(4):
        bm.bm_gibbs_sweep(m, c, 1, 1.0)
        bm.bm_device_status(m)
        cur = states_of(bm, c)
        check_sweep(orc, h, J, prev, cur, 4, k)
        prev = cur


@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_multi_sweep_call_equals_single_calls(bm, engine):
    """nsweeps in one call == the same sweeps one by one (keyed RNG)."""
    L, q, M = 33, 21, 500
    h, J = synth.planted_local_model(L, q, 7)
    m = load(bm, h, J, engine)
    a = bm.bm_chains_init(m, M, 8)
    b = bm.bm_chains_init(m, M, 8)
    bm.bm_gibbs_sweep(m, a, 5, 1.0)
    for _ in range(5):
        bm.bm_gibbs_sweep(m, b, 1, 1.0)
    assert np.array_equal(states_of(bm, a), states_of(bm, b))
    assert bm.bm_chains_sweep_counter(a) == bm.bm_chains_sweep_counter(b) == 5


@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_free_run_matches_oracle(bm, orc, engine):
    """Three free-running sweeps: chains whose every draw is far from a CDF
    boundary are identical to the oracle's own free run.  Each sweep is also
    checked teacher-forced, so every chain that left the oracle's trajectory
    is accounted for by a logged boundary flip (chain, site, margin)."""
    L, q, M = 16, 21, 256
    h, J = synth.planted_local_model(L, q, 9)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 10)
    s0 = states_of(bm, c)
    traj = [s0]
    for _ in range(3):  # one sweep per call equals one 3-sweep call (tested above)
        bm.bm_gibbs_sweep(m, c, 1, 1.0)
        traj.append(states_of(bm, c))
    got = traj[-1]
    flipped = set()
    for k in range(3):
        n0 = len(fliplog.FLIPS)
        check_sweep(orc, h, J, traj[k], traj[k + 1], 10, k)
        flipped |= {f["chain"] for f in fliplog.FLIPS[n0:]}
    want = orc.gibbs(h.astype(np.float64), J.astype(np.float64), s0, 10, 0, 3)
    differ = set(np.nonzero((got != want).any(axis=1))[0].tolist())
    assert differ <= flipped, f"chains off the oracle's trajectory without a logged flip: {differ - flipped}"
    assert len(differ) < 0.01 * M


@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_config2_launch_sampled_chains(bm, orc, engine):
    """Full-size launch (L=256, q=21, M=10000, contact-map model): one sweep,
    a sample of chains across CTAs and the ragged tail verified by the oracle."""
    L, q, M = 256, 21, 10000
    h, J = synth.planted_contact_model(L, q, 11)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 2024)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    bm.bm_device_status(m)
    s1 = states_of(bm, c)
    rng = np.random.default_rng(0)
    # CTA / cluster boundaries of the tensor-core forms (80 and 144 chains) and the tail
    sample = sorted(set(rng.choice(M, 24, replace=False).tolist()) | {0, 65, 66, 79, 80, 143, 144, M - 1})
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    for k in sample:
        bad, worst = fliplog.verify(orc, h64, J64, s0[k:k + 1], s1[k:k + 1], 2024, 0, 1.0, k, here())
        assert bad == 0 or worst < FLIP_MARGIN, (k, bad, worst)


@pytest.mark.parametrize("L,M", [(512, 300), (400, 200), (700, 64)])
@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_gibbs_long_sequences_teacher_forced(bm, orc, L, M, engine):
    """Long sequences: the main chunks after a pair's delta step outlast the
    redraw of the previous blocks, so any state a CTA reads too late (or a
    peer overwrites too early) shows up as wrong draws near the end of the
    sweep; every site of sampled chains over two sweeps is checked."""
    h, J = synth.planted_local_model(L, 21, 13, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 31)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    s1 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    bm.bm_device_status(m)
    s2 = states_of(bm, c)
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    sample = sorted(set(np.random.default_rng(2).choice(M, min(M, 40), replace=False).tolist()) | {M - 1})
    for k in sample:
        for sw, (a, b) in enumerate([(s0, s1), (s1, s2)]):
            bad, worst = fliplog.verify(orc, h64, J64, a[k:k + 1], b[k:k + 1], 31, sw, 1.0, k, here())
            assert bad == 0 or worst < FLIP_MARGIN, (k, sw, bad, worst)


@pytest.mark.parametrize("L,M", [(500, 200), (700, 150)])
def test_gibbs_pair_small_alphabet_long_rows_teacher_forced(bm, orc, L, M):
    """RNA alphabet at L = 500 and 700: the two-CTA sweep keeps the one-hot
    operand in tensor memory there (K chunks <= 4x the 20 sites of a block),
    and the state rows leave room for only 3 and 2 coupling-tile ring slots,
    so the ring wraps every few chunks.  Two sweeps of sampled chains,
    every site checked."""
    h, J = synth.planted_local_model(L, 5, 19, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, "mma_pair")
    c = bm.bm_chains_init(m, M, 41)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    s1 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    bm.bm_device_status(m)
    s2 = states_of(bm, c)
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    sample = sorted(set(np.random.default_rng(4).choice(M, 24, replace=False).tolist()) | {M - 1})
    for k in sample:
        for sw, (a, b) in enumerate([(s0, s1), (s1, s2)]):
            bad, worst = fliplog.verify(orc, h64, J64, a[k:k + 1], b[k:k + 1], 41, sw, 1.0, k, here())
            assert bad == 0 or worst < FLIP_MARGIN, (k, sw, bad, worst)


@pytest.mark.parametrize("L,q,M", [(900, 10, 160), (600, 16, 2000), (300, 32, 1500), (777, 21, 333)])
@pytest.mark.parametrize("engine", ["mma", "mma_pair"])
def test_gibbs_tensor_core_grid_teacher_forced(bm, orc, L, q, M, engine):
    """Tensor-core forms across alphabets (block sizes 12, 8, 4, 6 sites),
    long sequences, ragged chain counts: two sweeps, every site of sampled
    chains is the oracle's teacher-forced draw."""
    h, J = synth.planted_local_model(L, q, 17, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 41)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 2, 1.0)
    bm.bm_device_status(m)
    s2 = states_of(bm, c)
    # the intermediate states: replay the first sweep on a copy of the chains
    c1 = bm.bm_chains_init(m, M, 41)
    bm.bm_gibbs_sweep(m, c1, 1, 1.0)
    s1 = states_of(bm, c1)
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    sample = sorted(set(np.random.default_rng(3).choice(M, min(M, 14), replace=False).tolist()) | {0, M - 1})
    for k in sample:
        for sw, (a, b) in enumerate([(s0, s1), (s1, s2)]):
            bad, worst = fliplog.verify(orc, h64, J64, a[k:k + 1], b[k:k + 1], 41, sw, 1.0, k, here())
            assert bad == 0 or worst < FLIP_MARGIN, (k, sw, bad, worst)


@pytest.mark.parametrize("engine", ["mma", "mma_pair"])
def test_gibbs_more_chains_than_one_wave(bm, orc, engine):
    """M = 12000 chains: more CTAs (clusters) than the GPU runs at once, so
    later ones start when earlier ones finish; two sweeps, sampled chains of
    every part of the launch verified."""
    L, q, M = 24, 21, 12000
    h, J = synth.planted_local_model(L, q, 12, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 77)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    s1 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    bm.bm_device_status(m)
    s2 = states_of(bm, c)
    rng = np.random.default_rng(1)
    sample = sorted(set(rng.choice(M, 40, replace=False).tolist()) | {0, 159, 160, 11519, 11520, M - 1})
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    for k in sample:
        for sw, (a, b) in enumerate([(s0, s1), (s1, s2)]):
            bad, worst = fliplog.verify(orc, h64, J64, a[k:k + 1], b[k:k + 1], 77, sw, 1.0, k, here())
            assert bad == 0 or worst < FLIP_MARGIN, (k, sw, bad, worst)


def test_gibbs_rejects_bad_arguments(bm):
    h, J = synth.planted_local_model(8, 5, 1)
    m = load(bm, h, J)
    h2, J2 = synth.planted_local_model(9, 5, 1)
    m2 = load(bm, h2, J2)
    c = bm.bm_chains_init(m, 10, 1)
    for args in [(m2, c, 1, 1.0), (m, c, -1, 1.0), (m, c, 1, math.inf)]:
        with pytest.raises(bm.BmError) as e:
            bm.bm_gibbs_sweep(*args)
        assert e.value.code == bm.BM_EINVAL
    bm.bm_gibbs_sweep(m, c, 0, 1.0)  # zero sweeps is a no-op
    assert bm.bm_chains_sweep_counter(c) == 0


# ---------------------------------------------------------------- potts_load checks

def test_potts_load_checks(bm):
    h, J = synth.planted_local_model(6, 4, 3)
    bad = J.copy()
    bad[0, 1, 2, 3] += 1e-3
    with pytest.raises(bm.BmError) as e:
        load(bm, h, bad)
    assert e.value.code == bm.BM_EINVAL
    bad = J.copy()
    bad[2, 2, 0, 0] = 0.5
    with pytest.raises(bm.BmError) as e:
        load(bm, h, bad)
    assert e.value.code == bm.BM_EINVAL
    bad = h.copy()
    bad[1, 1] = np.nan
    with pytest.raises(bm.BmError) as e:
        load(bm, bad, J)
    assert e.value.code == bm.BM_ENUMERIC
    m = bm.bm_potts_load(torch.from_numpy(h), torch.from_numpy(J))  # host pointers
    hh = torch.empty_like(torch.from_numpy(h))
    JJ = torch.empty_like(torch.from_numpy(J))
    bm.bm_potts_get(m, hh, JJ)
    torch.cuda.synchronize()
    assert np.array_equal(hh.numpy(), h) and np.array_equal(JJ.numpy(), J)


@pytest.mark.parametrize("engine", ["mma", "mma_pair"])
def test_coupling_beyond_fp16_range_is_reported(bm, engine):
    """The tensor-core sweep holds J as fp16 hi + lo.  A coupling above the
    fp16 range is clamped (operands stay finite) and reported as
    BM_ENUMERIC by the status call; the FP32 engine takes the same model."""
    L, q, M = 8, 4, 64
    h, J = synth.planted_local_model(L, q, 3)
    J[1, 2, 0, 1] = J[2, 1, 1, 0] = 1.0e5
    m = load(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 1)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    with pytest.raises(bm.BmError) as e:
        bm.bm_device_status(m)
    assert e.value.code == bm.BM_ENUMERIC
    bm.bm_device_status(m)  # cleared
    m2 = load(bm, h, J, "simt")
    c2 = bm.bm_chains_init(m2, M, 1)
    bm.bm_gibbs_sweep(m2, c2, 1, 1.0)
    bm.bm_device_status(m2)


# ---------------------------------------------------------------- chain_stats

def upper_blocks_numpy(S, q, pairs):
    out = []
    for i, j in pairs:
        B = np.zeros((q, q), dtype=np.int64)
        np.add.at(B, (S[:, i], S[:, j]), 1)
        out.append(B)
    return out


STATS_ENGINES = ["simt", "mma_bf16", "mma_fp8"]


def set_stats_engine(bm, c, name):
    bm.bm_chains_set_stats_engine(c, {"simt": bm.BM_STATS_SIMT, "mma_bf16": bm.BM_STATS_MMA_BF16,
                                      "mma_fp8": bm.BM_STATS_MMA_FP8}[name])


@pytest.mark.parametrize("engine", STATS_ENGINES)
@pytest.mark.parametrize("M,L,q", [(1024, 16, 21), (333, 37, 5), (1, 3, 2), (700, 70, 32), (50, 1, 4),
                                   (129, 300, 21)])
def test_chain_stats_bit_exact(bm, orc, M, L, q, engine):
    h, J = synth.planted_local_model(L, q, 4)
    m = load(bm, h, J)
    S = synth.random_states(M, L, q, 5)
    c = bm.bm_chains_init(m, M, 0, to_dev(S))
    set_stats_engine(bm, c, engine)
    counts = torch.full((bm.n_blocks(L), q, q), -7, dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    bm.bm_chains_device_status(c)
    torch.cuda.synchronize()
    assert np.array_equal(counts.cpu().numpy(), orc.chain_stats(S, q))


@pytest.mark.parametrize("M,L,q", [(1024, 16, 21), (333, 37, 5), (129, 300, 21), (3000, 200, 21),
                                   (257, 1000, 4)])
def test_chain_stats_repeated_calls_on_one_handle(bm, orc, M, L, q):
    """Calls of the FP8 form on one chains handle, with sweeps between them:
    at these shapes some output tiles are split along the chains and summed
    through arrival tickets that each launch reuses, so every call must
    still equal the oracle's counts of the current states (Sec. 2.1)."""
    h, J = synth.planted_local_model(L, q, 6)
    m = load(bm, h, J)
    c = bm.bm_chains_init(m, M, 21)
    set_stats_engine(bm, c, "mma_fp8")
    counts = torch.full((bm.n_blocks(L), q, q), -3, dtype=torch.int32, device=DEV)
    for call in range(4):
        if call:
            bm.bm_gibbs_sweep(m, c, 1, 1.0)
        bm.bm_chain_stats(c, counts)
        bm.bm_chains_device_status(c)
        S = states_of(bm, c)
        assert np.array_equal(counts.cpu().numpy(), orc.chain_stats(S, q)), f"call {call}"


@pytest.mark.parametrize("engine", STATS_ENGINES)
def test_chain_stats_config2_properties_and_samples(bm, orc, engine):
    L, q, M = 256, 21, 10000
    h, J = synth.planted_contact_model(L, q, 3)
    m = load(bm, h, J)
    c = bm.bm_chains_init(m, M, 77)
    set_stats_engine(bm, c, engine)
    bm.bm_gibbs_sweep(m, c, 2, 1.0)
    S = states_of(bm, c)
    counts = torch.full((bm.n_blocks(L), q, q), -1, dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    bm.bm_chains_device_status(c)
    C = counts.cpu().numpy().astype(np.int64)
    assert C.min() >= 0
    diag = np.array([orc.block_index(L, i, i) for i in range(L)])
    single = np.stack([np.diag(C[d]) for d in diag])
    assert np.all(single.sum(axis=1) == M)
    rng = np.random.default_rng(1)
    pairs = [(0, 0), (0, 255), (254, 255), (7, 8)] + [tuple(sorted(rng.choice(L, 2, replace=False)))
                                                     for _ in range(40)]
    for (i, j), B in zip(pairs, upper_blocks_numpy(S, q, pairs)):
        assert np.array_equal(C[orc.block_index(L, i, j)], B)
        assert np.array_equal(C[orc.block_index(L, i, j)].sum(axis=1), single[i])


# ---------------------------------------------------------------- seq_weights

@pytest.mark.parametrize("N,L,seqid", [(500, 64, 0.8), (333, 37, 0.8), (130, 120, 0.8), (65, 300, 0.6),
                                       (1, 5, 0.8)])
def test_seq_weights_exact(bm, orc, N, L, seqid):
    X = synth.clustered_msa(N, L, 21, 6, n_ancestors=max(1, N // 10))
    w = torch.empty(N, dtype=torch.float32, device=DEV)
    meff = bm.bm_seq_weights(to_dev(X), w, seqid)
    w_o, meff_o = orc.seq_weights(X, seqid)
    assert np.array_equal(w.cpu().numpy(), w_o.astype(np.float32))
    assert meff == pytest.approx(meff_o, rel=1e-12)


def test_seq_weights_special_cases(bm):
    L = 40
    same = np.tile(synth.random_states(1, L, 21, 1), (70, 1))
    w = torch.empty(70, dtype=torch.float32, device=DEV)
    assert bm.bm_seq_weights(to_dev(same), w) == pytest.approx(1.0)
    assert torch.all(w == np.float32(1 / 70))
    far = np.array([[k % 21] * L for k in range(21)], dtype=np.uint8)
    w = torch.empty(21, dtype=torch.float32, device=DEV)
    assert bm.bm_seq_weights(to_dev(far), w) == 21.0


@pytest.mark.parametrize("top", [32, 256])
def test_seq_weights_byte_symbols(bm, orc, top):
    """Weights compare whole symbol bytes: symbols up to 255 (all eight bit
    planes of the bit-sliced comparison) and exactly 32 (the sixth plane),
    with near-identical rows so the threshold is exercised."""
    N, L = 300, 70
    rng = np.random.default_rng(top)
    base = rng.integers(0, top, size=(30, L), dtype=np.uint8)
    X = base[rng.integers(0, 30, size=N)].copy()
    flip = rng.random((N, L)) < 0.15
    X[flip] = rng.integers(0, top, size=int(flip.sum()), dtype=np.uint8)
    if top == 32:
        X[5, 3] = 32
    w = torch.empty(N, dtype=torch.float32, device=DEV)
    meff = bm.bm_seq_weights(to_dev(X), w, 0.8)
    w_o, meff_o = orc.seq_weights(X, 0.8)
    assert np.array_equal(w.cpu().numpy(), w_o.astype(np.float32))
    assert meff == pytest.approx(meff_o, rel=1e-12)
    assert 1.0 < meff < N


def test_seq_weights_config2_sampled_rows(bm, orc):
    N, L = 50000, 256
    X = synth.clustered_msa(N, L, 21, 12, n_ancestors=5000)
    w = torch.empty(N, dtype=torch.float32, device=DEV)
    meff = bm.bm_seq_weights(to_dev(X), w, 0.8)
    wh = w.cpu().numpy()
    thr = orc.identity_threshold(0.8, L)
    rng = np.random.default_rng(2)
    for m in rng.choice(N, 12, replace=False).tolist() + [0, N - 1]:
        Nm = ((X == X[m]).sum(axis=1) >= thr).sum()
        assert wh[m] == np.float32(1.0 / Nm)
    assert meff == pytest.approx(wh.astype(np.float64).sum(), rel=1e-6)
    assert 1.0 < meff < N


# ---------------------------------------------------------------- data_stats

@pytest.mark.parametrize("N,L,q,weighted,alpha", [(400, 16, 21, True, -1.0), (333, 37, 5, False, 0.1),
                                                  (90, 9, 32, True, 0.0), (10, 2, 2, True, 1.0)])
def test_data_stats_parity(bm, orc, N, L, q, weighted, alpha):
    X = synth.clustered_msa(N, L, q, 7, n_ancestors=max(1, N // 10))
    w = np.random.default_rng(3).uniform(0.05, 1.0, size=N).astype(np.float32) if weighted else None
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None if w is None else to_dev(w), q, alpha, fi, fij)
    meff = w.astype(np.float64).sum() if weighted else float(N)
    a = 1.0 / meff if alpha < 0 else alpha
    fi_o, fij_o = orc.data_stats(X, None if w is None else w.astype(np.float64), q, a)
    assert np.abs(fi.cpu().numpy() - fi_o).max() < 1e-6
    assert np.abs(fij.cpu().numpy() - fij_o).max() < 1e-6


def test_data_stats_rejects_bad_symbols(bm):
    X = synth.random_states(10, 5, 4, 1)
    X[2, 2] = 4
    fi = torch.empty((5, 4), dtype=torch.float32, device=DEV)
    fij = torch.empty((5, 5, 4, 4), dtype=torch.float32, device=DEV)
    with pytest.raises(bm.BmError) as e:
        bm.bm_data_stats(to_dev(X), None, 4, 0.1, fi, fij)
    assert e.value.code == bm.BM_EINVAL


# ---------------------------------------------------------------- update + pearson

@pytest.mark.parametrize("L,q,M", [(16, 21, 1024), (37, 5, 333), (2, 3, 10), (100, 21, 400), (9, 1, 20),
                                   (130, 2, 64), (600, 5, 300), (257, 21, 100)])
def test_update_and_pearson_parity(bm, orc, L, q, M):
    h, J = synth.planted_local_model(L, q, 8)
    m = load(bm, h, J)
    X = synth.clustered_msa(4 * M, L, q, 9, n_ancestors=M // 3 + 1)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None, q, 0.05, fi, fij)
    S = synth.random_states(M, L, q, 10)
    c = bm.bm_chains_init(m, M, 0, to_dev(S))
    counts = torch.empty((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    lr = 0.05
    rho, applied = bm.bm_update(m, fi, fij, counts, M, lr, 2.0)
    assert applied
    fih, fijh, Ch = fi.cpu().numpy(), fij.cpu().numpy(), counts.cpu().numpy()
    rho_o = orc.pearson(fih, fijh, Ch, M)
    if q == 1:  # every connected correlation is 0: the coefficient is undefined on both sides
        assert np.isnan(rho) and np.isnan(rho_o)
    else:
        assert abs(rho - rho_o) < 1e-6
    h_o, J_o = orc.update(h, J, fih, fijh, Ch, M, lr)
    hh = torch.empty((L, q), dtype=torch.float32)
    JJ = torch.empty((L, L, q, q), dtype=torch.float32)
    bm.bm_potts_get(m, hh, JJ)
    torch.cuda.synchronize()
    tolJ = 4 * np.spacing(np.abs(J_o).astype(np.float32)) + 1e-7
    assert np.all(np.abs(JJ.numpy() - J_o) <= tolJ)
    assert np.all(np.abs(hh.numpy() - h_o) <= 4 * np.spacing(np.abs(h_o).astype(np.float32)) + 1e-7)
    assert np.array_equal(JJ.numpy(), JJ.numpy().transpose(1, 0, 3, 2))


def test_update_respects_target(bm):
    """rho >= target: parameters unchanged; async form always applies."""
    L, q, M = 8, 4, 200
    h, J = synth.planted_local_model(L, q, 2)
    m = load(bm, h, J)
    S = synth.random_states(M, L, q, 3)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(S), None, q, 0.0, fi, fij)
    c = bm.bm_chains_init(m, M, 0, to_dev(S))
    counts = torch.empty((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    rho, applied = bm.bm_update(m, fi, fij, counts, M, 0.1, 0.95)
    assert rho == pytest.approx(1.0, abs=1e-6) and not applied
    JJ = torch.empty((L, L, q, q), dtype=torch.float32)
    bm.bm_potts_get(m, None, JJ)
    torch.cuda.synchronize()
    assert np.array_equal(JJ.numpy(), J)
    rho, applied = bm.bm_update(m, fi, fij, counts, M, 0.1, want_pearson=False)
    assert rho is None and applied


def test_pearson_config2_full_size(bm, orc):
    L, q, M = 256, 21, 10000
    h, J = synth.planted_contact_model(L, q, 5)
    m = load(bm, h, J)
    c = bm.bm_chains_init(m, M, 5)
    bm.bm_gibbs_sweep(m, c, 3, 1.0)
    counts = torch.empty((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    X = synth.clustered_msa(20000, L, q, 6, n_ancestors=2000)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None, q, -1.0, fi, fij)
    rho, _ = bm.bm_update(m, fi, fij, counts, M, 0.01, 2.0)
    # vectorised FP64 reference of the same definition on the same inputs
    fih, fijh = fi.cpu().numpy().astype(np.float64), fij.cpu().numpy().astype(np.float64)
    C = counts.cpu().numpy().astype(np.float64) / M
    iu, ju = np.triu_indices(L, 1)
    blk = iu * L - iu * (iu - 1) // 2 + (ju - iu)
    diag = np.arange(L) * L - np.arange(L) * (np.arange(L) - 1) // 2
    p1 = np.stack([np.diag(C[d]) for d in diag])
    x = (fijh[iu, ju] - fih[iu][:, :, None] * fih[ju][:, None, :]).ravel()
    y = (C[blk] - p1[iu][:, :, None] * p1[ju][:, None, :]).ravel()
    assert rho == pytest.approx(np.corrcoef(x, y)[0, 1], abs=1e-6)


# ---------------------------------------------------------------- energy / mutant scan

@pytest.mark.parametrize("n,L,q", [(300, 16, 21), (1000, 37, 5), (0, 4, 3), (5, 1, 2), (64, 256, 21),
                                   # batches with n*L >= 3.3e6 take the staged form
                                   (170000, 20, 21), (90000, 37, 5), (60000, 64, 21), (12000, 300, 21)])
def test_energy_parity(bm, orc, n, L, q):
    h, J = synth.planted_contact_model(L, q, 3, frac=0.3) if L > 2 else synth.planted_local_model(L, q, 3)
    m = load(bm, h, J)
    S = synth.random_states(max(n, 1), L, q, 4)[:n]
    E = torch.empty(n, dtype=torch.float32, device=DEV)
    bm.bm_energy_score(m, to_dev(S).reshape(n, L), E)
    torch.cuda.synchronize()
    if n == 0:
        return
    E_o = orc.energy(h.astype(np.float64), J.astype(np.float64), S)
    scale = np.abs(h).max() * L + np.abs(J).max() * L * L / 2
    assert np.abs(E.cpu().numpy() - E_o).max() < 2e-5 * scale + 1e-6


@pytest.mark.parametrize("n", [100, 300000])
def test_energy_invalid_symbol_flagged(bm, n):
    L, q = 12, 5
    h, J = synth.planted_local_model(L, q, 3)
    m = load(bm, h, J)
    S = synth.random_states(n, L, q, 4)
    S[n // 2, 3] = q + 1
    E = torch.empty(n, dtype=torch.float32, device=DEV)
    bm.bm_energy_score(m, to_dev(S), E)
    with pytest.raises(bm.BmError) as e:
        bm.bm_device_status(m)
    assert e.value.code == bm.BM_EINVAL
    bm.bm_device_status(m)  # cleared


@pytest.mark.parametrize("L,q", [(16, 21), (37, 5), (256, 21), (1, 3)])
def test_mutant_scan_parity(bm, orc, L, q):
    h, J = synth.planted_local_model(L, q, 12, sigma_h=1.0, sigma_J=0.2)
    m = load(bm, h, J)
    wt = synth.random_states(1, L, q, 13)[0]
    dE = torch.empty((L, q), dtype=torch.float32, device=DEV)
    bm.bm_mutant_scan(m, torch.from_numpy(wt), dE)
    torch.cuda.synchronize()
    got = dE.cpu().numpy()
    want = orc.mutant_scan(h.astype(np.float64), J.astype(np.float64), wt)
    assert np.all(got[np.arange(L), wt] == 0.0)
    assert np.abs(got - want).max() < 1e-5 * (1 + np.abs(want).max())
    dE2 = torch.empty((L, q), dtype=torch.float32, device=DEV)
    bm.bm_mutant_scan(m, to_dev(wt), dE2)  # device wild type
    torch.cuda.synchronize()
    assert torch.equal(dE2.cpu(), dE.cpu())


# ---------------------------------------------------------------- sharding

@pytest.mark.parametrize("engine", GIBBS_ENGINES)
def test_shards_reproduce_the_full_ensemble(bm, engine):
    """Chains split into shards with global chain indices draw the states of
    one handle holding all of them, and their counts sum to its counts."""
    from paper_2501_18456_gb300 import sharding
    L, q, M = 40, 21, 700
    h, J = synth.planted_local_model(L, q, 6, sigma_h=1.0, sigma_J=0.3)
    m = load(bm, h, J, engine)
    full = bm.bm_chains_init(m, M, 55)
    bm.bm_gibbs_sweep(m, full, 4, 1.0)
    shards = []
    for r in range(3):
        first, n = sharding.shard_range(M, r, 3)
        c = bm.bm_chains_init_shard(m, n, 55, first)
        bm.bm_gibbs_sweep(m, c, 4, 1.0)
        shards.append(c)
    bm.bm_device_status(m)
    assert np.array_equal(np.concatenate([states_of(bm, c) for c in shards]), states_of(bm, full))
    tot = torch.zeros((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    part = torch.empty_like(tot)
    for c in shards:
        bm.bm_chain_stats(c, part)
        tot += part
    ref = torch.empty_like(tot)
    bm.bm_chain_stats(full, ref)
    torch.cuda.synchronize()
    assert torch.equal(tot, ref)


def test_sweep_engine_resolution(bm):
    """AUTO (rules fitted to a measured L x q x M grid): CUDA cores for short
    sequences with few chains, tensor cores otherwise; among those the
    paired-tensor-core form for short coupling rows (L q^2 < 90000) and the
    two-CTA form for long ones; for small alphabets the two-CTA form runs
    its tensor-memory operand form unless that needs more waves of clusters
    than the paired form fitting one wave, or the paired form spreads the
    chains at most 32 per cluster.  Explicit engines are kept."""
    h, J = synth.planted_local_model(256, 21, 3)
    m = load(bm, h, J)
    assert bm.bm_model_sweep_engine(m, 10000) == bm.BM_ENGINE_MMA_PAIR
    assert bm.bm_model_sweep_engine(m, 1024) == bm.BM_ENGINE_MMA_PAIR
    assert bm.bm_model_sweep_engine(m, 1) == bm.BM_ENGINE_SIMT  # one chain: a small problem
    bm.bm_model_set_engine(m, bm.BM_ENGINE_MMA)
    assert bm.bm_model_sweep_engine(m, 1) == bm.BM_ENGINE_MMA
    assert bm.bm_model_sweep_engine(m, 10000) == bm.BM_ENGINE_MMA
    bm.bm_model_set_engine(m, bm.BM_ENGINE_MMA_PAIR2)
    assert bm.bm_model_sweep_engine(m, 10000) == bm.BM_ENGINE_MMA_PAIR2
    # short coupling rows: the paired tensor cores
    hs, Js = synth.planted_local_model(120, 21, 3)
    ms = load(bm, hs, Js)
    assert bm.bm_model_sweep_engine(ms, 10000) == bm.BM_ENGINE_MMA_PAIR2
    assert bm.bm_model_sweep_engine(ms, 1024) == bm.BM_ENGINE_MMA_PAIR2
    hm, Jm = synth.planted_local_model(200, 21, 3)
    mm = load(bm, hm, Jm)
    assert bm.bm_model_sweep_engine(mm, 10000) == bm.BM_ENGINE_MMA_PAIR2
    h5, J5 = synth.planted_local_model(64, 5, 3)
    m5 = load(bm, h5, J5)
    assert bm.bm_model_sweep_engine(m5, 10000) == bm.BM_ENGINE_SIMT
    # short sequences with few chains go to the gather even for large alphabets
    h48, J48 = synth.planted_local_model(48, 21, 3)
    m48 = load(bm, h48, J48)
    assert bm.bm_model_sweep_engine(m48, 1000) == bm.BM_ENGINE_SIMT
    assert bm.bm_model_sweep_engine(m48, 10000) == bm.BM_ENGINE_MMA_PAIR2
    # small alphabets: the two-CTA form's tensor-memory operand form while it
    # fits one wave with more than 32 chains per paired cluster
    h4, J4 = synth.planted_local_model(256, 4, 3)
    m4 = load(bm, h4, J4)
    assert bm.bm_model_sweep_engine(m4, 5000) == bm.BM_ENGINE_MMA_PAIR
    assert bm.bm_model_sweep_engine(m4, 10000) == bm.BM_ENGINE_MMA_PAIR2  # 79 clusters of 128: two waves
    assert bm.bm_model_sweep_engine(m4, 1000) == bm.BM_ENGINE_MMA_PAIR2
    assert bm.bm_model_sweep_engine(m4, 500) == bm.BM_ENGINE_SIMT
    with pytest.raises(bm.BmError) as e:
        bm.bm_model_sweep_engine(m5, 0)
    assert e.value.code == bm.BM_EINVAL
