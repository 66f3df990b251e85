"""GPU parity of the sparse-graph steps (Sec. 2.2, "Training sparse models").

Element decimation (edDCA) and activation (eaDCA) are scored in FP64 on both
sides, so the GPU must select the oracle's elements; an element may differ
only where its oracle score lies within rounding (1e-12 relative) of the
selection boundary, since the two sides' exp and log may differ in the
last bits.  The masked update is compared with the oracle's, and the graph
bookkeeping (counts, symmetry, zero couplings) is checked directly.
"""
import numpy as np
import pytest
import torch

from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu
DEV = "cuda"


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def element_index(L, q):
    """(i, j, a, b) arrays of every element in the library's numbering."""
    I, Jj = np.triu_indices(L, 1)
    a, b = np.divmod(np.arange(q * q), q)
    n = len(I)
    return np.repeat(I, q * q), np.repeat(Jj, q * q), np.tile(a, n), np.tile(b, n)


def setup(bm, L, q, M, seed, sweeps=3):
    h, J = synth.planted_contact_model(L, q, seed)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    c = bm.bm_chains_init(m, M, seed + 1)
    bm.bm_gibbs_sweep(m, c, sweeps, 1.0)
    counts = torch.empty((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    return m, c, counts


def params(bm, m):
    h = torch.empty((m.L, m.q), dtype=torch.float32)
    J = torch.empty((m.L, m.L, m.q, m.q), dtype=torch.float32)
    bm.bm_potts_get(m, h, J)
    torch.cuda.synchronize()
    return h.numpy().astype(np.float64), J.numpy().astype(np.float64)


def activity(bm, m):
    a = torch.empty((m.L, m.L, m.q, m.q), dtype=torch.uint8)
    bm.bm_graph_get(m, a)
    return a.numpy()


def assert_same_selection(sel_gpu, sel_orc, score, boundary):
    diff = sel_gpu != sel_orc
    assert sel_gpu.sum() == sel_orc.sum()
    if diff.any():
        assert np.isfinite(boundary), "selections differ at an infinite boundary"
        tol = 1e-12 * max(1.0, abs(boundary))
        far = np.abs(score[diff] - boundary) > tol
        assert not far.any(), (np.flatnonzero(diff)[far][:5], score[diff][far][:5], boundary)


def check_graph(bm, m, act, J):
    assert np.array_equal(act, act.transpose(1, 0, 3, 2))
    assert np.all(J[act == 0] == 0.0)
    L = m.L
    for i in range(L):
        assert not act[i, i].any()
    na, ne = bm.bm_graph_count(m)
    ii, jj, aa, bb = element_index(L, m.q)
    assert ne == len(ii)
    assert na == int(act[ii, jj, aa, bb].sum())


@pytest.mark.parametrize("L,q,M,frac", [(16, 21, 1024, 0.3), (37, 5, 600, 0.1), (64, 21, 2000, 0.02),
                                        (3, 2, 50, 0.5)])
def test_decimation_matches_oracle(bm, orc, L, q, M, frac):
    m, c, counts = setup(bm, L, q, M, 11)
    bm.bm_graph_enable(m, True)
    ne = L * (L - 1) // 2 * q * q
    assert bm.bm_graph_count(m) == (ne, ne)
    ii, jj, aa, bb = element_index(L, q)
    C = counts.cpu().numpy()
    for step in range(2):  # a second step from the decimated graph reuses the selection scratch
        _, J0 = params(bm, m)
        act0 = activity(bm, m)
        n = max(1, int(frac * bm.bm_graph_count(m)[0]))
        removed = bm.bm_graph_decimate(m, counts, M, n)
        assert removed == n
        pij = orc.pair_freqs(C, M, L, q)
        score = orc.decimation_scores(J0, pij, act0)
        J_o, act_o, rem_o = orc.graph_decimate(J0, act0, score, n)
        assert rem_o == n
        act_g = activity(bm, m)
        _, J_g = params(bm, m)
        was = act0[ii, jj, aa, bb] == 1
        gone_g = was & (act_g[ii, jj, aa, bb] == 0)
        gone_o = was & (act_o[ii, jj, aa, bb] == 0)
        assert_same_selection(gone_g, gone_o, score, score[gone_o].max())
        check_graph(bm, m, act_g, J_g)
        same = act_g == act_o
        assert np.array_equal(J_g[same], J_o[same])


@pytest.mark.parametrize("L,q,M,frac", [(16, 21, 1024, 0.05), (37, 5, 600, 0.01), (64, 21, 2000, 0.001)])
def test_activation_matches_oracle(bm, orc, L, q, M, frac):
    m, c, counts = setup(bm, L, q, M, 12)
    X = synth.clustered_msa(3 * M, L, q, 13, n_ancestors=M // 4 + 1)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None, q, 0.05, fi, fij)
    bm.bm_graph_enable(m, False)
    _, J0 = params(bm, m)
    assert not J0.any()
    ne = L * (L - 1) // 2 * q * q
    assert bm.bm_graph_count(m) == (0, ne)
    ii, jj, aa, bb = element_index(L, q)
    C = counts.cpu().numpy()
    fij_h = fij.cpu().numpy().astype(np.float64)
    pij = orc.pair_freqs(C, M, L, q)
    score = orc.activation_scores(fij_h, pij)
    act = activity(bm, m)
    total = 0
    for step in range(2):
        n = max(1, int(frac * ne))
        fresh = bm.bm_graph_activate(m, fij, counts, M, n)
        act_o, fresh_o = orc.graph_activate(act, score, n)
        act_g = activity(bm, m)
        chosen_g = act_g[ii, jj, aa, bb] == 1
        chosen_o = act_o[ii, jj, aa, bb] == 1
        boundary = np.sort(score)[::-1][min(n, ne) - 1]
        assert_same_selection(chosen_g, chosen_o, score, boundary)
        assert fresh == fresh_o
        total += fresh
        act = act_g
    # the same counts and data: the second step selects the same elements, so nothing new
    assert total == min(int(max(1, frac * ne)), ne)
    _, J_g = params(bm, m)
    assert not J_g.any()
    check_graph(bm, m, act, J_g)


def test_masked_update_matches_oracle(bm, orc):
    L, q, M = 24, 21, 1500
    m, c, counts = setup(bm, L, q, M, 14)
    X = synth.clustered_msa(3 * M, L, q, 15, n_ancestors=M // 4 + 1)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None, q, 0.05, fi, fij)
    bm.bm_graph_enable(m, True)
    ne = L * (L - 1) // 2 * q * q
    bm.bm_graph_decimate(m, counts, M, ne // 2)
    h0, J0 = params(bm, m)
    act = activity(bm, m)
    lr = 0.05
    rho, applied = bm.bm_update(m, fi, fij, counts, M, lr, 2.0)
    assert applied
    h_o, J_o = orc.update_masked(h0, J0, fi.cpu().numpy(), fij.cpu().numpy(), counts.cpu().numpy(), M, lr, act)
    h_g, J_g = params(bm, m)
    assert np.all(J_g[act == 0] == 0.0)
    tolJ = 4 * np.spacing(np.abs(J_o).astype(np.float32)) + 1e-7
    assert np.all(np.abs(J_g - J_o) <= tolJ)
    assert np.all(np.abs(h_g - h_o) <= 4 * np.spacing(np.abs(h_o).astype(np.float32)) + 1e-7)
    check_graph(bm, m, act, J_g)


def test_decimation_rounds_keep_the_graph_consistent(bm):
    """A short edDCA run: decimate, then updates with sweeps between them
    (the paper's gsteps), until a density; every round keeps inactive
    couplings at zero through the updates and the sweeps."""
    L, q, M = 40, 21, 2048
    m, c, counts = setup(bm, L, q, M, 16)
    X = synth.clustered_msa(3 * M, L, q, 17, n_ancestors=M // 4 + 1)
    fi = torch.empty((L, q), dtype=torch.float32, device=DEV)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=DEV)
    bm.bm_data_stats(to_dev(X), None, q, 0.05, fi, fij)
    bm.bm_graph_enable(m, True)
    drate, target = 0.2, 0.3
    ne = L * (L - 1) // 2 * q * q
    while bm.bm_graph_count(m)[0] > target * ne:
        na = bm.bm_graph_count(m)[0]
        assert bm.bm_graph_decimate(m, counts, M, int(drate * na)) == int(drate * na)
        for _ in range(3):
            bm.bm_gibbs_sweep(m, c, 2, 1.0)
            bm.bm_chain_stats(c, counts)
            bm.bm_update(m, fi, fij, counts, M, 0.05, 2.0)
        bm.bm_device_status(m)
        _, J = params(bm, m)
        check_graph(bm, m, activity(bm, m), J)
    assert bm.bm_graph_count(m)[0] <= target * ne


def test_decimation_full_size_matches_oracle(bm, orc):
    L, q, M = 256, 21, 10000
    m, c, counts = setup(bm, L, q, M, 18, sweeps=2)
    bm.bm_graph_enable(m, True)
    _, J0 = params(bm, m)
    act0 = activity(bm, m)
    ne = L * (L - 1) // 2 * q * q
    n = ne // 100
    assert bm.bm_graph_decimate(m, counts, M, n) == n
    C = counts.cpu().numpy()
    score = orc.decimation_scores(J0, orc.pair_freqs(C, M, L, q), act0)
    _, act_o, _ = orc.graph_decimate(J0, act0, score, n)
    act_g = activity(bm, m)
    ii, jj, aa, bb = element_index(L, q)
    gone_g = act_g[ii, jj, aa, bb] == 0
    gone_o = act_o[ii, jj, aa, bb] == 0
    assert_same_selection(gone_g, gone_o, score, score[gone_o].max())
    assert bm.bm_graph_count(m)[0] == ne - n


def test_graph_arguments_are_checked(bm):
    L, q, M = 8, 4, 64
    m, c, counts = setup(bm, L, q, M, 19)
    with pytest.raises(bm.BmError):
        bm.bm_graph_decimate(m, counts, M, 1)  # no graph yet
    act = torch.empty((L, L, q, q), dtype=torch.uint8)
    with pytest.raises(bm.BmError):
        bm.bm_graph_get(m, act)
    bm.bm_graph_enable(m, True)
    with pytest.raises(bm.BmError):
        bm.bm_graph_decimate(m, counts, 0, 1)
    with pytest.raises(bm.BmError):
        bm.bm_graph_decimate(m, counts, M, -1)
    ne = L * (L - 1) // 2 * q * q
    assert bm.bm_graph_decimate(m, counts, M, 10 * ne) == ne  # capped at the active count
    assert bm.bm_graph_count(m) == (0, ne)
    assert bm.bm_graph_decimate(m, counts, M, 5) == 0
    bm.bm_graph_disable(m)
    assert bm.bm_graph_count(m) == (ne, ne)
