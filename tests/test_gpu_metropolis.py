"""GPU parity of the Metropolis-Hastings sweeps (Sec. 2.1; the --sampler
option) against the FP64 oracle, through the C ABI.

Every site-update is checked teacher-forced: the oracle conditions on the
GPU's new states for j < i and old states for j > i, proposes and decides
with the same Philox uniforms and must agree, except where its acceptance
uniform lies within 1e-5 of the acceptance probability (FP32 against FP64
fields); every such flip is logged."""
import numpy as np
import pytest
import torch

import fliplog
from fliplog import FLIP_MARGIN
from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
ENGINES = ["simt", "mma", "mma_pair", "mma_pair2", "auto"]


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def load_mh(bm, h, J, engine):
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    bm.bm_model_set_engine(m, {"simt": bm.BM_ENGINE_SIMT, "mma": bm.BM_ENGINE_MMA, "mma_pair": bm.BM_ENGINE_MMA_PAIR,
                               "mma_pair2": bm.BM_ENGINE_MMA_PAIR2, "auto": bm.BM_ENGINE_AUTO}[engine])
    bm.bm_model_set_sampler(m, bm.BM_SAMPLER_METROPOLIS)
    return m


def states_of(bm, c):
    out = torch.empty((c.M, c.L), dtype=torch.uint8, device=DEV)
    bm.bm_chains_get(c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def check(orc, h, J, before, after, seed, sweep, beta, where, chain0=0):
    bad, worst = fliplog.verify(orc, h, J, before, after, seed, sweep, beta, chain0, where, metropolis=True)
    assert bad == 0 or worst < FLIP_MARGIN, (bad, worst)
    assert bad <= max(2, before.size // 10000)
    return bad


@pytest.mark.parametrize("M,L,q,beta", [
    (1024, 16, 21, 1.0),
    (333, 37, 5, 1.0),
    (70, 50, 21, 0.8),
    (129, 24, 32, 1.2),
    (17, 2, 1, 1.0),       # one symbol: nothing to propose
    (60, 9, 2, 1.0),       # two symbols: the proposal is the other one
    (300, 130, 8, 1.0),    # tensor-memory operand form of the two-CTA engine
    (400, 160, 21, 1.0),   # shared-memory operand form
])
@pytest.mark.parametrize("engine", ENGINES)
def test_metropolis_sweep_teacher_forced(bm, orc, M, L, q, beta, engine):
    h, J = synth.planted_local_model(L, q, 5, sigma_h=1.0, sigma_J=0.3)
    m = load_mh(bm, h, J, engine)
    c = bm.bm_chains_init(m, M, 21)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, beta)
    bm.bm_device_status(m)
    s1 = states_of(bm, c)
    check(orc, h, J, s0, s1, 21, 0, beta, f"metropolis {engine} L={L} q={q}")
    assert bm.bm_chains_sweep_counter(c) == 1
    if q > 1:
        assert 0.02 < (s1 != s0).mean() < 0.98


@pytest.mark.parametrize("engine", ["simt", "mma_pair", "mma_pair2"])
def test_metropolis_consecutive_and_multi_sweep_calls(bm, orc, engine):
    L, q, M = 40, 21, 300
    h, J = synth.planted_contact_model(L, q, 6, frac=0.2)
    m = load_mh(bm, h, J, engine)
    a = bm.bm_chains_init(m, M, 4)
    b = bm.bm_chains_init(m, M, 4)
    prev = states_of(bm, a)
    for k in range(3):
        bm.bm_gibbs_sweep(m, a, 1, 1.0)
        cur = states_of(bm, a)
        check(orc, h, J, prev, cur, 4, k, 1.0, f"metropolis {engine} consecutive")
        prev = cur
    bm.bm_gibbs_sweep(m, b, 3, 1.0)
    assert np.array_equal(states_of(bm, b), prev)


def test_metropolis_full_size_launch_sampled_chains(bm, orc):
    """L=256, q=21, M=10000 (the training shape), AUTO engine, one sweep;
    sampled chains across clusters and the tail verified."""
    L, q, M = 256, 21, 10000
    h, J = synth.planted_contact_model(L, q, 11)
    m = load_mh(bm, h, J, "auto")
    c = bm.bm_chains_init(m, M, 2024)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    bm.bm_device_status(m)
    s1 = states_of(bm, c)
    sample = sorted(set(np.random.default_rng(0).choice(M, 24, replace=False).tolist()) | {0, 71, 72, 143, 144, M - 1})
    for k in sample:
        check(orc, h, J, s0[k:k + 1], s1[k:k + 1], 2024, 0, 1.0, "metropolis full size", chain0=k)


def test_sampler_switch_and_rejects_unknown(bm, orc):
    L, q, M = 20, 5, 200
    h, J = synth.planted_local_model(L, q, 3, sigma_h=1.0, sigma_J=0.3)
    m = load_mh(bm, h, J, "auto")
    with pytest.raises(bm.BmError) as e:
        bm.bm_model_set_sampler(m, 7)
    assert e.value.code == bm.BM_EINVAL
    bm.bm_model_set_sampler(m, bm.BM_SAMPLER_GIBBS)
    c = bm.bm_chains_init(m, M, 9)
    s0 = states_of(bm, c)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    s1 = states_of(bm, c)
    bad, worst = fliplog.verify(orc, h, J, s0, s1, 9, 0, 1.0, 0, "sampler switched back to gibbs")
    assert bad == 0 or worst < FLIP_MARGIN
