"""GPU tests of batched sweeps (bm_batch_*): one graph launch sweeps many
models of uneven L and must draw exactly the states of per-model CUDA-core
sweeps (same Philox uniforms, same FP32 summation order)."""
import numpy as np
import pytest
import torch

from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
SHAPES = [(50, 300), (130, 200), (17, 90), (96, 500), (512, 64), (33, 1)]  # (L, M)


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def states(bm, c):
    out = torch.empty((c.M, c.L), dtype=torch.uint8, device=DEV)
    bm.bm_chains_get(c, out)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def build(bm, q=21, seed=0):
    models, chains = [], []
    for k, (L, M) in enumerate(SHAPES):
        h, J = synth.planted_local_model(L, q, seed + k, sigma_h=1.0, sigma_J=0.3)
        m = bm.bm_potts_load(to_dev(h), to_dev(J))
        bm.bm_model_set_engine(m, bm.BM_ENGINE_SIMT)
        models.append(m)
        chains.append(bm.bm_chains_init(m, M, 100 + k))
    return models, chains


@pytest.mark.parametrize("tune", [False, True])
def test_batch_equals_per_model_sweeps(bm, tune):
    models, chains = build(bm)
    ref_m, ref_c = build(bm)
    b = bm.Batch(models, chains)
    if tune:
        b.autotune()
        shp = b.shape()
        assert shp["chains_per_cta"] > 0 and shp["stages"] >= 2
    b.sweep(3, 1.0)
    b.sweep(2, 0.8)
    for m, c in zip(ref_m, ref_c):
        bm.bm_gibbs_sweep(m, c, 3, 1.0)
        bm.bm_gibbs_sweep(m, c, 2, 0.8)
    for m in models:
        bm.bm_device_status(m)
    for c, rc in zip(chains, ref_c):
        assert bm.bm_chains_sweep_counter(c) == 5
        assert np.array_equal(states(bm, c), states(bm, rc))
    b.close()


def test_batch_follows_parameter_updates(bm):
    """An applied bm_update swaps the model's parameter buffers; the next
    batched sweep uses the new ones."""
    models, chains = build(bm, seed=7)
    ref_m, ref_c = build(bm, seed=7)
    b = bm.Batch(models, chains)
    b.sweep(1)
    for m, c in zip(ref_m, ref_c):
        bm.bm_gibbs_sweep(m, c, 1, 1.0)
    q = 21
    for m, rm, c in zip(models, ref_m, chains):
        L = m.L
        fi = torch.full((L, q), 1.0 / q, dtype=torch.float32, device=DEV)
        fij = torch.full((L, L, q, q), 1.0 / q ** 2, dtype=torch.float32, device=DEV)
        counts = torch.zeros((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
        bm.bm_chain_stats(c, counts)
        for mm in (m, rm):
            _, applied = bm.bm_update(mm, fi, fij, counts, c.M, 0.05, 2.0, True)
            assert applied
    b.sweep(2)
    for m, c in zip(ref_m, ref_c):
        bm.bm_gibbs_sweep(m, c, 2, 1.0)
    for c, rc in zip(chains, ref_c):
        assert np.array_equal(states(bm, c), states(bm, rc))
    b.close()


def test_batch_rejects_mixed_alphabets(bm):
    h1, J1 = synth.planted_local_model(10, 21, 1)
    h2, J2 = synth.planted_local_model(10, 5, 2)
    m1, m2 = bm.bm_potts_load(to_dev(h1), to_dev(J1)), bm.bm_potts_load(to_dev(h2), to_dev(J2))
    c1, c2 = bm.bm_chains_init(m1, 10, 1), bm.bm_chains_init(m2, 10, 2)
    with pytest.raises(bm.BmError) as e:
        bm.Batch([m1, m2], [c1, c2])
    assert e.value.code == bm.BM_EINVAL
