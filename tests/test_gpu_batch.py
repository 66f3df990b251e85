"""GPU tests of batched sweeps (bm_batch_*): one graph launch sweeps many
models of uneven L and must draw exactly the states of per-model CUDA-core
sweeps (same Philox uniforms, same FP32 summation order)."""
import numpy as np
import pytest
import torch

import fliplog
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


# ---------------------------------------------------------------- tensor-core form

TC_SHAPES = [(256, 700), (37, 300), (512, 500), (90, 1), (150, 2048), (21, 64)]  # (L, M)


def build_tc(bm, seed=0, engine=None, q=21):
    models, chains = [], []
    for k, (L, M) in enumerate(TC_SHAPES):
        h, J = synth.planted_local_model(L, q, seed + k, sigma_h=1.0, sigma_J=0.3)
        m = bm.bm_potts_load(to_dev(h), to_dev(J))
        if engine is not None:
            bm.bm_model_set_engine(m, engine)
        models.append((m, h, J))
        chains.append(bm.bm_chains_init(m, M, 200 + k))
    return models, chains


@pytest.mark.parametrize("q", [21, 5])
def test_tensor_core_batch_matches_oracle_and_per_model_sweeps(bm, orc, q):
    """A batch of models with default engines runs the two-CTA form over
    (model, tile) clusters: every sampled chain's sweep is the oracle's
    teacher-forced draw, and further sweeps equal per-model two-CTA sweeps
    of the same chains (protein and RNA alphabets)."""
    mh, chains = build_tc(bm, q=q)
    models = [m for m, _, _ in mh]
    b = bm.Batch(models, chains)
    shp = b.shape()
    assert shp["chains_per_cta"] >= 96 and shp["ctas"] % 2 == 0, shp
    before = [states(bm, c) for c in chains]
    b.sweep(1, 1.0)
    after = [states(bm, c) for c in chains]
    rng = np.random.default_rng(4)
    for (m, h, J), c, s0, s1 in zip(mh, chains, before, after):
        bm.bm_device_status(m)
        assert bm.bm_chains_sweep_counter(c) == 1
        pick = sorted(set(rng.choice(c.M, min(c.M, 12), replace=False).tolist()) | {c.M - 1})
        for k in pick:
            bad, worst = fliplog.verify(orc, h, J, s0[k:k + 1], s1[k:k + 1],
                                        200 + TC_SHAPES.index((m.L, c.M)), 0, 1.0, k, f"batch L={m.L}")
            assert bad == 0 or worst < 1e-5, (m.L, k, bad, worst)
    # continue: batch vs the same chains swept per model
    ref_mh, ref_c = build_tc(bm, engine=bm.BM_ENGINE_MMA_PAIR, q=q)
    for (m, _, _), c, s in zip(ref_mh, ref_c, after):
        bm.bm_chains_set(c, to_dev(s))
        bm.bm_chains_set_sweep_counter(c, 1)
    b.sweep(2, 0.9)
    for (m, _, _), c in zip(ref_mh, ref_c):
        bm.bm_gibbs_sweep(m, c, 2, 0.9)
    for c, rc in zip(chains, ref_c):
        assert np.array_equal(states(bm, c), states(bm, rc))
    b.close()


def test_tensor_core_batch_autotune_and_updates(bm):
    """Autotuning leaves the chains where they were; after an applied update
    the next batched sweep uses the new parameters (its split layouts are
    rebuilt), matching per-model sweeps."""
    mh, chains = build_tc(bm, seed=9)
    models = [m for m, _, _ in mh]
    ref_mh, ref_c = build_tc(bm, seed=9, engine=bm.BM_ENGINE_MMA_PAIR)
    b = bm.Batch(models, chains)
    s0 = [states(bm, c) for c in chains]
    b.autotune()
    for c, s in zip(chains, s0):
        assert np.array_equal(states(bm, c), s) and bm.bm_chains_sweep_counter(c) == 0
    b.sweep(1)
    for (m, _, _), c in zip(ref_mh, ref_c):
        bm.bm_gibbs_sweep(m, c, 1, 1.0)
    q = 21
    for (m, _, _), (rm, _, _), c in zip(mh, ref_mh, chains):
        L = m.L
        fi = torch.full((L, q), 1.0 / q, dtype=torch.float32, device=DEV)
        fij = torch.full((L, L, q, q), 1.0 / q ** 2, dtype=torch.float32, device=DEV)
        counts = torch.zeros((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
        bm.bm_chain_stats(c, counts)
        for mm in (m, rm):
            _, applied = bm.bm_update(mm, fi, fij, counts, c.M, 0.05, 2.0, True)
            assert applied
    b.sweep(2)
    for (m, _, _), c in zip(ref_mh, ref_c):
        bm.bm_gibbs_sweep(m, c, 2, 1.0)
    for c, rc in zip(chains, ref_c):
        assert np.array_equal(states(bm, c), states(bm, rc))
    b.close()
