"""GPU parity of bm_fields (local fields of a batch of sequences) against the
FP64 oracle, for the three numerical forms, and the split-precision error
report on the RNA-like shape (L=120, q=5).

Tolerances, relative to S = |h_i(a)| + sum_j |J_ij(a, s_j)| for each output:
  * FP32 CUDA-core sum of L terms:               L * 2^-24 * S
  * fp16 hi + lo (residual <= 2^-22 |J|), FP32:   (2^-22 + L * 2^-24) * S
  * bf16 hi + lo (residual <= 2^-16 |J|), FP32:   (2^-16 + L * 2^-24) * S
plus 1e-30 absolute for all-zero rows.
"""
import json

import numpy as np
import pytest
import torch

from paper_2501_18456_gb300 import synth

pytestmark = pytest.mark.gpu

DEV = "cuda"
FORMS = {"fp32": (0, 0.0), "fp16x2": (1, 2.0 ** -22), "bf16x2": (2, 2.0 ** -16)}


def to_dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def oracle_fields(orc, h, J, S):
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    n, L = S.shape
    q = h.shape[1]
    H = np.empty((n, L, q))
    for k in range(n):
        for i in range(L):
            H[k, i] = orc.fields(h64, J64, S[k], i)
    return H


def abs_scale(h, J, S):
    """|h_i(a)| + sum_j |J_ij(a, s_j)| for every (k, i, a)."""
    L = S.shape[1]
    aJ = np.abs(J.astype(np.float64))
    out = np.empty((S.shape[0],) + h.shape)
    for k in range(S.shape[0]):
        # aJ[:, j, :, s_j] over j has shape (j, i, a): sum over j
        out[k] = np.abs(h) + aJ[:, np.arange(L), :, S[k]].sum(axis=0)
    return out


def gpu_fields(bm, m, S, form):
    n, L = S.shape
    H = torch.full((n, L, m.q), float("nan"), dtype=torch.float32, device=DEV)
    bm.bm_fields(m, to_dev(S), H, form)
    bm.bm_device_status(m)
    torch.cuda.synchronize()
    return H.cpu().numpy().astype(np.float64)


@pytest.mark.parametrize("form", list(FORMS))
@pytest.mark.parametrize("n,L,q", [(100, 16, 21), (300, 37, 5), (50, 24, 32), (257, 61, 4), (3, 2, 1),
                                   (513, 20, 21), (1, 1, 3)])
def test_fields_parity(bm, orc, n, L, q, form):
    h, J = synth.planted_local_model(L, q, 8, sigma_h=1.0, sigma_J=0.3)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    S = synth.random_states(n, L, q, 9)
    code, rep = FORMS[form]
    H = gpu_fields(bm, m, S, code)
    ref = oracle_fields(orc, h, J, S)
    tol = (rep + L * 2.0 ** -24) * abs_scale(h, J, S) + 1e-30
    err = np.abs(H - ref)
    assert np.all(err <= tol), f"max err {err.max():.3e}, worst ratio {(err / tol).max():.2f}"


def test_fields_follow_parameter_updates(bm, orc):
    """The tensor-core forms rebuild their split copy of J after bm_potts_set."""
    L, q, n = 20, 21, 40
    h, J = synth.planted_local_model(L, q, 1, sigma_h=1.0, sigma_J=0.3)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    S = synth.random_states(n, L, q, 2)
    for code, _ in FORMS.values():
        gpu_fields(bm, m, S, code)
    h2, J2 = synth.planted_local_model(L, q, 3, sigma_h=1.0, sigma_J=0.3)
    bm.bm_potts_set(m, to_dev(h2), to_dev(J2))
    ref = oracle_fields(orc, h2, J2, S)
    for form, (code, rep) in FORMS.items():
        tol = (rep + L * 2.0 ** -24) * abs_scale(h2, J2, S) + 1e-30
        assert np.all(np.abs(gpu_fields(bm, m, S, code) - ref) <= tol), form


def test_fields_invalid_symbol_flagged(bm):
    L, q, n = 6, 4, 5
    h, J = synth.planted_local_model(L, q, 4)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    S = synth.random_states(n, L, q, 5)
    S[2, 3] = q + 7
    for code, _ in FORMS.values():
        H = torch.empty((n, L, q), dtype=torch.float32, device=DEV)
        bm.bm_fields(m, to_dev(S), H, code)
        with pytest.raises(bm.BmError) as e:
            bm.bm_device_status(m)
        assert e.value.code == bm.BM_EINVAL
        bm.bm_device_status(m)  # cleared


def test_fields_rejects_bad_form(bm):
    L, q = 4, 3
    h, J = synth.planted_local_model(L, q, 4)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    S = torch.zeros((2, L), dtype=torch.uint8, device=DEV)
    H = torch.empty((2, L, q), dtype=torch.float32, device=DEV)
    with pytest.raises(bm.BmError) as e:
        bm.bm_fields(m, S, H, 7)
    assert e.value.code == bm.BM_EINVAL


def test_split_precision_report_rna_shape(bm, orc):
    """Split-precision report on the RNA-like shape (L=120, q=5, M=20000 chains):
    max |error| of the fields of every form against FP64 (on sampled chains
    after 5 sweeps), and of f_i, f_ij from the chain counts (exact integers)."""
    L, q, M = 120, 5, 20000
    h, J = synth.planted_contact_model(L, q, 11)
    m = bm.bm_potts_load(to_dev(h), to_dev(J))
    c = bm.bm_chains_init(m, M, 21)
    bm.bm_gibbs_sweep(m, c, 5, 1.0)
    bm.bm_device_status(m)
    S_all = torch.empty((M, L), dtype=torch.uint8, device=DEV)
    bm.bm_chains_get(c, S_all)
    torch.cuda.synchronize()
    S_all = S_all.cpu().numpy()
    sample = S_all[np.random.default_rng(0).choice(M, 300, replace=False)]
    ref = oracle_fields(orc, h, J, sample)
    scale = abs_scale(h, J, sample)
    report = {"shape": {"L": L, "q": q, "M": M}, "fields_max_abs_err": {}, "fields_max_rel_err": {}}
    for form, (code, rep) in FORMS.items():
        err = np.abs(gpu_fields(bm, m, sample, code) - ref)
        report["fields_max_abs_err"][form] = float(err.max())
        report["fields_max_rel_err"][form] = float((err / scale).max())
        assert np.all(err <= (rep + L * 2.0 ** -24) * scale + 1e-30), form
    counts = torch.empty((bm.n_blocks(L), q, q), dtype=torch.int32, device=DEV)
    bm.bm_chain_stats(c, counts)
    bm.bm_chains_device_status(c)
    C = counts.cpu().numpy().astype(np.float64)
    Cref = orc.chain_stats(S_all, q).astype(np.float64)
    report["f_ij_max_abs_err"] = float(np.abs(C - Cref).max() / M)
    diag = [orc.block_index(L, i, i) for i in range(L)]
    report["f_i_max_abs_err"] = float(max(np.abs(np.diag(C[d]) - np.diag(Cref[d])).max() for d in diag) / M)
    assert report["f_ij_max_abs_err"] == 0.0 and report["f_i_max_abs_err"] == 0.0
    print("split-precision report:", json.dumps(report))
