"""GPU tests of the planted-data workload (the dense protein-like training
set sampled from a planted model by the library's own sweeps): the gap
field shift reaches its target, the clustered MSA is made of model samples,
and its weights and frequencies agree with the FP64 oracle on a subsample
(Eq. 7 bit-exact, Eqs. 3, 8-9 within 1e-6)."""
import numpy as np
import pytest
import torch

import fliplog
from paper_2501_18456_gb300 import bmdca, planted, synth


@pytest.mark.gpu
def test_planted_data_small_shape(bm, orc):
    L, q, N, n_anc = 48, 21, 3000, 300
    data = planted.build(N, n_anc, 100, 7, L, q)
    msa = data["msa"]
    assert msa.shape == (N, L) and msa.max() < q
    assert abs(float((msa == 0).mean()) - 0.2) < 0.03, float((msa == 0).mean())
    # the ancestors and donors are chains of the library's sampler: one more
    # sweep of a few of them is the oracle's teacher-forced draw
    m = bm.bm_potts_load(torch.from_numpy(data["h"]).cuda(), torch.from_numpy(data["J"]).cuda())
    c = bm.bm_chains_init(m, 64, 7 + 11)
    s0 = torch.empty((64, L), dtype=torch.uint8, device="cuda")
    bm.bm_chains_get(c, s0)
    bm.bm_gibbs_sweep(m, c, 1, 1.0)
    s1 = torch.empty_like(s0)
    bm.bm_chains_get(c, s1)
    torch.cuda.synchronize()
    bad, worst = fliplog.verify(orc, data["h"], data["J"], s0.cpu().numpy(), s1.cpu().numpy(), 7 + 11, 0,
                                1.0, 0, "planted sampler")
    assert bad == 0 or worst < fliplog.FLIP_MARGIN
    # clustering: relatives of one ancestor exceed the 80% identity threshold,
    # so reweighting matters
    sub = msa[:1200]
    w_o, meff_o = orc.seq_weights(sub, 0.8)
    assert meff_o < 0.8 * sub.shape[0]
    X = torch.from_numpy(sub).cuda()
    w = torch.empty(sub.shape[0], dtype=torch.float32, device="cuda")
    meff = bm.bm_seq_weights(X, w, 0.8)
    assert np.array_equal(w.cpu().numpy(), w_o.astype(np.float32))
    assert abs(meff - meff_o) <= 1e-9 * meff_o
    fi = torch.empty((L, q), dtype=torch.float32, device="cuda")
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device="cuda")
    bm.bm_data_stats(X, w, q, -1.0, fi, fij)
    fi_o, fij_o = orc.data_stats(sub, w.cpu().numpy().astype(np.float64), q, 1.0 / meff_o)
    assert np.abs(fi.cpu().numpy() - fi_o).max() < 1e-6
    assert np.abs(fij.cpu().numpy() - fij_o).max() < 1e-6


def test_cluster_mix_takes_ancestor_and_donor_symbols():
    anc = synth.random_states(10, 300, 21, 1)
    don = synth.random_states(200, 300, 21, 2)
    X = synth.cluster_mix(anc, don, 3)
    assert X.shape == (200, 300)
    # every row matches one ancestor on ~70-98% of its sites (U[2%, 30%]
    # resampling) and takes the rest from its donor
    ident = (X[:, None, :] == anc[None, :, :]).mean(axis=2).max(axis=1)
    assert ident.min() >= 0.6 and ident.max() <= 1.0
    assert 0.8 < ident.mean() < 0.88
