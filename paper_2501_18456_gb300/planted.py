"""Dense protein-like training workload on data sampled from a planted model.

The paper trains on natural protein families (e.g. PF00072), which are not
available here.  This module builds their stand-in from a planted Potts
model, with the library's own sampler (Sec. 2.1 Gibbs sweeps), so that the
trained model has a generating model to recover:

  * planted model: L = 256, q = 21, h ~ N(0, 1), J ~ N(0, 0.2^2) on a contact
    map of ~3% of the pairs (every |i-j| <= 2 plus random long-range pairs);
    the gap symbol's field h_i(0) of every site is shifted by one constant,
    found by bisection on short pilot runs, so that ~20% of the sampled
    symbols are gaps (Sec. 2.3: natural alignments hold gaps);
  * data MSA: 5,000 ancestors and 50,000 donors, each an independent chain
    after 500 sweeps from a uniform random start; descendant m copies
    ancestor m mod 5,000 and takes a U[2%, 30%] fraction of its sites from
    donor m, so family members exceed 80% identity and the Eq. 7 reweighting
    matters (a few full sweeps would leave only ~10% identity at these
    fields);
  * training (Sec. 3.3): M = 10,000 chains, 10 sweeps per update, lr = 0.01,
    from the independent-site profile model h = log f_i, J = 0, until the
    Pearson criterion reaches 0.95 or 500 iterations.

Only inputs are prepared here; every step of the method runs in the
library's kernels (sampling, weights, frequencies, counts, update).
"""
from __future__ import annotations

import time

import numpy as np
import torch

from . import bmdca, synth, train

L_SITES, Q = 256, 21


def gap_fraction(model: bmdca.Model, n_chains: int, nsweeps: int, seed: int) -> float:
    c = bmdca.bm_chains_init(model, n_chains, seed)
    bmdca.bm_gibbs_sweep(model, c, nsweeps, 1.0)
    s = torch.empty((n_chains, model.L), dtype=torch.uint8, device="cuda")
    bmdca.bm_chains_get(c, s)
    return float((s == 0).float().mean())


def gap_shifted_model(L: int = L_SITES, q: int = Q, seed: int = 2024, target: float = 0.2,
                      pilot_chains: int = 2048, pilot_sweeps: int = 60, iters: int = 14):
    """Planted contact model with h_i(0) shifted by the constant that brings
    the sampled gap fraction to `target` (bisection on pilot runs)."""
    h, J = synth.planted_contact_model(L, q, seed)
    Jd = torch.from_numpy(J).cuda()
    lo, hi = -10.0, 10.0
    shift = 0.0
    for _ in range(iters):
        shift = 0.5 * (lo + hi)
        hs = h.copy()
        hs[:, 0] += shift
        m = bmdca.bm_potts_load(torch.from_numpy(hs).cuda(), Jd)
        g = gap_fraction(m, pilot_chains, pilot_sweeps, seed + 7)
        m.free()
        if g < target:
            lo = shift
        else:
            hi = shift
    h = h.copy()
    h[:, 0] += shift
    return h, J, shift


def sample_chains(model: bmdca.Model, n: int, nsweeps: int, seed: int) -> torch.Tensor:
    c = bmdca.bm_chains_init(model, n, seed)
    bmdca.bm_gibbs_sweep(model, c, nsweeps, 1.0)
    s = torch.empty((n, model.L), dtype=torch.uint8, device="cuda")
    bmdca.bm_chains_get(c, s)
    c.free()
    return s


def planted_msa(model: bmdca.Model, N: int = 50000, n_anc: int = 5000, nsweeps: int = 500,
                seed: int = 2024) -> np.ndarray:
    """Clustered data MSA sampled from the planted model (see module doc)."""
    anc = sample_chains(model, n_anc, nsweeps, seed + 11).cpu().numpy()
    don = sample_chains(model, N, nsweeps, seed + 12).cpu().numpy()
    return synth.cluster_mix(anc, don, seed + 13)


def build(N: int = 50000, n_anc: int = 5000, nsweeps: int = 500, seed: int = 2024, L: int = L_SITES,
          q: int = Q):
    """Planted model (h, J, gap shift) and its data MSA, with the time taken."""
    t0 = time.perf_counter()
    h, J, shift = gap_shifted_model(L, q, seed)
    m = bmdca.bm_potts_load(torch.from_numpy(h).cuda(), torch.from_numpy(J).cuda())
    msa = planted_msa(m, N, n_anc, nsweeps, seed)
    m.free()
    torch.cuda.synchronize()
    return {"h": h, "J": J, "gap_shift": shift, "msa": msa, "seconds": time.perf_counter() - t0}


def train_to_target(msa_d: torch.Tensor, q: int, cfg: train.TrainConfig, stats: train.DataStats | None = None):
    """Profile-initialised training on a device MSA until the Pearson target
    or cfg.max_iters; returns the run's record."""
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    if stats is None:
        stats = train.data_statistics(msa_d, q, cfg)
    h0, J0 = train.profile_init(stats)
    model = bmdca.bm_potts_load(h0, J0)
    chains = bmdca.bm_chains_init(model, cfg.M, cfg.seed)
    hist = train.train(model, chains, stats, cfg)
    torch.cuda.synchronize()
    wall = time.perf_counter() - t0
    rhos = [r["pearson"] for r in hist]
    hit = next((r["iteration"] for r in hist if r["pearson"] >= cfg.target), None)
    out = {"iterations": len(hist), "reached_target": hit is not None, "target": cfg.target,
           "iteration_at_target": hit, "pearson_first": rhos[0], "pearson_last": rhos[-1],
           "pearson_max": max(rhos), "wall_s": wall, "meff": stats.meff,
           "pearson_every_50": [round(rhos[k], 4) for k in range(0, len(rhos), 50)]}
    return out, model, chains
