"""Host-side bmDCA training loop (adabmDCA 2.0, Sec. 2.1 and Sec. 3).

Every step runs in libbmdca.so kernels; this module only sequences the C
entry points:

  preprocessing (once):  bm_seq_weights (Eq. 7) -> bm_data_stats (Eqs. 3, 8-9)
  per iteration t:       bm_gibbs_sweep x nsweeps (PCD chains, theta_t)
                         -> bm_chain_stats -> bm_update: Pearson of the
                         connected correlations of theta_t's chains; stop if
                         rho >= target (theta_t kept), else Eq. 5 -> theta_{t+1}

Sparse models (Sec. 2.2): `eadca` grows the coupling graph from empty and
`eddca` prunes a trained model's graph, both through the bm_graph_* calls.

Initial parameters are the caller's choice.  `profile_init` offers the
independent-site model h_i(a) = log f_i(a), J = 0 (finite thanks to the
pseudocount); it is a one-off element-wise log of L*q numbers done with torch
before training starts, outside the hot path.
"""
from __future__ import annotations

import dataclasses
import time

import torch

from . import bmdca


@dataclasses.dataclass
class TrainConfig:
    M: int = 10000          # persistent chains (paper default, Sec. 3.3)
    nsweeps: int = 10       # sweeps per update (Sec. 3.3)
    lr: float = 0.01        # learning rate; set explicitly by every workload
    max_iters: int = 500
    target: float = 0.95    # Pearson target (Sec. 2.1)
    seed: int = 0
    seqid: float = 0.8      # identity threshold of Eq. 7
    pseudocount: float = -1.0  # < 0: 1 / M_eff (Sec. 3.3)
    reweight: bool = True


@dataclasses.dataclass
class DataStats:
    fi: torch.Tensor
    fij: torch.Tensor
    meff: float
    weights: torch.Tensor | None


def data_statistics(msa: torch.Tensor, q: int, cfg: TrainConfig, stream=None) -> DataStats:
    """Weights (if enabled) and pseudocounted frequencies of a device MSA."""
    N, L = msa.shape
    w = None
    meff = float(N)
    if cfg.reweight:
        w = torch.empty(N, dtype=torch.float32, device=msa.device)
        meff = bmdca.bm_seq_weights(msa, w, cfg.seqid, True, stream)
    fi = torch.empty((L, q), dtype=torch.float32, device=msa.device)
    fij = torch.empty((L, L, q, q), dtype=torch.float32, device=msa.device)
    bmdca.bm_data_stats(msa, w, q, cfg.pseudocount, fi, fij, stream)
    return DataStats(fi, fij, meff, w)


def profile_init(stats: DataStats):
    """Initial model: h_i(a) = log f_i(a), J = 0 (device tensors)."""
    L, q = stats.fi.shape
    h = torch.log(stats.fi)
    J = torch.zeros((L, L, q, q), dtype=torch.float32, device=stats.fi.device)
    return h, J


def train(model: bmdca.Model, chains: bmdca.Chains, stats: DataStats, cfg: TrainConfig,
          log=None, stream=None):
    """Run up to cfg.max_iters iterations; returns the list of per-iteration records."""
    L, q = model.L, model.q
    counts = torch.empty((bmdca.n_blocks(L), q, q), dtype=torch.int32, device=stats.fi.device)
    history = []
    for it in range(cfg.max_iters):
        t0 = time.perf_counter()
        bmdca.bm_gibbs_sweep(model, chains, cfg.nsweeps, 1.0, stream)
        bmdca.bm_chain_stats(chains, counts, stream)
        rho, applied = bmdca.bm_update(model, stats.fi, stats.fij, counts, chains.M, cfg.lr,
                                       cfg.target, True, stream)
        rec = {"iteration": it, "pearson": rho, "applied": applied,
               "seconds": time.perf_counter() - t0}
        history.append(rec)
        if log is not None:
            log(rec)
        if not applied:
            break
    return history


# ---------------------------------------------------------------- sparse models (Sec. 2.2)

def eadca(model: bmdca.Model, chains: bmdca.Chains, stats: DataStats, cfg: TrainConfig,
          factivate: float = 0.001, gsteps: int = 10, max_graph_steps: int = 1000, log=None, stream=None):
    """Element activation DCA (Sec. 2.2, "Element activation DCA").

    Starts from an empty graph (couplings zero; the fields are the caller's,
    e.g. `profile_init`).  Each graph step makes active the
    floor(factivate * inactive) elements whose model pair frequency is
    farthest from the data's, then applies `gsteps` updates (Eq. 5, cfg.lr)
    with cfg.nsweeps sweeps before each.  Stops once the Pearson coefficient
    of the statistics reaches cfg.target.  Returns per-graph-step records."""
    L, q = model.L, model.q
    counts = torch.empty((bmdca.n_blocks(L), q, q), dtype=torch.int32, device=stats.fi.device)
    bmdca.bm_graph_enable(model, False, stream)
    history = []
    for g in range(max_graph_steps):
        t0 = time.perf_counter()
        bmdca.bm_gibbs_sweep(model, chains, cfg.nsweeps, 1.0, stream)
        bmdca.bm_chain_stats(chains, counts, stream)
        na, ne = bmdca.bm_graph_count(model)
        fresh = bmdca.bm_graph_activate(model, stats.fij, counts, chains.M, int(factivate * (ne - na)), stream)
        rho = None
        for _ in range(gsteps):
            bmdca.bm_gibbs_sweep(model, chains, cfg.nsweeps, 1.0, stream)
            bmdca.bm_chain_stats(chains, counts, stream)
            rho, applied = bmdca.bm_update(model, stats.fi, stats.fij, counts, chains.M, cfg.lr,
                                           cfg.target, True, stream)
            if not applied:
                break
        na, ne = bmdca.bm_graph_count(model)
        rec = {"graph_step": g, "activated": fresh, "density": na / ne, "pearson": rho,
               "seconds": time.perf_counter() - t0}
        history.append(rec)
        if log is not None:
            log(rec)
        if rho is not None and rho >= cfg.target:
            break
    return history


def eddca(model: bmdca.Model, chains: bmdca.Chains, stats: DataStats, cfg: TrainConfig,
          density: float = 0.02, drate: float = 0.01, gsteps: int = 10, max_rounds: int = 10000,
          log=None, stream=None):
    """Element decimation DCA (Sec. 2.2, "Element decimation DCA").

    Starts from the model as trained (a fully connected graph) and repeats
    until the graph's density is at most `density`: bring the model to the
    Pearson target cfg.target with updates in groups of `gsteps` (cfg.nsweeps
    sweeps before each; at most `max_rounds` groups in total), then remove
    floor(drate * active) elements, those whose removal perturbs the model
    least.  Returns per-decimation records."""
    L, q = model.L, model.q
    counts = torch.empty((bmdca.n_blocks(L), q, q), dtype=torch.int32, device=stats.fi.device)
    bmdca.bm_graph_enable(model, True, stream)
    history = []
    rounds = 0
    while True:
        t0 = time.perf_counter()
        rho = None
        while rounds < max_rounds:  # convergence on the current graph
            rounds += 1
            for _ in range(gsteps):
                bmdca.bm_gibbs_sweep(model, chains, cfg.nsweeps, 1.0, stream)
                bmdca.bm_chain_stats(chains, counts, stream)
                rho, applied = bmdca.bm_update(model, stats.fi, stats.fij, counts, chains.M, cfg.lr,
                                               cfg.target, True, stream)
                if not applied:
                    break
            if rho is not None and rho >= cfg.target:
                break
        na, ne = bmdca.bm_graph_count(model)
        if na <= density * ne or rounds >= max_rounds:
            break
        bmdca.bm_gibbs_sweep(model, chains, cfg.nsweeps, 1.0, stream)
        bmdca.bm_chain_stats(chains, counts, stream)
        removed = bmdca.bm_graph_decimate(model, counts, chains.M, max(1, int(drate * na)), stream)
        na, ne = bmdca.bm_graph_count(model)
        rec = {"removed": removed, "density": na / ne, "pearson_before": rho,
               "seconds": time.perf_counter() - t0}
        history.append(rec)
        if log is not None:
            log(rec)
    return history
