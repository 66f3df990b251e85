"""Batched training workload: many independent models of uneven length swept
together (bm_batch_*), against one launch per model.

Workload (the batched configuration): 64 models, L ~ U[50, 512], q = 21,
M = 2048 chains each, planted local models (h ~ N(0, 0.5^2), J ~ N(0,
0.05^2) for 1 <= |i-j| <= 3), 10 sweeps per iteration.  Reported: aggregate
site-updates/s of (a) the batched launch in the default (tensor-core) form,
autotuned, (b) the batched launch in the CUDA-core form (graph replay,
autotuned), (c) 64 sequential launches of the plain FP32 CUDA-core sweep,
(d) 64 sequential launches with the default engine (AUTO: the measured
faster form per model).

This module only builds inputs and times the library's entry points.
"""
from __future__ import annotations

import argparse
import json

import numpy as np
import torch

from . import bmdca, synth


def make_batch(count: int = 64, M: int = 2048, q: int = 21, seed: int = 0):
    rng = np.random.default_rng(seed)
    models, chains = [], []
    for k in range(count):
        L = int(rng.integers(50, 513))
        h, J = synth.planted_local_model(L, q, seed + k)
        m = bmdca.bm_potts_load(torch.from_numpy(h).cuda(), torch.from_numpy(J).cuda())
        models.append(m)
        chains.append(bmdca.bm_chains_init(m, M, 1000 + k))
    return models, chains


def _time(fn, reps: int = 3) -> float:
    fn()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    torch.cuda.synchronize()
    return a.elapsed_time(b) / reps


def run(count: int = 64, M: int = 2048, nsweeps: int = 10, seed: int = 0) -> dict:
    models, chains = make_batch(count, M, 21, seed)
    units = float(sum(c.M * c.L for c in chains)) * nsweeps
    batch = bmdca.Batch(models, chains)
    batch.autotune()
    t_batch = _time(lambda: batch.sweep(nsweeps, 1.0))
    shape = batch.shape()
    batch.close()
    for m in models:
        bmdca.bm_model_set_engine(m, bmdca.BM_ENGINE_SIMT)
    batch_cc = bmdca.Batch(models, chains)
    batch_cc.autotune()
    t_batch_cc = _time(lambda: batch_cc.sweep(nsweeps, 1.0))
    shape_cc = batch_cc.shape()
    batch_cc.close()

    def per_model(engine):
        for m in models:
            bmdca.bm_model_set_engine(m, engine)

        def go():
            for m, c in zip(models, chains):
                bmdca.bm_gibbs_sweep(m, c, nsweeps, 1.0)
        return go

    t_plain = _time(per_model(bmdca.BM_ENGINE_SIMT))
    t_auto = _time(per_model(bmdca.BM_ENGINE_AUTO))
    for m in models:
        bmdca.bm_device_status(m)
    return {"models": count, "chains_per_model": M, "nsweeps": nsweeps,
            "L_min": min(c.L for c in chains), "L_max": max(c.L for c in chains),
            "site_updates_per_iter": units,
            "batched": {"ms": t_batch, "site_updates_per_s": units / (t_batch * 1e-3), "form": "tensor cores",
                        **shape},
            "batched_cuda_cores": {"ms": t_batch_cc, "site_updates_per_s": units / (t_batch_cc * 1e-3), **shape_cc},
            "sequential_plain_fp32": {"ms": t_plain, "site_updates_per_s": units / (t_plain * 1e-3)},
            "sequential_default_engine": {"ms": t_auto, "site_updates_per_s": units / (t_auto * 1e-3)},
            "speedup_vs_plain": t_plain / t_batch}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--models", type=int, default=64)
    ap.add_argument("--chains", type=int, default=2048)
    ap.add_argument("--sweeps", type=int, default=10)
    a = ap.parse_args()
    print(json.dumps(run(a.models, a.chains, a.sweeps)))


if __name__ == "__main__":
    main()
