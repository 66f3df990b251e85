"""Serving workload: a Poisson stream of sampling, scoring and single-mutant
scan requests over many resident models, run through the library's
continuous-batching server (bm_server_*), with latency percentiles and
sequences/s.

Workload (the serving configuration of the method's use cases: Sec. 4.1
sampling at inverse temperature beta, Sec. 4.3 scoring, Sec. 4.4 mutant
scans):
  * 32 resident models, L ~ U[60, 400], q alternating 21 (proteins) and 5
    (RNA), planted contact-map couplings (synthetic stand-ins for trained
    models);
  * requests in equal proportions: sample n ~ logU[100, 10^4] sequences at
    beta in {0.8, 1.0, 1.2} with U[20, 200] sweeps; score n ~ logU[10^3,
    10^6] sequences; full single-mutant scan of a random wild type;
  * Poisson arrivals at `rate` requests/s for `duration` s.
Sequences counted: sampled n, scored n, and L*q mutants per scan.

This module only builds inputs and drives the server; every computation runs
in the library's kernels.
"""
from __future__ import annotations

import argparse
import json
import threading
import time

import numpy as np
import torch

from . import bmdca, synth


def make_models(count: int = 32, seed: int = 0, device: str = "cuda"):
    rng = np.random.default_rng(seed)
    models = []
    for k in range(count):
        L = int(rng.integers(60, 401))
        q = 21 if k % 2 == 0 else 5
        h, J = synth.planted_contact_model(L, q, seed + k)
        models.append(bmdca.bm_potts_load(torch.from_numpy(h).to(device), torch.from_numpy(J).to(device)))
    return models


def request_stream(models, rate: float, duration: float, seed: int):
    """[(t_arrival, type, model_index, n, nsweeps, beta, request_seed)] of the Poisson stream."""
    rng = np.random.default_rng(seed)
    out, t = [], 0.0
    while True:
        t += rng.exponential(1.0 / rate)
        if t > duration:
            return out
        kind = int(rng.integers(1, 4))
        mi = int(rng.integers(len(models)))
        n, sweeps, beta = 0, 0, 1.0
        if kind == bmdca.BM_REQ_SAMPLE:
            n = int(round(10 ** rng.uniform(2, 4)))
            sweeps = int(rng.integers(20, 201))
            beta = float(rng.choice([0.8, 1.0, 1.2]))
        elif kind == bmdca.BM_REQ_SCORE:
            n = int(round(10 ** rng.uniform(3, 6)))
        out.append((t, kind, mi, n, sweeps, beta, int(rng.integers(1 << 62))))


def run_stream(models, rate: float = 10.0, duration: float = 8.0, seed: int = 1, slots: int = 16,
               budget_bytes: int = 8 << 30, engine: int | None = None, burst: bool = False) -> dict:
    """Runs the request stream through a fresh server; returns its statistics.
    engine: a BM_ENGINE_* value applied to every model before it is served.
    burst: submit every request of the stream at once (arrival times
    ignored), so the figures are those of a saturated server: sequences/s is
    then its capacity rather than the offered load."""
    if engine is not None:
        for m in models:
            bmdca.bm_model_set_engine(m, engine)
    stream = request_stream(models, rate, duration, seed)
    max_n_score = max((r[3] for r in stream if r[1] == bmdca.BM_REQ_SCORE), default=1)
    max_L = max(m.L for m in models)
    # one pinned buffer of symbols < 5 (valid for q = 5 and q = 21) feeds every scoring request
    pool = torch.from_numpy(np.random.default_rng(seed).integers(0, 5, size=max_n_score * max_L,
                                                                 dtype=np.uint8)).pin_memory()
    wts = [torch.from_numpy(synth.random_states(1, m.L, m.q, seed + k)[0]).pin_memory()
           for k, m in enumerate(models)]
    srv = bmdca.Server(budget_bytes, slots)
    ids = [srv.add_model(m) for m in models]
    torch.cuda.synchronize()

    pending, lock, errors = [], threading.Condition(), []
    done_flag = [False]

    def waiter():
        while True:
            with lock:
                while not pending and not done_flag[0]:
                    lock.wait()
                if not pending:
                    return
                rid = pending.pop(0)
            st, _ = srv.wait(rid)
            if st != bmdca.BM_OK:
                errors.append(st)

    th = threading.Thread(target=waiter, daemon=True)
    th.start()
    t0 = time.perf_counter()
    for (ta, kind, mi, n, sweeps, beta, rseed) in stream:
        delay = ta - (time.perf_counter() - t0)
        if delay > 0 and not burst:
            time.sleep(delay)
        m = models[mi]
        if kind == bmdca.BM_REQ_SAMPLE:
            out = torch.empty((n, m.L), dtype=torch.uint8, pin_memory=True)
            rid = srv.submit(kind, ids[mi], out, n=n, nsweeps=sweeps, beta=beta, seed=rseed)
        elif kind == bmdca.BM_REQ_SCORE:
            out = torch.empty(n, dtype=torch.float32, pin_memory=True)
            rid = srv.submit(kind, ids[mi], out, inp=pool[: n * m.L], n=n)
        else:
            out = torch.empty((m.L, m.q), dtype=torch.float32, pin_memory=True)
            rid = srv.submit(kind, ids[mi], out, inp=wts[mi])
        with lock:
            pending.append(rid)
            lock.notify()
    with lock:
        done_flag[0] = True
        lock.notify()
    th.join()
    wall = time.perf_counter() - t0
    st = srv.stats()
    srv.close()
    if errors:
        raise RuntimeError(f"{len(errors)} serving requests failed: {sorted(set(errors))}")
    return {"requests": int(st["completed"]), "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"],
            "mean_ms": st["mean_ms"], "sequences_per_s": st["sequences"] / max(st["span_s"], 1e-9),
            "max_running": int(st["max_running"]), "offered_rate_per_s": None if burst else rate,
            "duration_s": duration, "wall_s": wall, "slots": slots, "budget_bytes": int(budget_bytes),
            "burst": burst, "seed": seed}


def run_seeds(models, rate: float, requests: int, seeds, engine: int | None = None, **kw) -> dict:
    """The Poisson stream for several seeds (about requests/len(seeds)
    requests each): per-seed results and the spread of p50 / p99."""
    per = max(1, requests // len(seeds))
    runs = [run_stream(models, rate, per / rate, sd, engine=engine, **kw) for sd in seeds]
    p50 = [r["p50_ms"] for r in runs]
    p99 = [r["p99_ms"] for r in runs]
    return {"requests": sum(r["requests"] for r in runs), "seeds": list(seeds),
            "p50_ms": float(np.median(p50)), "p50_ms_range": [min(p50), max(p50)],
            "p99_ms": float(np.median(p99)), "p99_ms_range": [min(p99), max(p99)],
            "mean_ms": float(np.mean([r["mean_ms"] for r in runs])),
            "sequences_per_s": float(np.mean([r["sequences_per_s"] for r in runs])),
            "max_running": max(r["max_running"] for r in runs), "offered_rate_per_s": rate,
            "per_seed": [{k: r[k] for k in ("seed", "requests", "p50_ms", "p99_ms", "sequences_per_s")}
                         for r in runs]}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--models", type=int, default=32)
    ap.add_argument("--rate", type=float, default=10.0)
    ap.add_argument("--duration", type=float, default=10.0)
    ap.add_argument("--slots", type=int, default=16)
    ap.add_argument("--budget-gb", type=float, default=8.0)
    ap.add_argument("--seed", type=int, default=1)
    ap.add_argument("--engine", choices=["auto", "simt", "mma"], default="auto")
    a = ap.parse_args()
    models = make_models(a.models, 0)
    eng = {"auto": bmdca.BM_ENGINE_AUTO, "simt": bmdca.BM_ENGINE_SIMT, "mma": bmdca.BM_ENGINE_MMA}[a.engine]
    print(json.dumps(run_stream(models, a.rate, a.duration, a.seed, a.slots, int(a.budget_gb * (1 << 30)), eng)))


if __name__ == "__main__":
    main()
