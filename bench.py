"""Benchmark of the bmDCA hot path on one GB300 (or N replicas under torchrun).

Workload (dense protein-like bmDCA): planted contact-map Potts model L=256,
q=21 (h ~ N(0,1), J ~ N(0, 0.2^2) on ~3% of pairs), synthetic clustered MSA
N=50,000 (~20% gaps, 5,000 ancestors x 10), reweighted at 80% identity,
M=10,000 persistent chains, 10 sweeps per iteration, lr = 0.01.

One timed step = one training iteration = 10 Gibbs sweeps over all chains +
chain pair counts + the update with its Pearson check (the Pearson scalar
is read back every step, as the stopping rule needs it).  Preprocessing
(weights, data frequencies, chain init) runs once and is timed separately;
energy scoring and mutant scans are serving calls, timed separately too.

Metric: Gibbs site-updates/s = M * L * nsweeps / step time.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has here) on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time
from pathlib import Path

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

L_SITES, Q, M_CHAINS, N_SEQS, NSWEEPS, LR, SEED = 256, 21, 10000, 50000, 10, 0.01, 2024
WORKLOAD = "bmDCA dense protein-like: L=256 q=21 M=10000 chains, 10 sweeps/iter, MSA N=50000"
METRIC = "Gibbs site-updates/s (L=256,q=21,M=10k)"
UNIT = "site-updates/s"
# DRAM bytes per 10-sweep launch of each sweep kernel (dram__bytes_read.sum +
# dram__bytes_write.sum from one ncu capture of this bench's launch); None
# whenever the kernel has changed since it was captured.
TRAFFIC_GIBBS = {"k_gibbs_pair": 1192470272 + 3264256}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-chains", type=int, default=0,
                    help="chains in the oracle sample (0: sized for ~15 s)")
    ap.add_argument("--no-serve", action="store_true", help="skip the serving-latency leg")
    ap.add_argument("--no-batched", action="store_true", help="skip the batched-models leg")
    ap.add_argument("--serve-seconds", type=float, default=8.0)
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


# ----------------------------------------------------------------- clocks

class ClockSampler:
    """nvidia-smi SM clocks / throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.idx = gpu_index
        self.proc = None
        self.file = None

    def start(self):
        try:
            self.file = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.idx}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=self.file, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.file.flush()
        rows = []
        with open(self.file.name) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.file.name)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in rows for k in range(4) if r[5 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons, "samples": len(rows)}


# ----------------------------------------------------------------- CPU oracle legs

def oracle_sample(n_chains: int, nsweeps: int = 1):
    """Time the oracle's Gibbs sweep on n_chains chains of the workload."""
    import oracle
    from paper_2501_18456_gb300 import synth
    oracle.build()
    h, J = synth.planted_contact_model(L_SITES, Q, SEED)
    s0 = oracle.chains_init(n_chains, L_SITES, Q, SEED)
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    t0 = time.perf_counter()
    oracle.gibbs(h64, J64, s0, SEED, 0, nsweeps)
    dt = time.perf_counter() - t0
    return n_chains * L_SITES * nsweeps / dt, dt


def calibrate_oracle_chains(target_s: float) -> int:
    rate, _ = oracle_sample(8)
    return max(8, int(rate * target_s / L_SITES))


def run_reference(args, rank):
    if rank != 0:
        return
    n = args.cpu_chains or calibrate_oracle_chains(1.5)
    for _ in range(args.warmup):
        oracle_sample(max(8, n // 4))
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_sample(n)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    sample = f"oracle Gibbs sweep on {n} of the {M_CHAINS} chains per step (FP64 C, 1 thread)"
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm

def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2501_18456_gb300 import _build, bmdca, synth, train

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    def barrier():
        if world > 1:
            dist.barrier()

    # ---- inputs (seeded; each rank runs its own replica with its own seed)
    seed = SEED + rank
    h, J = synth.planted_contact_model(L_SITES, Q, SEED)
    msa = synth.clustered_msa(N_SEQS, L_SITES, Q, SEED, n_ancestors=N_SEQS // 10)
    msa_d = torch.from_numpy(msa).to(dev)
    model = bmdca.bm_potts_load(torch.from_numpy(h).to(dev), torch.from_numpy(J).to(dev))
    st = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1):
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    rows = {}
    cfg = train.TrainConfig(M=M_CHAINS, nsweeps=NSWEEPS, lr=LR, seed=seed)
    w = torch.empty(N_SEQS, dtype=torch.float32, device=dev)
    meff_box = {}
    rows["seq_weights_ms"] = timed(lambda: meff_box.setdefault("m", bmdca.bm_seq_weights(msa_d, w, 0.8)))
    fi = torch.empty((L_SITES, Q), dtype=torch.float32, device=dev)
    fij = torch.empty((L_SITES, L_SITES, Q, Q), dtype=torch.float32, device=dev)
    rows["data_stats_ms"] = timed(lambda: bmdca.bm_data_stats(msa_d, w, Q, -1.0, fi, fij))
    chains_box = {}
    rows["chains_init_ms"] = timed(lambda: chains_box.setdefault("c", bmdca.bm_chains_init(model, M_CHAINS, seed)))
    chains = chains_box["c"]
    counts = torch.empty((bmdca.n_blocks(L_SITES), Q, Q), dtype=torch.int32, device=dev)

    # L2 flush buffer (larger than the 129 MB L2)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    gibbs_ms = []

    def step(record=False):
        if record:
            a, b = ev(), ev()
            a.record(st)
        bmdca.bm_gibbs_sweep(model, chains, NSWEEPS, 1.0)
        if record:
            b.record(st)
            gibbs_ms.append((a, b))
        bmdca.bm_chain_stats(chains, counts)
        rho, applied = bmdca.bm_update(model, fi, fij, counts, M_CHAINS, LR, 2.0, True)
        return rho

    def measure(engine, steps, sample_clocks=False):
        """W warm-up steps, then `steps` timed steps (L2 flushed before each)."""
        bmdca.bm_model_set_engine(model, engine)
        gibbs_ms.clear()
        for _ in range(args.warmup):
            flush.zero_()
            step()
        torch.cuda.synchronize()
        clocks = ClockSampler(local) if sample_clocks else None
        barrier()
        torch.cuda.synchronize()
        if clocks:
            clocks.start()
        t_wall0 = time.perf_counter()
        step_events = []
        rho = None
        for _ in range(steps):
            flush.zero_()
            a, b = ev(), ev()
            a.record(st)
            rho = step(record=True)
            b.record(st)
            step_events.append((a, b))
        torch.cuda.synchronize()
        t_wall = time.perf_counter() - t_wall0
        barrier()
        clk = clocks.stop() if clocks else None
        ms_s = float(np.mean([a.elapsed_time(b) for a, b in step_events]))
        ms_g = float(np.mean([a.elapsed_time(b) for a, b in gibbs_ms]))
        if world > 1:
            t = torch.tensor([ms_s, ms_g], dtype=torch.float64, device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            ms_s, ms_g = float(t[0]), float(t[1])
        bmdca.bm_device_status(model)
        return ms_s, ms_g, rho, clk, t_wall

    site_updates_per_step = M_CHAINS * L_SITES * NSWEEPS
    # plain FP32 path (CUDA-core gather) on the same workload, for comparison
    ms_plain, ms_plain_gibbs, _, _, _ = measure(bmdca.BM_ENGINE_SIMT, max(2, args.steps // 2))
    # headline: the library's default engine (tensor cores)
    ms_step, ms_gibbs, rho, clk, t_wall = measure(bmdca.BM_ENGINE_AUTO, args.steps, sample_clocks=True)
    value = world * site_updates_per_step / (ms_step * 1e-3)

    # ---- per-row timings of the other steps (one step's worth each)
    rows["gibbs_sweep_ms_per_sweep"] = ms_gibbs / NSWEEPS
    rows["chain_stats_ms"] = timed(lambda: bmdca.bm_chain_stats(chains, counts), 5)
    rows["update_pearson_ms"] = timed(lambda: bmdca.bm_update(model, fi, fij, counts, M_CHAINS, LR, 2.0, True), 5)
    n_score = 100000
    seqs = torch.from_numpy(synth.random_states(n_score, L_SITES, Q, 5)).to(dev)
    E = torch.empty(n_score, dtype=torch.float32, device=dev)
    rows["energy_score_ms_1e5_seqs"] = timed(lambda: bmdca.bm_energy_score(model, seqs, E), 2)
    dE = torch.empty((L_SITES, Q), dtype=torch.float32, device=dev)
    wt = msa_d[0].contiguous()
    rows["mutant_scan_ms"] = timed(lambda: bmdca.bm_mutant_scan(model, wt, dE), 5)

    # ---- end to end through the public API with host buffers
    h_pin = torch.from_numpy(h).pin_memory()
    J_pin = torch.from_numpy(J).pin_memory()
    s_pin = torch.empty((M_CHAINS, L_SITES), dtype=torch.uint8).pin_memory()
    bmdca.bm_chains_get(chains, s_pin)
    s_out = torch.empty_like(s_pin).pin_memory()
    torch.cuda.synchronize()

    def e2e_step():
        bmdca.bm_potts_set(model, h_pin, J_pin)
        bmdca.bm_chains_set(chains, s_pin)
        r = step()
        bmdca.bm_chains_get(chains, s_out)
        return r

    for _ in range(max(1, args.warmup)):
        e2e_step()
    torch.cuda.synchronize()
    a, b = ev(), ev()
    a.record(st)
    for _ in range(args.steps):
        e2e_step()
    b.record(st)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / args.steps
    h2d = h_pin.numel() * 4 + J_pin.numel() * 4 + s_pin.numel()
    d2h = s_out.numel() + 8

    # ---- roofline of the dominant kernel: the tensor-core Gibbs sweep.
    # Algorithmic work per launch: the one-hot x J contraction of every site
    # block, 2*M*(Lq)^2 flops per sweep, done twice (fp16 hi and lo parts of J).
    peaks, peak_src = {}, "fallback 1700 TFLOP/s bf16 sustained"
    try:
        peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
        peak_src = "measured bf16_tflops_sustained (MEASURED_PEAKS.json)"
    except (OSError, ValueError):
        pass
    peak_tf = float(peaks.get("bf16_tflops_sustained", 1700.0))
    Qd = float(L_SITES * Q)
    flops_per_launch = 2.0 * 2.0 * M_CHAINS * Qd * Qd * NSWEEPS
    achieved = flops_per_launch / (ms_gibbs * 1e-3) / 1e12
    bmdca.bm_model_set_engine(model, bmdca.BM_ENGINE_AUTO)
    form = bmdca.bm_model_sweep_engine(model, M_CHAINS)
    kname = {bmdca.BM_ENGINE_MMA_PAIR: "k_gibbs_pair", bmdca.BM_ENGINE_MMA: "k_gibbs_mma"}.get(form, "k_gibbs_staged")
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": TRAFFIC_GIBBS.get(kname),
                "kernel": kname,
                "note": "achieved = 2 passes (fp16 hi, lo) x 2*M*(L*q)^2 flops per sweep x sweeps per "
                        "launch / CUDA-event launch time; peak: " + peak_src +
                        "; fp16 and bf16 share the dense rate"}

    # ---- roofline of the chain counts (the other tensor-core row of the step):
    # one-hot X^T X over the upper block triangle, 2*M*(L(L+1)/2)*q^2 flops,
    # FP8 operands; peak = the measured bf16 rate x 2 (nominal fp8/bf16 ratio).
    cs_flops = 2.0 * M_CHAINS * (L_SITES * (L_SITES + 1) / 2) * Q * Q
    cs_ach = cs_flops / (rows["chain_stats_ms"] * 1e-3) / 1e12
    roofline_counts = {"bound": "tensor", "achieved": cs_ach, "peak": 2 * peak_tf, "unit": "TFLOP/s",
                       "frac": cs_ach / (2 * peak_tf), "kernel": "k_onehot_t + k_counts_tc",
                       "note": "achieved = 2*M*(L(L+1)/2)*q^2 flops / CUDA-event time of bm_chain_stats "
                               "(one-hot build included); peak: fp8 = 2 x " + peak_src}

    # ---- serving: Poisson stream of sample / score / mutant-scan requests over
    # 32 resident models through the continuous-batching server (rank 0), with
    # the tensor-core engine (default) and with plain FP32 sampling.
    serve = None
    if rank == 0 and not args.no_serve:
        from paper_2501_18456_gb300 import serving
        smodels = serving.make_models(32, 0)
        tc = serving.run_stream(smodels, 10.0, args.serve_seconds, 1, engine=bmdca.BM_ENGINE_AUTO)
        plain = serving.run_stream(smodels, 10.0, args.serve_seconds, 1, engine=bmdca.BM_ENGINE_SIMT)
        serve = {"workload": "32 resident models (L U[60,400], q 21/5), Poisson 10 req/s: sample "
                             "logU[1e2,1e4] seqs x U[20,200] sweeps at beta {0.8,1,1.2}, score "
                             "logU[1e3,1e6] seqs, single-mutant scans",
                 "p50_ms": tc["p50_ms"], "p99_ms": tc["p99_ms"], "mean_ms": tc["mean_ms"],
                 "sequences_per_s": tc["sequences_per_s"], "requests": tc["requests"],
                 "max_running": tc["max_running"],
                 "plain_fp32": {k: plain[k] for k in ("p50_ms", "p99_ms", "mean_ms", "sequences_per_s",
                                                      "requests", "max_running")}}
        del smodels
        torch.cuda.empty_cache()

    # ---- batched: 64 models of uneven L swept in one graph launch (rank 0),
    # against 64 sequential per-model launches.
    batched = None
    if rank == 0 and not args.no_batched:
        from paper_2501_18456_gb300 import batched as batched_mod
        batched = batched_mod.run(64, 2048, 10, 0)
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and not args.no_cpu_baseline:
        n = args.cpu_chains or calibrate_oracle_chains(15.0)
        r, dt = oracle_sample(n)
        cpu = {"value": r, "unit": UNIT, "cores": 1, "kind": "oracle",
               "sample": f"oracle Gibbs sweep on {n} of the {M_CHAINS} chains, 1 sweep, "
                         f"{dt:.1f} s, FP64 C, 1 thread"}

    # Kernels launched per step: J tensor-core layout rebuild (the previous
    # update changed J) + Gibbs sweep, chain counts (one-hot build + product),
    # update (pairs, fields, Pearson partial sum) + gather-layout rebuild.
    launches_per_step = 2 + 2 + 3 + 1
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
                "data": "synthetic",
                "config": {"workload": WORKLOAD, "L": L_SITES, "q": Q, "M": M_CHAINS,
                           "N": N_SEQS, "nsweeps": NSWEEPS, "lr": LR, "meff": meff_box.get("m"),
                           "engine": "tensor cores (tcgen05, fp16 hi+lo J, f32 accumulate)",
                           "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world}", "pearson_last": rho},
                "plain_fp32": {"value": world * site_updates_per_step / (ms_plain * 1e-3), "unit": UNIT,
                               "ms_per_step": ms_plain, "gibbs_ms_per_sweep": ms_plain_gibbs / NSWEEPS,
                               "engine": "CUDA-core FP32 gather (k_gibbs_staged)",
                               "speedup_of_value": ms_plain / ms_step},
                "roofline": roofline, "roofline_chain_stats": roofline_counts, "cpu_baseline": cpu,
                "e2e": {"value": world * site_updates_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clk, "rows_ms": rows, "serve": serve, "batched": batched, "wall_s_timed": t_wall}
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank)
        return
    run_ours(args, rank, world, local)


if __name__ == "__main__":
    main()
