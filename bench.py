"""Benchmark of the bmDCA hot path on one GB300 (or N replicas under torchrun).

Workload (dense protein-like bmDCA, Sec. 3.3 defaults): a planted
contact-map Potts model L=256, q=21 (h ~ N(0,1) with the gap field shifted
so ~20% of sampled symbols are gaps, J ~ N(0, 0.2^2) on ~3% of pairs); its
data MSA of N=50,000 sequences is sampled from it by the library's own Gibbs
sweeps (5,000 ancestor clusters, reweighted at 80% identity); training from
the profile model h = log f_i, J = 0 with M=10,000 persistent chains, 10
sweeps per iteration, lr = 0.01.

One timed step = one training iteration = 10 Gibbs sweeps over all chains +
chain pair counts + the update with its Pearson check (the Pearson scalar
is read back every step, as the stopping rule needs it).  Preprocessing
(weights, data frequencies, chain init) runs once and is timed separately;
energy scoring and mutant scans are serving calls, timed separately too.
A separate run trains from the profile model to the Pearson target.

Metric: Gibbs site-updates/s = M * L * nsweeps / step time.

Other legs: the split-precision RNA-like shape (L=120, q=5, M=20,000), 64
batched models of uneven L, and the serving stream; each against the plain
FP32 CUDA-core path on the same GPU.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the only reference this method
has here) on a bounded sample of the same workload, on all host cores.
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
# DRAM bytes per 10-sweep launch of each sweep kernel: dram__bytes_read.sum +
# dram__bytes_write.sum of one ncu capture of a one-sweep launch at this
# shape, times the 10 sweeps of the bench's launch (the couplings are read
# once per sweep, so the traffic grows in proportion); absent whenever the
# kernel has changed since it was captured.
TRAFFIC_GIBBS = {"k_gibbs_pair": 10 * (122337536 + 3695872)}


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
    ap.add_argument("--no-split", action="store_true", help="skip the split-precision leg")
    ap.add_argument("--no-train", action="store_true", help="skip the training-to-target run")
    ap.add_argument("--no-sparse", action="store_true", help="skip the sparse-graph (edDCA / eaDCA) leg")
    ap.add_argument("--serve-requests", type=int, default=1000,
                    help="requests per engine in the serving stream (Poisson, --serve-rate per s)")
    ap.add_argument("--serve-rate", type=float, default=20.0)
    ap.add_argument("--serve-burst", type=int, default=200,
                    help="requests submitted at once for the saturated-throughput figure")
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

def host_cpu():
    """(logical cores, CPU model string) of this host."""
    cores = os.cpu_count() or 1
    model = None
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                model = line.split(":", 1)[1].strip()
                break
    except (OSError, subprocess.SubprocessError):
        pass
    if not model:
        try:
            for line in Path("/proc/cpuinfo").read_text().splitlines():
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
        except OSError:
            pass
    return cores, model or "unknown"


_ORACLE_INPUTS = {}


def oracle_sample(n_chains: int, nsweeps: int = 1, threads: int = 1):
    """Time the oracle's Gibbs sweep on n_chains chains of the workload's
    planted model; with threads > 1 the chains are split into contiguous
    slices, one per host thread (each slice keeps its global chain indices,
    so the draws are those of one call over all chains; the oracle's ctypes
    calls release the GIL).  Returns (site-updates/s, seconds)."""
    import oracle
    from paper_2501_18456_gb300 import synth
    oracle.build()
    if not _ORACLE_INPUTS:
        h, J = synth.planted_contact_model(L_SITES, Q, SEED)
        _ORACLE_INPUTS["hJ"] = (h.astype(np.float64), J.astype(np.float64))
    h64, J64 = _ORACLE_INPUTS["hJ"]
    s0 = oracle.chains_init(n_chains, L_SITES, Q, SEED)
    threads = max(1, min(threads, n_chains))
    bounds = [n_chains * k // threads for k in range(threads + 1)]

    def part(k):
        a, b = bounds[k], bounds[k + 1]
        oracle.gibbs(h64, J64, s0[a:b], SEED, 0, nsweeps, 1.0, a)

    t0 = time.perf_counter()
    if threads == 1:
        part(0)
    else:
        ths = [threading.Thread(target=part, args=(k,)) for k in range(threads)]
        for t in ths:
            t.start()
        for t in ths:
            t.join()
    dt = time.perf_counter() - t0
    return n_chains * L_SITES * nsweeps / dt, dt


def calibrate_oracle_chains(target_s: float, threads: int = 1) -> int:
    """Chains for a ~target_s one-sweep sample (at most the workload's M)."""
    rate, _ = oracle_sample(8)
    return min(M_CHAINS, max(8 * threads, int(rate * threads * target_s / L_SITES)))


def cpu_baselines(args):
    """The oracle on one host thread and on every host core (chains split
    across threads), each a ~12 s sample of the workload."""
    cores, model = host_cpu()
    out = {}
    for name, th in (("single_thread", 1), ("all_cores", cores)):
        n = min(M_CHAINS, args.cpu_chains * th) if args.cpu_chains else calibrate_oracle_chains(12.0, th)
        r, dt = oracle_sample(n, 1, th)
        out[name] = {"value": r, "unit": UNIT, "cores": th, "kind": "oracle",
                     "sample": f"oracle Gibbs sweep on {n} of the {M_CHAINS} chains, 1 sweep, "
                               f"{dt:.1f} s, FP64 C, {th} thread(s)"}
    best = out["all_cores"]
    return {"value": best["value"], "unit": UNIT, "cores": best["cores"], "kind": "oracle",
            "sample": best["sample"], "nproc": cores, "cpu_model": model,
            "single_thread": out["single_thread"]}


def run_reference(args, rank):
    if rank != 0:
        return
    cores, cpu_model = host_cpu()
    n = min(M_CHAINS, args.cpu_chains * cores) if args.cpu_chains else calibrate_oracle_chains(1.5, cores)
    for _ in range(args.warmup):
        oracle_sample(max(8, n // 4), 1, cores)
    rates, times = [], []
    for _ in range(args.steps):
        r, dt = oracle_sample(n, 1, cores)
        rates.append(r)
        times.append(dt)
    value = statistics.median(rates)
    sample = (f"oracle Gibbs sweep on {n} of the {M_CHAINS} chains per step (FP64 C, {cores} threads, "
              f"chains split across host cores; {cpu_model})")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT,
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * statistics.median(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": sample},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": sample, "nproc": cores, "cpu_model": cpu_model},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------- GPU arm

def sparse_leg(bmdca, model, fi, fij, L, q, M, seed):
    """Sparse-graph steps (Sec. 2.2) at the bench shape, on a copy of the
    trained model: one edDCA decimation step at the paper's default rate
    (1 % of the active elements), a short edDCA run (10 graph steps, each
    followed by gsteps = 10 parameter updates with 10 sweeps before each),
    and one eaDCA activation step on an empty graph (0.1 % of the elements).
    The graph calls synchronise their stream (the selection is host-driven),
    so their times are CUDA-event times that include those round trips."""
    import torch

    dev = "cuda"
    h = torch.empty((L, q), dtype=torch.float32, device=dev)
    J = torch.empty((L, L, q, q), dtype=torch.float32, device=dev)
    bmdca.bm_potts_get(model, h, J)
    m = bmdca.bm_potts_load(h, J)
    del h, J
    c = bmdca.bm_chains_init(m, M, seed + 7)
    bmdca.bm_gibbs_sweep(m, c, 10, 1.0)
    counts = torch.empty((bmdca.n_blocks(L), q, q), dtype=torch.int32, device=dev)
    bmdca.bm_chain_stats(c, counts)
    st = torch.cuda.current_stream()

    def timed_call(fn):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        a.record(st)
        r = fn()
        b.record(st)
        torch.cuda.synchronize()
        return r, a.elapsed_time(b)

    bmdca.bm_graph_enable(m, True)
    na, ne = bmdca.bm_graph_count(m)
    removed, dec_ms = timed_call(lambda: bmdca.bm_graph_decimate(m, counts, M, int(0.01 * na)))
    gsteps, nsw, nsteps = 10, 10, 10
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    torch.cuda.synchronize()
    a.record(st)
    for _ in range(nsteps):
        bmdca.bm_graph_decimate(m, counts, M, int(0.01 * bmdca.bm_graph_count(m)[0]))
        for _ in range(gsteps):
            bmdca.bm_gibbs_sweep(m, c, nsw, 1.0)
            bmdca.bm_chain_stats(c, counts)
            bmdca.bm_update(m, fi, fij, counts, M, LR, 2.0, False)
    b.record(st)
    torch.cuda.synchronize()
    run_ms = a.elapsed_time(b)
    density = bmdca.bm_graph_count(m)[0] / ne
    bmdca.bm_graph_enable(m, False)
    bmdca.bm_chain_stats(c, counts)
    activated, act_ms = timed_call(lambda: bmdca.bm_graph_activate(m, fij, counts, M, int(0.001 * ne)))
    bmdca.bm_device_status(m)
    del m, c, counts
    return {"elements": ne, "decimate_ms": dec_ms, "decimate_removed": removed,
            "activate_ms": act_ms, "activated": activated,
            "eddca_graph_steps": nsteps, "gsteps": gsteps, "nsweeps": nsw,
            "eddca_ms_per_graph_step": run_ms / nsteps, "eddca_density_after": density,
            "note": "graph steps select exactly n elements by FP64 score (symmetric KL for "
                    "decimation, Bernoulli KL for activation), ties by element number"}


def split_precision_leg(bmdca, synth, timed):
    """Split-precision RNA-like shape (L=120, q=5, M=20,000): the sweep with
    fp16 hi+lo J on the tensor cores (the engine AUTO picks) against the
    plain FP32 CUDA-core sweep, the FP8 one-hot counts against CUDA-core
    histograms, and the max |error| of fields, f_i and f_ij against an FP64
    evaluation of the same definitions (numpy, FP64) on the same states."""
    import torch
    L, q, M, seed = 120, 5, 20000, 21
    h, J = synth.planted_contact_model(L, q, 11)
    model = bmdca.bm_potts_load(torch.from_numpy(h).cuda(), torch.from_numpy(J).cuda())
    out = {"shape": {"L": L, "q": q, "M": M}}
    for name, eng in (("split", bmdca.BM_ENGINE_AUTO), ("plain_fp32", bmdca.BM_ENGINE_SIMT)):
        bmdca.bm_model_set_engine(model, eng)
        c = bmdca.bm_chains_init(model, M, seed)
        bmdca.bm_gibbs_sweep(model, c, 3, 1.0)  # warm-up (layouts, code)
        ms = timed(lambda: bmdca.bm_gibbs_sweep(model, c, 10, 1.0), 2) / 10
        bmdca.bm_device_status(model)
        out[f"sweep_ms_{name}"] = ms
        out[f"site_updates_per_s_{name}"] = M * L / (ms * 1e-3)
        form = bmdca.bm_model_sweep_engine(model, M)
        out[f"engine_{name}"] = {bmdca.BM_ENGINE_MMA_PAIR: "two-CTA tensor cores (fp16 hi+lo)",
                                 bmdca.BM_ENGINE_MMA_PAIR2: "paired two-CTA tensor cores (fp16 hi+lo)",
                                 bmdca.BM_ENGINE_MMA: "one-CTA tensor cores (fp16 hi+lo)"}.get(
                                     form, "CUDA-core FP32 gather")
        c.free()
    out["sweep_speedup_vs_plain_fp32"] = out["sweep_ms_plain_fp32"] / out["sweep_ms_split"]
    bmdca.bm_model_set_engine(model, bmdca.BM_ENGINE_AUTO)
    c = bmdca.bm_chains_init(model, M, seed)
    bmdca.bm_gibbs_sweep(model, c, 5, 1.0)
    counts = torch.empty((bmdca.n_blocks(L), q, q), dtype=torch.int32, device="cuda")
    for name, eng in (("fp8", bmdca.BM_STATS_MMA_FP8), ("plain", bmdca.BM_STATS_SIMT)):
        bmdca.bm_chains_set_stats_engine(c, eng)
        bmdca.bm_chain_stats(c, counts)
        out[f"counts_ms_{name}"] = timed(lambda: bmdca.bm_chain_stats(c, counts), 5)
    bmdca.bm_chains_set_stats_engine(c, bmdca.BM_STATS_MMA_FP8)
    bmdca.bm_chain_stats(c, counts)
    S = torch.empty((M, L), dtype=torch.uint8, device="cuda")
    bmdca.bm_chains_get(c, S)
    torch.cuda.synchronize()
    S = S.cpu().numpy()
    C = counts.cpu().numpy().astype(np.int64)
    # FP64 definitions: f_ij(a,b) = #{m: s_i=a, s_j=b} / M over i <= j
    X = np.zeros((M, L * q), dtype=np.float64)
    X[np.repeat(np.arange(M), L), (np.arange(L) * q)[None, :].repeat(M, 0).ravel() + S.ravel()] = 1.0
    G = X.T @ X
    iu = [(i, j) for i in range(L) for j in range(i, L)]
    ref = np.stack([G[i * q:(i + 1) * q, j * q:(j + 1) * q] for i, j in iu]).astype(np.int64)
    out["f_ij_max_abs_err"] = float(np.abs(C - ref).max() / M)
    diag = [i * L - i * (i - 1) // 2 for i in range(L)]
    out["f_i_max_abs_err"] = float(max(np.abs(np.diag(C[d]) - np.diag(ref[d])).max() for d in diag) / M)
    # fields H_i(a) = h_i(a) + sum_{j != i} J_ij(a, s_j) of 300 sampled chains
    samp = S[np.random.default_rng(0).choice(M, 300, replace=False)]
    h64, J64 = h.astype(np.float64), J.astype(np.float64)
    Href = np.empty((300, L, q))
    for k in range(300):
        # J64[:, j, :, s_j] over j: shape (j, i, a); the sum over j gives (i, a)
        Href[k] = h64 + J64[:, np.arange(L), :, samp[k]].sum(axis=0)
    out["fields_max_abs_err"] = {}
    for name, form in (("fp32", bmdca.BM_FIELDS_FP32), ("fp16x2", bmdca.BM_FIELDS_FP16X2),
                       ("bf16x2", bmdca.BM_FIELDS_BF16X2)):
        H = torch.empty((300, L, q), dtype=torch.float32, device="cuda")
        bmdca.bm_fields(model, torch.from_numpy(samp).cuda(), H, form)
        bmdca.bm_device_status(model)
        out["fields_max_abs_err"][name] = float(np.abs(H.cpu().numpy().astype(np.float64) - Href).max())
    c.free()
    model.free()
    return out


def run_ours(args, rank, world, local):
    import torch
    import torch.distributed as dist
    from paper_2501_18456_gb300 import _build, bmdca, planted, synth, train

    if world > 1:
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    _build.build()

    def barrier():
        if world > 1:
            dist.barrier()

    st = torch.cuda.current_stream()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    def timed(fn, reps=1, warm=True):
        """CUDA-event ms per call; one untimed call first, so that the first
        launch of each kernel (module loading) and the first allocation from
        the stream's pool stay outside the timed region."""
        if warm:
            fn()
        a, b = ev(), ev()
        torch.cuda.synchronize()
        a.record(st)
        for _ in range(reps):
            fn()
        b.record(st)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    # ---- inputs: the planted model and its data MSA, sampled by the library's
    # own sweeps (each rank runs its own replica with its own chain seed)
    seed = SEED + rank
    data = planted.build(N_SEQS, N_SEQS // 10, 500, SEED, L_SITES, Q)
    msa_d = torch.from_numpy(data["msa"]).to(dev)

    rows = {}
    w = torch.empty(N_SEQS, dtype=torch.float32, device=dev)
    meff_box = {}
    rows["seq_weights_ms"] = timed(lambda: meff_box.setdefault("m", bmdca.bm_seq_weights(msa_d, w, 0.8)))
    fi = torch.empty((L_SITES, Q), dtype=torch.float32, device=dev)
    fij = torch.empty((L_SITES, L_SITES, Q, Q), dtype=torch.float32, device=dev)
    rows["data_stats_ms"] = timed(lambda: bmdca.bm_data_stats(msa_d, w, Q, -1.0, fi, fij))
    stats = train.DataStats(fi, fij, meff_box["m"], w)
    h0, J0 = train.profile_init(stats)
    model = bmdca.bm_potts_load(h0, J0)
    chains_box = {}
    bmdca.bm_chains_init(model, M_CHAINS, seed).free()  # untimed first call
    rows["chains_init_ms"] = timed(lambda: chains_box.setdefault("c", bmdca.bm_chains_init(model, M_CHAINS, seed)),
                                   warm=False)
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
    # the same sweep with Metropolis-Hastings steps (the sampler option)
    bmdca.bm_model_set_sampler(model, bmdca.BM_SAMPLER_METROPOLIS)
    bmdca.bm_gibbs_sweep(model, chains, 2, 1.0)
    rows["metropolis_sweep_ms_per_sweep"] = timed(lambda: bmdca.bm_gibbs_sweep(model, chains, NSWEEPS, 1.0), 2) / NSWEEPS
    bmdca.bm_model_set_sampler(model, bmdca.BM_SAMPLER_GIBBS)
    rows["chain_stats_ms"] = timed(lambda: bmdca.bm_chain_stats(chains, counts), 5)
    rows["update_pearson_ms"] = timed(lambda: bmdca.bm_update(model, fi, fij, counts, M_CHAINS, LR, 2.0, True), 5)
    n_score = 100000
    seqs = torch.from_numpy(synth.random_states(n_score, L_SITES, Q, 5)).to(dev)
    E = torch.empty(n_score, dtype=torch.float32, device=dev)
    rows["energy_score_ms_1e5_seqs"] = timed(lambda: bmdca.bm_energy_score(model, seqs, E), 2)
    dE = torch.empty((L_SITES, Q), dtype=torch.float32, device=dev)
    wt = msa_d[0].contiguous()
    rows["mutant_scan_ms"] = timed(lambda: bmdca.bm_mutant_scan(model, wt, dE), 5)

    # ---- end to end through the public API with host buffers: every step
    # uploads the parameters and the chain states from pinned host memory and
    # reads the new states back
    h_pin = torch.empty((L_SITES, Q), dtype=torch.float32).pin_memory()
    J_pin = torch.empty((L_SITES, L_SITES, Q, Q), dtype=torch.float32).pin_memory()
    bmdca.bm_potts_get(model, h_pin, J_pin)
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
    # The launch (10 sweeps) takes ~15 ms, so the burst peak applies.
    peaks, peak_src = {}, "fallback"
    try:
        peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
        peak_src = "measured"
    except (OSError, ValueError):
        pass
    peak_tf = float(peaks.get("bf16_tflops", 1900.0))
    peak_tf_sus = float(peaks.get("bf16_tflops_sustained", 1700.0))
    Qd = float(L_SITES * Q)
    flops_per_launch = 2.0 * 2.0 * M_CHAINS * Qd * Qd * NSWEEPS
    achieved = flops_per_launch / (ms_gibbs * 1e-3) / 1e12
    bmdca.bm_model_set_engine(model, bmdca.BM_ENGINE_AUTO)
    form = bmdca.bm_model_sweep_engine(model, M_CHAINS)
    kname = {bmdca.BM_ENGINE_MMA_PAIR: "k_gibbs_pair", bmdca.BM_ENGINE_MMA_PAIR2: "k_gibbs_pair (paired tensor cores)",
             bmdca.BM_ENGINE_MMA: "k_gibbs_mma"}.get(form, "k_gibbs_staged")
    roofline = {"bound": "tensor", "achieved": achieved, "peak": peak_tf, "unit": "TFLOP/s",
                "frac": achieved / peak_tf, "traffic": TRAFFIC_GIBBS.get(kname),
                "kernel": kname,
                "frac_of_sustained_peak": achieved / peak_tf_sus,
                "method_adds_per_site_update": L_SITES * Q,
                "tensor_flops_per_site_update": 4 * L_SITES * Q * Q,
                "note": "achieved = 2 passes (fp16 hi, lo) x 2*M*(L*q)^2 flops per sweep x sweeps per launch / "
                        "CUDA-event launch time; peak: " + peak_src + " bf16_tflops (burst; a 10-sweep "
                        "launch lasts ~15 ms), fp16 and bf16 share the dense rate; the contraction issues "
                        "4*L*q^2 tensor flops per site-update where the method's field needs L*q adds"}

    # ---- roofline of the chain counts (the other tensor-core row of the step):
    # one-hot X^T X over the upper block triangle, 2*M*(L(L+1)/2)*q^2 flops,
    # FP8 operands; peak = the measured bf16 rate x 2 (nominal fp8/bf16 ratio).
    cs_flops = 2.0 * M_CHAINS * (L_SITES * (L_SITES + 1) / 2) * Q * Q
    cs_ach = cs_flops / (rows["chain_stats_ms"] * 1e-3) / 1e12
    roofline_counts = {"bound": "tensor", "achieved": cs_ach, "peak": 2 * peak_tf, "unit": "TFLOP/s",
                       "frac": cs_ach / (2 * peak_tf), "kernel": "k_onehot_t + k_counts_pair",
                       "note": "achieved = 2*M*(L(L+1)/2)*q^2 flops / CUDA-event time of bm_chain_stats "
                               "(one-hot build included); peak: fp8 = 2 x " + peak_src + " bf16_tflops (burst)"}
    # update + Pearson: 16 B per coupling parameter (read J and f_ij, the
    # counts, write the new J) over the L^2 q^2 parameters; the time is the
    # whole call, including the read-back of the Pearson moments
    upd_bytes = 16.0 * (L_SITES * Q) ** 2
    peak_hbm = float(peaks.get("hbm_gbs", 6800.0))
    upd_ach = upd_bytes / (rows["update_pearson_ms"] * 1e-3) / 1e9
    roofline_update = {"bound": "hbm", "achieved": upd_ach, "peak": peak_hbm, "unit": "GB/s",
                       "frac": upd_ach / peak_hbm, "kernel": "k_update_rows + k_update_fields + k_sum_partials",
                       "note": "achieved = 16 B x (L q)^2 parameters / CUDA-event time of bm_update with the Pearson "
                               "check (moments read back to the host); peak: " + peak_src + " hbm_gbs"}

    # ---- split precision (RNA-like shape), rank 0
    split = None
    if rank == 0 and not args.no_split:
        split = split_precision_leg(bmdca, synth, timed)
        torch.cuda.empty_cache()

    # ---- training from the profile model to the Pearson target (rank 0)
    train_run = None
    if rank == 0 and not args.no_train:
        cfg = train.TrainConfig(M=M_CHAINS, nsweeps=NSWEEPS, lr=LR, seed=seed, max_iters=500, target=0.95)
        train_run, m_t, c_t = planted.train_to_target(msa_d, Q, cfg, stats)
        hT = torch.empty((L_SITES, Q), dtype=torch.float32, device=dev)
        JT = torch.empty((L_SITES, L_SITES, Q, Q), dtype=torch.float32, device=dev)
        bmdca.bm_potts_get(m_t, hT, JT)
        # recovery of the planted couplings (zero-sum gauge, contact pairs and all pairs)
        Jp = torch.from_numpy(data["J"]).to(dev)

        def zs(x):
            return x - x.mean(dim=2, keepdim=True) - x.mean(dim=3, keepdim=True) + x.mean(dim=(2, 3), keepdim=True)

        a_, b_ = zs(JT).flatten(), zs(Jp).flatten()
        train_run["J_pearson_vs_planted"] = float(torch.corrcoef(torch.stack([a_, b_]))[0, 1])
        train_run["planted_gap_shift"] = data["gap_shift"]
        train_run["data_gap_fraction"] = float((msa_d == 0).float().mean())
        train_run["data_generation_s"] = data["seconds"]
        train_run["lr"] = LR
        del m_t, c_t, hT, JT, a_, b_
        torch.cuda.empty_cache()
        # the same run with a larger learning rate (the paper's text and table
        # disagree on the default; the gradient of Eq. 5 is small here)
        cfg2 = train.TrainConfig(M=M_CHAINS, nsweeps=NSWEEPS, lr=0.5, seed=seed, max_iters=500, target=0.95)
        run2, m2, c2 = planted.train_to_target(msa_d, Q, cfg2, stats)
        JT = torch.empty((L_SITES, L_SITES, Q, Q), dtype=torch.float32, device=dev)
        bmdca.bm_potts_get(m2, None, JT)
        a_, b_ = zs(JT).flatten(), zs(Jp).flatten()
        run2["J_pearson_vs_planted"] = float(torch.corrcoef(torch.stack([a_, b_]))[0, 1])
        run2["lr"] = 0.5
        train_run["lr_0.5"] = run2
        del m2, c2, JT, Jp, a_, b_
        torch.cuda.empty_cache()

    # ---- sparse graphs (edDCA / eaDCA steps) on a copy of the model (rank 0)
    sparse = None
    if rank == 0 and not args.no_sparse:
        sparse = sparse_leg(bmdca, model, fi, fij, L_SITES, Q, M_CHAINS, seed)
        torch.cuda.empty_cache()

    # ---- serving: Poisson streams of sample / score / mutant-scan requests over
    # 32 resident models through the continuous-batching server (rank 0), with
    # the default engines and with plain FP32 sampling; then the same mix
    # submitted at once (saturated capacity).
    serve = None
    if rank == 0 and not args.no_serve:
        from paper_2501_18456_gb300 import serving
        smodels = serving.make_models(32, 0)
        seeds = (1, 2, 3, 4)
        tc = serving.run_seeds(smodels, args.serve_rate, args.serve_requests, seeds, engine=bmdca.BM_ENGINE_AUTO)
        plain = serving.run_seeds(smodels, args.serve_rate, args.serve_requests, seeds, engine=bmdca.BM_ENGINE_SIMT)
        dur = args.serve_burst / args.serve_rate
        tc_b = serving.run_stream(smodels, args.serve_rate, dur, 9, engine=bmdca.BM_ENGINE_AUTO, burst=True)
        plain_b = serving.run_stream(smodels, args.serve_rate, dur, 9, engine=bmdca.BM_ENGINE_SIMT, burst=True)
        keys = ("p50_ms", "p50_ms_range", "p99_ms", "p99_ms_range", "mean_ms", "sequences_per_s", "requests",
                "max_running", "offered_rate_per_s", "per_seed")
        bkeys = ("requests", "sequences_per_s", "p50_ms", "p99_ms", "max_running", "wall_s")
        serve = {"workload": "32 resident models (L U[60,400], q 21/5), Poisson arrivals: sample "
                             "logU[1e2,1e4] seqs x U[20,200] sweeps at beta {0.8,1,1.2}, score "
                             "logU[1e3,1e6] seqs, single-mutant scans; 4 seeds",
                 **{k: tc[k] for k in keys},
                 "saturated": {k: tc_b[k] for k in bkeys},
                 "plain_fp32": {**{k: plain[k] for k in keys}, "saturated": {k: plain_b[k] for k in bkeys}},
                 "capacity_speedup_vs_plain_fp32": tc_b["sequences_per_s"] / plain_b["sequences_per_s"]}
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
        cpu = cpu_baselines(args)

    # Kernels launched per step: the tensor-core layout and in-block coupling
    # rebuilds (the previous update changed J) + the Gibbs sweep, chain counts
    # (one-hot build + product), update (row tiles, fields, Pearson partial
    # sum).  The gather layout is not rebuilt: only the CUDA-core forms read it.
    launches_per_step = 3 + 2 + 3
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "fp16 hi+lo J x fp16 one-hot, f32 accumulate",
                "data": "synthetic (planted Potts model; MSA sampled from it by the library's Gibbs sweeps)",
                "config": {"workload": WORKLOAD, "L": L_SITES, "q": Q, "M": M_CHAINS,
                           "N": N_SEQS, "nsweeps": NSWEEPS, "lr": LR, "meff": meff_box.get("m"),
                           "init": "profile model h = log f_i, J = 0",
                           "engine": "tcgen05 tensor cores: J as fp16 hi + fp16 lo, one-hot fp16 (exact), "
                                     "f32 accumulate in TMEM; draws in f32",
                           "l2": "flushed between steps (256 MB write)",
                           "parallelism": f"replicas x{world}", "pearson_last": rho},
                "plain_fp32": {"value": world * site_updates_per_step / (ms_plain * 1e-3), "unit": UNIT,
                               "ms_per_step": ms_plain, "gibbs_ms_per_sweep": ms_plain_gibbs / NSWEEPS,
                               "engine": "CUDA-core FP32 gather (k_gibbs_staged)",
                               "speedup_of_value": ms_plain / ms_step},
                "roofline": roofline, "roofline_chain_stats": roofline_counts, "roofline_update": roofline_update, "cpu_baseline": cpu,
                "e2e": {"value": world * site_updates_per_step / (e2e_ms * 1e-3), "unit": UNIT,
                        "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
                "gpu_launches": launches_per_step * args.steps,
                "clocks": clk, "rows_ms": rows, "train_to_target": train_run,
                "split_precision": split, "sparse": sparse, "serve": serve, "batched": batched,
                "wall_s_timed": t_wall}
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
