"""Benchmark: exact L x L Ising-PEPS energy evaluations per second on GB300.

Workload (one "step"): a batch of B independent 8x8 open-boundary PEPS of bond
D = 2 (seeded uniform[-1,1) site tensors, one fresh seed set per rank), each
contracted exactly into its norm, all 64 <X_k> and all 112 nearest-neighbour
<Z_i Z_j>, from which E is formed at h in {2.0, 3.04, 4.0} (J = 1).  The whole
hot path -- site matrices, every corner chain, ring closure, environments,
observable insertions, FP64 ratios -- runs in libtn's kernels; the launch
sequence is a replayed CUDA graph.

value  : lattice energy evaluations/s, inputs resident in HBM, CUDA events on
         the library's stream, L2 flushed (256 MB write) between timed steps.
e2e    : the same metric through the C-ABI with host buffers: per step the
         pinned host tensors are copied in, the batch runs, the result array is
         read back.
--impl reference: the FP64 CPU oracle on the host cores (a bounded sample).
Multi-GPU (torchrun): each rank runs its own batch (replicas, weak scaling).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L_, W_, D_ = 8, 8, 2
H_FIELDS = (2.0, 3.04, 4.0)
METRIC = "exact LxL Ising-PEPS energy evals/s"
ABSORB_DRAM_PER_BYTE = 89.35 / 134.22      # k_absorb4<16,16,1,0> capture, profiles/k_absorb4_8x8_d2_batch64.md
GEMM_DRAM_PER_MAC = 373.1e6 / (640 * 256.0 ** 3)   # k_gemm3<1,0,1> capture, profiles/k_gemm3_8x8_d2_batch64.md
WORKLOAD = "8x8 open-boundary TFIM PEPS, D=2, E at h in {2.0, 3.04, 4.0}"


def _peak_key(key, default):
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)[key])
    except Exception:
        return default


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), float(p["bf16_tflops"]), float(p.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 1900.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device: int, path: str | None = None):
        import tempfile
        self.device = device
        self.proc = None
        self.path = path or os.path.join(tempfile.gettempdir(), f"tn_clocks_{os.getpid()}_{device}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.device), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.fh, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        try:
            for line in open(self.path):
                f = [x.strip() for x in line.split(",")]
                if len(f) < 9:
                    continue
                try:
                    sm.append(float(f[1]))
                    mx.append(float(f[2]))
                except ValueError:
                    continue
                for n, v in zip(names, f[5:9]):
                    if v.lower() == "active":
                        reasons.add(n)
        except OSError:
            pass
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def absorb_stream_roofline(ctx, stream, hbm: float, src: str) -> dict:
    """The single-step absorption kernel on single tasks larger than L2: the
    forced row scheme of one 12x12 D=2 norm (interior steps of 268 MB in and
    268 MB out), timed per launch with CUDA events after two warm-up runs."""
    import numpy as np
    import torch

    from paper_1908_08553_gb300 import inputs, tn
    L, W, D = 12, 12, 2
    b = tn.tn_batch_create(ctx, [L], [W], [D], tn.TN_FP32, tn.TN_SCHED_ROW, tn.TN_WORK_NORM)
    try:
        tn.tn_batch_set_tensors(b, inputs.random_lattice(L, W, D, 1214))
        hs = np.array([3.04])
        for _ in range(2):
            tn.tn_batch_run(b, 1.0, hs)
        torch.cuda.synchronize()
        tn.tn_ctx_set_profiling(ctx, True)
        for _ in range(3):
            tn.tn_batch_run(b, 1.0, hs)
        torch.cuda.synchronize()
        a = tn.tn_ctx_kernel_stats(ctx, 0)
        tn.tn_ctx_set_profiling(ctx, False)
    finally:
        tn.tn_batch_destroy(b)
    achieved = a["bytes"] / (a["ms"] / 1e3) / 1e9
    return {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
            "traffic": None, "kernel": "absorb (k_absorb4, single step)",
            "workload": "12x12 D=2 norm, forced row scheme, FP32 (steps of 268 MB in + 268 MB out)",
            "launches": a["launches"] / 3, "ms_per_run": a["ms"] / 3,
            "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs (of {src})"}


def max_over_ranks(x: float, ws: int, device: str = "cuda") -> float:
    """The largest of every rank's x (the job's time is its slowest replica)."""
    if ws <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(ws: int, units_per_rank: int, steps: int, t_max: float) -> float:
    """Whole-job throughput: the units all replicas processed over the slowest time."""
    return ws * units_per_rank * steps / t_max


def replica_seed(rank: int) -> int:
    """Batch seed of a rank's replica: every rank contracts its own lattices."""
    return 4242 + rank


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def cpu_baseline(n_lattices: int, seed: int):
    """The FP64 oracle, as it stands, on a bounded sample of the same workload."""
    import oracle
    from paper_1908_08553_gb300 import inputs
    t0 = time.perf_counter()
    for k in range(n_lattices):
        A = inputs.random_lattice(L_, W_, D_, inputs.lattice_seed(seed, k))
        ob = oracle.observables(L_, W_, D_, A)
        _ = [ob.energy(1.0, h) for h in H_FIELDS]
    dt = time.perf_counter() - t0
    return {"value": n_lattices / dt, "unit": "lattice evals/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": f"{n_lattices} seeded 8x8 D=2 lattices, full observable set, FP64 row-sweep oracle, "
                      f"{dt:.1f} s wall"}


def run_reference(args):
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    per_step = max(1, args.ref_lattices)
    for _ in range(args.warmup):
        cpu_baseline(1, 99)
    t0 = time.perf_counter()
    for s in range(args.steps):
        cpu_baseline(per_step, 1000 + s)
    dt = time.perf_counter() - t0
    value = args.steps * per_step / dt
    line = {"metric": METRIC, "value": value, "unit": "lattice evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "impl": "reference",
            "config": {"workload": WORKLOAD, "batch": per_step, "L": L_, "W": W_, "D": D_,
                       "h": list(H_FIELDS)},
            "cpu_baseline": {"value": value, "unit": "lattice evals/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": f"{per_step} lattice(s) per step x {args.steps} steps"},
            "e2e": {"value": value, "unit": "lattice evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def run_large(args):
    """Large single instances: 12x12 D=2 and 8x8 D=3 (forced row scheme for the
    absorption roofline, AUTO for energies), one line of JSON."""
    import numpy as np
    import torch

    from paper_1908_08553_gb300 import inputs, tn

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = tn.tn_ctx_create(0, 0, stream)
    hbm, bf16, sm_max, src = _peaks()
    out = {"workload": "large single instances (12x12 D=2, 8x8 D=3)", "peak_hbm_gbs": hbm}
    for (L, W, D) in [(12, 12, 2), (8, 8, 3)]:
        A = inputs.random_lattice(L, W, D, 1000 + L + D)
        key = f"{L}x{W}_D{D}"
        res = {}
        for label, sched, prec, work in [("row_norm_fp32", tn.TN_SCHED_ROW, tn.TN_FP32, tn.TN_WORK_NORM),
                                         ("auto_norm_fp32", tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_NORM),
                                         ("auto_energy_fp32", tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY),
                                         ("auto_energy_bf16x3", tn.TN_SCHED_AUTO, tn.TN_BF16X3, tn.TN_WORK_ENERGY),
                                         ("auto_energy_fp64", tn.TN_SCHED_AUTO, tn.TN_FP64, tn.TN_WORK_ENERGY)]:
            b = tn.tn_batch_create(ctx, [L], [W], [D], prec, sched, work)
            tn.tn_batch_set_tensors(b, A)
            hs = np.array([3.04])
            for _ in range(2):
                tn.tn_batch_run(b, 1.0, hs)
            torch.cuda.synchronize()
            reps = 3
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(reps):
                tn.tn_batch_run(b, 1.0, hs)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / reps
            tn.tn_ctx_set_profiling(ctx, True)
            tn.tn_batch_run(b, 1.0, hs)
            torch.cuda.synchronize()
            fam = {n: tn.tn_ctx_kernel_stats(ctx, k) for k, n in
                   enumerate(["absorb", "absorb_dot", "gemm_simt", "gemm_tc", "other", "absorb_pair"])}
            tn.tn_ctx_set_profiling(ctx, False)
            r = tn.tn_batch_results_host(b)
            entry = {"ms": ms, "evals_per_s": 1000.0 / ms, "log2_norm": float(r[1])}
            if work == tn.TN_WORK_ENERGY:
                entry["energy_per_site"] = float(r[0]) / (L * W)
            a = fam["absorb"]
            if a["ms"]:
                gbs = a["bytes"] / (a["ms"] / 1e3) / 1e9
                entry["absorb"] = {"ms": a["ms"], "launches": a["launches"], "GBps": gbs, "frac_hbm": gbs / hbm,
                                   "TFLOPs": 2 * a["macs"] / (a["ms"] / 1e3) / 1e12}
            entry["families_ms"] = {n: v["ms"] for n, v in fam.items() if v["launches"]}
            res[label] = entry
            tn.tn_batch_destroy(b)
        out[key] = res
    tn.tn_ctx_destroy(ctx)
    print(json.dumps(out), flush=True)
    return 0


def run_serve(args):
    """Serving: a Poisson stream of requests (L, W ~ U{4..12}, D ~ U{2,3},
    h ~ U[0.5, 5], seeded tensors) at 80% of the measured capacity, admitted by
    exact footprint against a 160 GB budget; p50/p99 latency and throughput,
    beside sequential FP64 solves of a sample of the same requests."""
    import threading

    import numpy as np
    import torch

    from paper_1908_08553_gb300 import tn

    torch.cuda.set_device(0)
    prec = tn.PRECISIONS[args.precision]
    budget = int(160e9)
    rng = np.random.default_rng(3)
    n = args.requests
    reqs = [(int(rng.integers(4, 13)), int(rng.integers(4, 13)), int(rng.choice([2, 3])),
             float(rng.uniform(0.5, 5.0)), 10_000 + k) for k in range(n + args.calibrate)]
    ctx = tn.tn_ctx_create(0, budget)
    probe = tn.tn_ctx_create(-1)
    fits = []
    for (L, W, D, h, seed) in reqs:
        lat = tn.tn_create_lattice(probe, L, W, D)
        fits.append(tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY) <= budget)
        tn.tn_destroy_lattice(lat)
    tn.tn_ctx_destroy(probe)
    calib = [r for r, f in zip(reqs[n:], fits[n:]) if f]
    stream_reqs = list(zip(reqs[:n], fits[:n]))

    # capacity: a burst of admissible requests
    t0 = time.perf_counter()
    ts = [tn.tn_submit(ctx, L, W, D, prec, 1.0, h, seed=sd) for (L, W, D, h, sd) in calib]
    for t, (L, W, D, h, sd) in zip(ts, calib):
        tn.tn_wait(ctx, t, 600.0, L, W)
    cap = len(calib) / (time.perf_counter() - t0)
    rate = 0.8 * cap

    # Poisson stream with a polling collector
    pending, done, lock = {}, {}, threading.Lock()
    stop = threading.Event()

    deadline = time.perf_counter() + 900.0

    def collector():
        while (not stop.is_set() or pending) and time.perf_counter() < deadline:
            with lock:
                items = list(pending.items())
            for t, (L, W, ts_) in items:
                r = tn.tn_poll(ctx, t, L, W)
                if r is not None:
                    with lock:
                        done[t] = (ts_, time.perf_counter(), r[0].energy)
                        del pending[t]
            time.sleep(0.0005)

    th = threading.Thread(target=collector)
    th.start()
    rejected = 0
    gaps = rng.exponential(1.0 / rate, size=n)
    t_start = time.perf_counter()
    t_next = t_start
    for ((L, W, D, h, sd), fit), g in zip(stream_reqs, gaps):
        t_next += g
        while time.perf_counter() < t_next:
            time.sleep(0.0002)
        try:
            t = tn.tn_submit(ctx, L, W, D, prec, 1.0, h, seed=sd)
        except tn.TNError as e:
            if e.status == tn.TN_ERR_OVER_BUDGET:
                rejected += 1
                continue
            raise
        with lock:
            pending[t] = (L, W, time.perf_counter())
    stop.set()
    th.join()
    t_end = max(v[1] for v in done.values())
    lat = np.array([v[1] - v[0] for v in done.values()])
    served = len(done)

    # sequential plain FP64 solves of a sample of the admitted requests (those
    # whose FP64 footprint also fits the budget)
    probe = tn.tn_ctx_create(-1)

    def fits64(L, W, D):
        lat_ = tn.tn_create_lattice(probe, L, W, D)
        ok = tn.tn_footprint(lat_, tn.TN_SCHED_AUTO, tn.TN_FP64, tn.TN_WORK_ENERGY) <= budget
        tn.tn_destroy_lattice(lat_)
        return ok

    sample = [r for r, f in stream_reqs if f and fits64(*r[:3])][: args.seq_sample]
    tn.tn_ctx_destroy(probe)
    t0 = time.perf_counter()
    n_seq = 0
    for (L, W, D, h, sd) in sample:
        l = tn.tn_create_lattice(ctx, L, W, D)
        tn.tn_fill_random(l, sd)
        tn.tn_energy(l, 1.0, h, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
        tn.tn_destroy_lattice(l)
        n_seq += 1
        if time.perf_counter() - t0 > args.seq_seconds:
            break
    seq_rate = n_seq / (time.perf_counter() - t0)
    tn.tn_ctx_destroy(ctx)
    line = {"metric": "served p50/p99 latency", "workload": "Poisson stream of TFIM-PEPS energy requests",
            "unit": "s", "precision": args.precision, "requests": n, "served": served, "rejected_over_budget": rejected,
            "budget_gb": budget / 1e9, "capacity_jobs_per_s": cap, "offered_rate_jobs_per_s": rate,
            "p50_latency_s": float(np.percentile(lat, 50)), "p99_latency_s": float(np.percentile(lat, 99)),
            "mean_latency_s": float(lat.mean()), "throughput_energies_per_s": served / (t_end - t_start),
            "sequential_fp64": {"energies_per_s": seq_rate, "sample": n_seq},
            "distribution": "L, W ~ U{4..12}, D ~ U{2,3}, h ~ U[0.5,5], seeded uniform[-1,1) tensors"}
    print(json.dumps(line), flush=True)
    return 0


def run_batch(args):
    """512 independent lattices, L, W ~ U{4..10}, D ~ U{2,3}, h ~ U[0.5,5]: as few
    graph-captured batches as the HBM budget allows (members run together,
    every wave of all members one grouped launch); members whose footprint
    alone exceeds the budget are reported, not run."""
    import numpy as np
    import torch

    from paper_1908_08553_gb300 import tn

    torch.cuda.set_device(0)
    prec = tn.PRECISIONS[args.precision]
    budget = int(200e9)
    rng = np.random.default_rng(2)
    n = args.members
    Ls = rng.integers(4, 11, size=n)
    Ws = rng.integers(4, 11, size=n)
    Ds = rng.choice([2, 3], size=n)
    hs = rng.uniform(0.5, 5.0, size=n)
    probe = tn.tn_ctx_create(-1)
    fp = []
    for L, W, D in zip(Ls, Ws, Ds):
        lat = tn.tn_create_lattice(probe, int(L), int(W), int(D))
        fp.append(tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY))
        tn.tn_destroy_lattice(lat)
    tn.tn_ctx_destroy(probe)
    ok = [k for k in range(n) if fp[k] <= budget]
    excluded = [k for k in range(n) if fp[k] > budget]
    # pack members in order into sub-batches of at most the budget
    groups, cur, used = [], [], 0
    for k in ok:
        if cur and used + fp[k] > budget:
            groups.append(cur)
            cur, used = [], 0
        cur.append(k)
        used += fp[k]
    if cur:
        groups.append(cur)
    stream = torch.cuda.Stream()
    ctx = tn.tn_ctx_create(0, int(250e9), stream)
    total_ms, results, launches = 0.0, {}, 0
    for g in groups:
        b = tn.tn_batch_create(ctx, Ls[g], Ws[g], Ds[g], prec)
        tn.tn_batch_fill_random(b, args.batch_seed)      # member seeds from the batch seed
        hh = hs[g].copy()
        tn.tn_batch_run(b, 1.0, hh)                      # capture + first run
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        tn.tn_batch_run(b, 1.0, hh)
        e1.record(stream)
        torch.cuda.synchronize()
        total_ms += e0.elapsed_time(e1)
        launches += tn.tn_batch_launch_count(b)
        r = tn.tn_batch_results_host(b)
        off = 0
        for k in g:
            L, W = int(Ls[k]), int(Ws[k])
            nres = 6 + 2 * L * W + L * (W - 1) + W * (L - 1)
            results[k] = r[off:off + nres]
            off += nres
        tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    m = len(ok)
    line = {"metric": "batched exact TFIM-PEPS energy evals/s", "workload": "512 mixed lattices, L, W in 4..10, D in {2,3}",
            "precision": args.precision, "members": n, "evaluated": m, "excluded_over_budget": len(excluded),
            "excluded_shapes": sorted({(int(Ls[k]), int(Ws[k]), int(Ds[k])) for k in excluded}),
            "graphs": len(groups), "kernel_launches": launches, "ms": total_ms,
            "evals_per_s": m / (total_ms / 1e3), "energies_per_s": m / (total_ms / 1e3),
            "budget_gb": budget / 1e9,
            "distribution": "L, W ~ U{4..10}, D ~ U{2,3}, h ~ U[0.5,5], seeded uniform[-1,1) tensors"}
    print(json.dumps(line), flush=True)
    return 0


def run_case(args):
    """One lattice (--L, --W, --D, --seed) contracted --steps times after
    --warmup runs, in one precision, schedule and work kind: the small,
    self-contained command that kernel captures run on."""
    import numpy as np
    import torch

    from paper_1908_08553_gb300 import inputs, tn

    torch.cuda.set_device(0)
    stream = torch.cuda.Stream()
    ctx = tn.tn_ctx_create(0, 0, stream)
    sched = {"auto": tn.TN_SCHED_AUTO, "row": tn.TN_SCHED_ROW, "col": tn.TN_SCHED_COL,
             "quadrant": tn.TN_SCHED_QUADRANT}[args.schedule]
    work = tn.TN_WORK_ENERGY if args.work == "energy" else tn.TN_WORK_NORM
    prec = tn.PRECISIONS[args.precision]
    L, W, D = args.L, args.W, args.D
    b = tn.tn_batch_create(ctx, [L] * args.batch, [W] * args.batch, [D] * args.batch, prec, sched, work)
    A = np.concatenate([inputs.random_lattice(L, W, D, inputs.lattice_seed(args.seed, k))
                        for k in range(args.batch)])
    tn.tn_batch_set_tensors(b, A)
    hs = np.full(args.batch, 3.04)
    for _ in range(args.warmup):
        tn.tn_batch_run(b, 1.0, hs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        tn.tn_batch_run(b, 1.0, hs)
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / max(1, args.steps)
    r = tn.tn_batch_results_host(b)
    line = {"workload": f"{args.batch} x {L}x{W} D={D}", "precision": args.precision,
            "schedule": args.schedule, "work": args.work, "ms_per_run": ms,
            "launches_per_run": tn.tn_batch_launch_count(b),
            "log2_norm": float(r[1]), "energy_per_site": float(r[0]) / (L * W)}
    tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=256, help="8x8 lattices per step per GPU")
    ap.add_argument("--precision", default="fp32", choices=["fp64", "fp32", "bf16x3", "bf16x6"])
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--ref-lattices", type=int, default=2)
    ap.add_argument("--cpu-lattices", type=int, default=10)
    ap.add_argument("--no-extras", action="store_true", help="skip the FP64 line and the CPU baseline")
    ap.add_argument("--workload", default="8x8", choices=["8x8", "large", "serve", "batch", "case"],
                    help="8x8: the bench line; large: 12x12 D=2 / 8x8 D=3; serve: Poisson request "
                         "stream; batch: 512 mixed lattices; case: --batch copies of one L x W lattice")
    ap.add_argument("--L", type=int, default=8, help="case: rows")
    ap.add_argument("--W", type=int, default=8, help="case: columns")
    ap.add_argument("--D", type=int, default=2, help="case: bond dimension")
    ap.add_argument("--seed", type=int, default=7, help="case: tensor seed")
    ap.add_argument("--schedule", default="auto", choices=["auto", "row", "col", "quadrant"])
    ap.add_argument("--work", default="energy", choices=["energy", "norm"], help="case: work kind")
    ap.add_argument("--clock-log", default=None, help="CSV file for the nvidia-smi clock samples")
    ap.add_argument("--members", type=int, default=512, help="batch: lattices")
    ap.add_argument("--batch-seed", type=int, default=2, help="batch: tensor seed")
    ap.add_argument("--requests", type=int, default=300, help="serve: requests in the stream")
    ap.add_argument("--calibrate", type=int, default=60, help="serve: burst size for the capacity")
    ap.add_argument("--seq-sample", type=int, default=30, help="serve: sequential FP64 sample")
    ap.add_argument("--seq-seconds", type=float, default=60.0, help="serve: time cap of the FP64 sample")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "large":
        return run_large(args)
    if args.workload == "serve":
        return run_serve(args)
    if args.workload == "batch":
        return run_batch(args)
    if args.workload == "case":
        return run_case(args)

    import numpy as np
    import torch

    from paper_1908_08553_gb300 import inputs, tn

    ws, rank, local = _dist()
    torch.cuda.set_device(local)
    if ws > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    stream = torch.cuda.Stream()
    ctx = tn.tn_ctx_create(local, 0, stream)
    B = args.batch
    prec = tn.PRECISIONS[args.precision]
    hs = np.array([H_FIELDS[k % 3] for k in range(B)])
    b = tn.tn_batch_create(ctx, [L_] * B, [W_] * B, [D_] * B, prec)
    n_in = tn.tn_batch_elems(b)
    host_in = torch.empty(n_in, dtype=torch.float64).pin_memory()
    A = np.concatenate([inputs.random_lattice(L_, W_, D_, inputs.lattice_seed(replica_seed(rank), k))
                        for k in range(B)])
    host_in.numpy()[:] = A
    n_res = tn.tn_batch_result_size(b)
    host_out = torch.empty(n_res, dtype=torch.float64).pin_memory()
    dev_in = torch.from_numpy(A).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2

    def step():
        tn.tn_batch_run(b, 1.0, hs)

    # inputs resident in HBM
    tn.tn_batch_set_tensors_device(b, dev_in, n_in)
    for _ in range(max(3, args.warmup)):
        step()
    torch.cuda.synchronize()
    launches_per_step = tn.tn_batch_launch_count(b)

    # ---- timed region: device time, L2 flushed between steps
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, args.clock_log) as clk:
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(s))
            ev[s][0].record(stream)
            step()
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = [a.elapsed_time(e) for a, e in ev]
    t_total = max_over_ranks(sum(ms) / 1000.0, ws)
    value = job_rate(ws, B, args.steps, t_total)
    res = tn.tn_batch_results_host(b)

    # ---- end to end through the C-ABI with host buffers
    def e2e_step():
        tn.lib().tn_batch_set_tensors(b, tn.c_void_p(host_in.data_ptr()), n_in)
        tn.tn_batch_run(b, 1.0, hs)
        tn.lib().tn_batch_results_host(b, tn.c_void_p(host_out.data_ptr()), n_res)

    for _ in range(2):
        e2e_step()
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": job_rate(ws, B, args.steps, t_e2e), "unit": "lattice evals/s",
           "h2d_bytes_per_step": int(n_in * 8), "d2h_bytes_per_step": int(n_res * 8)}

    # ---- per-kernel-family time with CUDA events around every launch (separate pass)
    tn.tn_ctx_set_profiling(ctx, True)
    for _ in range(3):
        step()
    torch.cuda.synchronize()
    fams = {name: tn.tn_ctx_kernel_stats(ctx, k) for k, name in
            enumerate(["absorb", "absorb_dot", "gemm_simt", "gemm_tc", "other", "absorb_pair"])}
    tn.tn_ctx_set_profiling(ctx, False)
    hbm, bf16, sm_max, src = _peaks()
    bf16_sus = _peak_key("bf16_tflops_sustained", bf16)
    dom = max(fams, key=lambda k: fams[k]["ms"])
    products = {"bf16x3": 3, "bf16x6": 6}.get(args.precision, 1)

    def roofline_of(name):
        fd = fams[name]
        if not fd["ms"]:
            return None
        if name in ("absorb", "absorb_dot", "other", "absorb_pair"):
            achieved = fd["bytes"] / (fd["ms"] / 1e3) / 1e9
            traffic, note = None, None
            if name == "absorb" and prec == tn.TN_FP32:
                # DRAM bytes per algorithmic byte of the interior FP32 absorption,
                # from one ncu capture (8x8 D=2, 64 lattices: 89.4 MB of DRAM
                # traffic for 134.2 MB in + out), applied to this run's average launch
                traffic = ABSORB_DRAM_PER_BYTE * fd["bytes"] / fd["launches"]
                note = "ncu dram bytes/algorithmic bytes of one interior launch x mean bytes per launch"
            r = {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s", "frac": achieved / hbm,
                 "traffic": traffic, "kernel": name,
                 "peak_source": f"{src} MEASURED_PEAKS.json hbm_gbs (of {src})"}
            if note:
                r["traffic_source"] = note
            return r
        if name == "gemm_tc":
            algo = 2 * fd["macs"] / (fd["ms"] / 1e3) / 1e12
            achieved = products * algo
            return {"bound": "tensor", "achieved": achieved, "peak": bf16_sus, "unit": "TFLOP/s",
                    "frac": achieved / bf16_sus, "traffic": None, "kernel": name,
                    "algorithmic_tflops": algo, "tensor_products_per_mac": products,
                    "peak_source": f"MEASURED_PEAKS.json bf16_tflops_sustained (of {src})"}
        achieved = 2 * fd["macs"] / (fd["ms"] / 1e3) / 1e12
        if esize == 8:
            peak = 152 * 64 * 2 * sm_max * 1e6 / 1e12 / 32    # FP64: 1/64 of the FP32 lane rate
        else:
            peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12        # FP32 FMA lanes x 2 flop x max clock
        r = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
             "traffic": None, "kernel": name,
             "peak_source": "152 SMs x 128 FP32 lanes x 2 flop x sm_max clock (derived)"}
        if name == "gemm_simt" and prec == tn.TN_FP32 and fd["launches"]:
            # DRAM bytes per multiply-add of the batched 256^3 products, from one
            # ncu capture (640 products: 373.1 MB), times this run's mean per launch
            r["traffic"] = GEMM_DRAM_PER_MAC * fd["macs"] / fd["launches"]
            r["traffic_source"] = "ncu dram bytes/multiply-add of one product launch x mean multiply-adds per launch"
        return r

    esize = 4 if prec != tn.TN_FP64 else 8
    roof = roofline_of(dom)
    roof_absorb = roofline_of("absorb")
    per_launch = {k: {"launches": v["launches"] / 3, "ms": v["ms"] / 3,
                      "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] else 0.0,
                      "TFLOPs": (2 * v["macs"] / (v["ms"] / 1e3) / 1e12) if v["ms"] else 0.0}
                  for k, v in fams.items() if v["launches"]}

    line = {"metric": METRIC, "value": value, "unit": "lattice evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "f32+bf16x3", "bf16x6": "f32+bf16x6"}[args.precision],
            "data": "synthetic: seeded uniform[-1,1) site tensors (SplitMix64), fresh seeds per rank",
            "config": {"workload": WORKLOAD, "batch": B, "L": L_, "W": W_, "D": D_, "h": list(H_FIELDS),
                       "schedule": "auto (paper's min-bottleneck cut)",
                       "l2": "flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "energies_per_s": value * len(H_FIELDS),
            "e2e": e2e, "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roof, "roofline_absorb": roof_absorb, "kernel_families": per_launch,
            "clocks": clk.summary(),
            "sample_energy": float(res[0])}
    if rank == 0 and not args.no_extras:
        # FP64 GPU path on the same workload (the plain path the reduced precisions must beat)
        if prec != tn.TN_FP64:
            b64 = tn.tn_batch_create(ctx, [L_] * B, [W_] * B, [D_] * B, tn.TN_FP64)
            tn.tn_batch_set_tensors_device(b64, dev_in, n_in)
            for _ in range(2):
                tn.tn_batch_run(b64, 1.0, hs)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(3):
                tn.tn_batch_run(b64, 1.0, hs)
            e1.record(stream)
            torch.cuda.synchronize()
            r64 = tn.tn_batch_results_host(b64)
            t64 = e0.elapsed_time(e1) / 3 / 1e3
            stride = n_res // B     # per member: header, <X_k>, <Z_i Z_j>, <Z_k>
            rel = float(np.max(np.abs(res[0::stride][:B] - r64[0::stride][:B]) /
                               np.maximum(1.0, np.abs(r64[0::stride][:B]))))
            line["fp64_gpu"] = {"value": B / t64, "unit": "lattice evals/s",
                                "max_rel_energy_err_vs_fp64": rel}
            tn.tn_batch_destroy(b64)
        line["roofline_absorb_stream"] = absorb_stream_roofline(ctx, stream, hbm, src)
        line["cpu_baseline"] = cpu_baseline(args.cpu_lattices, 4242)
    tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
