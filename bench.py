"""Benchmark: exact Ising-PEPS energy evaluations per second on GB300.

Headline workload (one "step", the default): the two large single instances,
a 12x12 PEPS of bond D = 2 and an 8x8 PEPS of bond D = 3 (seeded uniform[-1,1)
site tensors), each contracted exactly in FP64 into its norm, every <X_k>,
every <Z_k> and every nearest-neighbour <Z_i Z_j>, from which E is formed at
any h (reported at h = 3.04, J = 1).  Both lattices run as one batch (one
replayed CUDA graph of grouped launches); the whole hot path -- site matrices,
corner chains, ring closure, environments, observable insertions, FP64 ratios
-- runs in libtn's kernels.

value  : lattice energy evaluations/s (2 per step), inputs resident in HBM,
         CUDA events on the library's stream; the step's working set (~23 GB)
         is far above L2, which is also flushed (256 MB write) between steps.
e2e    : the same metric through the C-ABI with host buffers: per step the
         pinned host tensors are copied in, the batch runs, the result array is
         read back (3 steps).
extras : the FP32 / BF16x6 / BF16x3 rates of the same workload with their energy
         errors against this run's FP64 results and against stored oracle
         samples; the 8x8 D=2 batch (256 lattices); a short served stream; the
         FP64 oracle timed on a bounded sample of the workload (cpu_baseline).
--impl reference: the FP64 CPU oracle on the host cores (bounded samples).
Other workloads: --workload 8x8 | serve | batch | case (see --help).
Multi-GPU (torchrun): each rank runs its own lattices (replicas, weak scaling).
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

METRIC = "exact LxL Ising-PEPS energy evals/s"
LARGE = ((12, 12, 2), (8, 8, 3))
LARGE_SEEDS = (1212, 883)          # rank 0: the lattices whose oracle samples are stored in tests/golden
H_LARGE = 3.04
WORKLOAD = "large single instances: 12x12 D=2 and 8x8 D=3 TFIM-PEPS energies"
GOLDEN = os.path.join(ROOT, "tests", "golden", "large_samples.json")
L_, W_, D_ = 8, 8, 2               # the 8x8 D=2 batch workload
H_FIELDS = (2.0, 3.04, 4.0)
WORKLOAD_8X8 = "8x8 open-boundary TFIM PEPS, D=2, E at h in {2.0, 3.04, 4.0}"
FAMILIES = ["absorb", "absorb_dot", "gemm_simt", "gemm_tc", "other", "absorb_pair"]
# DRAM bytes per algorithmic byte of one interior k_absorb4<16,16,1,0> launch (ncu dram__bytes_read.sum +
# dram__bytes_write.sum, `bench.py --workload case --batch 64 --precision fp32`, 8x8 D=2 lattices)
ABSORB_DRAM_PER_BYTE = 86.88 / 134.22
# DRAM bytes per multiply-add of one k_gemm3<1,0,1> launch (640 products of 256^3, the same capture command)
GEMM_DRAM_PER_MAC = 373.1e6 / (640 * 256.0 ** 3)


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


# ----------------------------------------------------------------- helpers --

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


def large_seeds(rank: int):
    """Seeds of a rank's two large lattices: rank 0 takes the ones with stored
    oracle samples, every other rank fresh ones."""
    if rank == 0:
        return list(LARGE_SEEDS)
    from paper_1908_08553_gb300 import inputs
    return [inputs.lattice_seed(replica_seed(rank), k) for k in range(len(LARGE))]


def _dist():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


def split_results(res, shapes):
    """Per-member views of a batch's result array (layout of tn_batch_results_host)."""
    out, off = [], 0
    for (L, W, _D) in shapes:
        nb = L * (W - 1) + W * (L - 1)
        n = 6 + 2 * L * W + nb
        seg = res[off:off + n]
        off += n
        out.append({"E": float(seg[0]), "log2_norm": float(seg[1]), "sum_x": float(seg[4]),
                    "sum_zz": float(seg[5]), "sx": seg[6:6 + L * W], "zz": seg[6 + L * W:6 + L * W + nb],
                    "sz": seg[6 + L * W + nb:n]})
    return out


def energy_errors(got, ref, J: float, h: float):
    """|dE| / |E|, |dE| / S with S = |J| sum |<ZZ>| + |h| sum |<X>| (the energy's
    scale), and the largest per-term difference, for one lattice."""
    import numpy as np
    E_ref = -J * ref["sum_zz"] - h * ref["sum_x"]
    E = -J * got["sum_zz"] - h * got["sum_x"]
    S = abs(J) * float(np.abs(ref["zz"]).sum()) + abs(h) * float(np.abs(ref["sx"]).sum())
    d = abs(E - E_ref)
    term = max(float(np.max(np.abs(got["sx"] - ref["sx"]))), float(np.max(np.abs(got["zz"] - ref["zz"]))) if
               len(ref["zz"]) else 0.0)
    return {"rel": d / abs(E_ref) if E_ref else float("inf"), "rel_scale": d / S if S else d, "max_term": term,
            "scale_over_abs_E": S / abs(E_ref) if E_ref else float("inf")}


def worst(errs):
    return {k: max(e[k] for e in errs) for k in ("rel", "rel_scale", "max_term")}


def golden_errors(members, shapes, seeds):
    """Differences from the stored FP64 oracle samples (tests/golden/large_samples.json,
    written by a script that calls only the oracle) for the lattices that have them."""
    import math
    try:
        with open(GOLDEN) as f:
            cases = json.load(f)["cases"]
    except OSError:
        return None
    from paper_1908_08553_gb300 import inputs
    out = {}
    for m, (L, W, D), seed in zip(members, shapes, seeds):
        case = next((c for c in cases if (c["L"], c["W"], c["D"], c["seed"]) == (L, W, D, seed)), None)
        if case is None:
            continue
        bonds = [(a[0] * W + a[1], b[0] * W + b[1]) for a, b in inputs.bonds(L, W)]
        dmax = 0.0
        for s in case["samples"]:
            got = m["sx"][s["i"]] if s["op"] == "x" else m["zz"][bonds.index((s["i"], s["j"]))]
            dmax = max(dmax, abs(got - s["value"]))
        s0 = case["samples"][0]
        lg = math.log2(abs(s0["norm_mant"])) + s0["norm_exp2"]
        out[f"{L}x{W}_D{D}"] = {"samples": len(case["samples"]), "max_abs_diff": dmax,
                                "log2_norm_rel_diff": abs(m["log2_norm"] - lg) / abs(lg)}
    return out


def timed_runs(tn, torch, b, hs, stream, warm: int, reps: int) -> float:
    """Mean ms of `reps` runs after `warm` runs (CUDA events on the library's stream)."""
    for _ in range(warm):
        tn.tn_batch_run(b, 1.0, hs)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(reps):
        tn.tn_batch_run(b, 1.0, hs)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def family_stats(tn, torch, ctx, b, hs, runs: int = 1):
    """Per kernel family: launches, ms, bytes, multiply-adds per run (CUDA events
    around every launch in a separate, synchronised pass)."""
    tn.tn_ctx_set_profiling(ctx, True)
    for _ in range(runs):
        tn.tn_batch_run(b, 1.0, hs)
    torch.cuda.synchronize()
    fams = {name: tn.tn_ctx_kernel_stats(ctx, k) for k, name in enumerate(FAMILIES)}
    tn.tn_ctx_set_profiling(ctx, False)
    for v in fams.values():
        for k in ("launches", "ms", "bytes", "macs"):
            v[k] = v[k] / runs
    return fams


def roofline_of(fam: dict, name: str, prec_name: str, peaks: dict):
    """Roofline entry of one kernel family: HBM for the absorption families, the
    measured FMA rate for SIMT products, the measured BF16 rate for tensor cores."""
    fd = fam[name]
    if not fd["ms"]:
        return None
    if name in ("absorb", "absorb_dot", "other", "absorb_pair") and prec_name != "fp64":
        achieved = fd["bytes"] / (fd["ms"] / 1e3) / 1e9
        r = {"bound": "hbm", "achieved": achieved, "peak": peaks["hbm"], "unit": "GB/s",
             "frac": achieved / peaks["hbm"], "traffic": None, "kernel": name,
             "peak_source": f"MEASURED_PEAKS.json hbm_gbs (of {peaks['src']})"}
        if name == "absorb" and prec_name == "fp32":
            r["traffic"] = ABSORB_DRAM_PER_BYTE * fd["bytes"] / fd["launches"]
            r["traffic_source"] = ("ncu dram bytes / algorithmic bytes of one interior 8x8 D=2 launch x this "
                                   "run's mean algorithmic bytes per launch")
        return r
    if name == "gemm_tc":
        products = {"bf16x3": 3, "bf16x6": 6}.get(prec_name, 1)
        algo = 2 * fd["macs"] / (fd["ms"] / 1e3) / 1e12
        achieved = products * algo
        return {"bound": "tensor", "achieved": achieved, "peak": peaks["bf16_sus"], "unit": "TFLOP/s",
                "frac": achieved / peaks["bf16_sus"], "traffic": None, "kernel": name,
                "algorithmic_tflops": algo, "tensor_products_per_mac": products,
                "peak_source": f"MEASURED_PEAKS.json bf16_tflops_sustained (of {peaks['src']})"}
    achieved = 2 * fd["macs"] / (fd["ms"] / 1e3) / 1e12
    peak = peaks["fp64"] if prec_name == "fp64" else peaks["fp32"]
    return {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": None, "kernel": name,
            "peak_source": ("measured in this run: tn_peak_probe, " +
                            ("FP64 fma" if prec_name == "fp64" else "FP32 fma.rn.f32x2") +
                            ", 2048 threads per SM, 8 chains each")}


# ------------------------------------------------------------ CPU baseline --

# Bounded samples of the oracle's row sweep: full rows, then the first sites of
# the next row (the rows after the first cost about the same).
ORACLE_SAMPLE = {(12, 12, 2): (1, 6), (8, 8, 3): (1, 2)}


def oracle_sample(shape, seed):
    """Time the oracle on a bounded part of one lattice's row sweep; return
    (seconds, sampled multiply-adds, multiply-adds of the lattice's full energy
    evaluation, estimated seconds of that evaluation at the sampled rate)."""
    import oracle
    from paper_1908_08553_gb300 import inputs
    L, W, D = shape
    nrows, ncols = ORACLE_SAMPLE[shape]
    A = inputs.random_lattice(L, W, D, seed)
    t0 = time.perf_counter()
    oracle.sweep_rows(L, W, D, A, nrows, ncols)
    dt = time.perf_counter() - t0
    macs = oracle.sweep_macs(L, W, D, nrows, ncols)
    full = oracle.energy_macs(L, W, D)
    return dt, macs, full, dt * full / macs


def cpu_baseline(seeds):
    """The FP64 oracle, as it stands, on a bounded sample of the headline workload."""
    import oracle
    total_s, parts, sample_s = 0.0, [], 0.0
    for shape, seed in zip(LARGE, seeds):
        dt, macs, full, est = oracle_sample(shape, seed)
        total_s += est
        sample_s += dt
        nr, nc = ORACLE_SAMPLE[shape]
        parts.append(f"{shape[0]}x{shape[1]} D={shape[2]}: {nr} row(s) + {nc} site(s) of the row sweep, "
                     f"{macs:.3g} MAC in {dt:.1f} s ({macs / dt / 1e9:.2f} GMAC/s), scaled to the "
                     f"{full:.3g} MAC of its energy evaluation")
    return {"value": len(LARGE) / total_s, "unit": "lattice evals/s", "cores": oracle.num_threads(),
            "kind": "oracle",
            "sample": "; ".join(parts) + f" ({sample_s:.1f} s of CPU work in all; the full evaluations "
                                         f"would take {total_s / 3600:.1f} h)"}


def run_reference(args):
    """The reference arm: the FP64 oracle on the host cores, on the headline
    workload; each step is a bounded sample (the 12x12 D=2 lattice on even
    steps, the 8x8 D=3 lattice on odd ones), scaled to lattice evals/s by the
    multiply-adds of the full energy evaluations."""
    ws, rank, _ = _dist()
    if rank != 0:
        return 0
    import oracle
    seeds = list(LARGE_SEEDS)
    for s in range(args.warmup):
        oracle_sample(LARGE[s % 2], seeds[s % 2])
    spent = [0.0, 0.0]
    full_s = [0.0, 0.0]
    count = [0, 0]
    t0 = time.perf_counter()
    for s in range(args.steps):
        k = s % 2
        dt, macs, full, est = oracle_sample(LARGE[k], seeds[k])
        spent[k] += dt
        full_s[k] += est
        count[k] += 1
    wall = time.perf_counter() - t0
    # estimated seconds of one energy evaluation of each lattice, averaged over its samples
    per = [full_s[k] / max(1, count[k]) for k in range(2)]
    value = len(LARGE) / sum(per)
    line = {"metric": METRIC, "value": value, "unit": "lattice evals/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * wall / max(1, args.steps),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic: seeded uniform[-1,1) site tensors", "impl": "reference",
            "config": {"workload": WORKLOAD, "lattices": ["12x12 D=2", "8x8 D=3"], "h": H_LARGE,
                       "schedule": "row sweep (the oracle's order)"},
            "cpu_baseline": {"value": value, "unit": "lattice evals/s", "cores": oracle.num_threads(),
                             "kind": "oracle",
                             "sample": ("per step one bounded part of one lattice's FP64 row sweep (12x12 D=2: "
                                        "1 row + 6 sites; 8x8 D=3: 1 row + 2 sites; alternating), its "
                                        "multiply-add rate applied to the multiply-adds of the lattice's full "
                                        f"energy evaluation; estimated {per[0]:.0f} s and {per[1]:.0f} s per "
                                        "evaluation")},
            "e2e": {"value": value, "unit": "lattice evals/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- headline --

def run_headline(args):
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
    prec_name = args.precision or "fp64"
    prec = tn.PRECISIONS[prec_name]
    shapes = list(LARGE)
    seeds = large_seeds(rank)
    Ls, Ws, Ds = zip(*shapes)
    hs = np.full(len(shapes), H_LARGE)
    b = tn.tn_batch_create(ctx, Ls, Ws, Ds, prec)
    n_in = tn.tn_batch_elems(b)
    A = np.concatenate([inputs.random_lattice(L, W, D, s) for (L, W, D), s in zip(shapes, seeds)])
    host_in = torch.empty(n_in, dtype=torch.float64).pin_memory()
    host_in.numpy()[:] = A
    n_res = tn.tn_batch_result_size(b)
    host_out = torch.empty(n_res, dtype=torch.float64).pin_memory()
    dev_in = torch.from_numpy(A).cuda()
    flush = torch.empty(64 * 1024 * 1024, dtype=torch.float32, device="cuda")   # 256 MB > 129 MB L2

    tn.tn_batch_set_tensors_device(b, dev_in, n_in)
    for _ in range(max(3, args.warmup)):
        tn.tn_batch_run(b, 1.0, hs)
    torch.cuda.synchronize()
    launches_per_step = tn.tn_batch_launch_count(b)

    # ---- timed region: device time on the library's stream
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, args.clock_log) as clk:
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(s))
            ev[s][0].record(stream)
            tn.tn_batch_run(b, 1.0, hs)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    ms = [a.elapsed_time(e) for a, e in ev]
    t_total = max_over_ranks(sum(ms) / 1000.0, ws)
    value = job_rate(ws, len(shapes), args.steps, t_total)
    res = tn.tn_batch_results_host(b).copy()
    members = split_results(res, shapes)

    # ---- end to end through the C-ABI with host buffers
    def e2e_step():
        tn.check(tn.lib().tn_batch_set_tensors(b, tn.c_void_p(host_in.data_ptr()), n_in), "set tensors")
        tn.tn_batch_run(b, 1.0, hs)
        tn.check(tn.lib().tn_batch_results_host(b, tn.c_void_p(host_out.data_ptr()), n_res), "results")

    n_e2e = max(1, min(args.steps, args.e2e_steps))
    e2e_step()
    if ws > 1:
        torch.distributed.barrier()
    t0 = time.perf_counter()
    for _ in range(n_e2e):
        e2e_step()
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    e2e = {"value": job_rate(ws, len(shapes), n_e2e, t_e2e), "unit": "lattice evals/s",
           "h2d_bytes_per_step": int(n_in * 8), "d2h_bytes_per_step": int(n_res * 8), "steps": n_e2e}

    # ---- per-family device time (separate pass) and measured peaks
    fams = family_stats(tn, torch, ctx, b, hs)
    hbm, bf16, sm_max, src = _peaks()
    peaks = {"hbm": hbm, "bf16": bf16, "bf16_sus": _peak_key("bf16_tflops_sustained", bf16), "src": src,
             "fp64": tn.tn_peak_probe(ctx, 0), "fp32": tn.tn_peak_probe(ctx, 1)}
    dom = max(fams, key=lambda k: fams[k]["ms"])
    roof = roofline_of(fams, dom, prec_name, peaks)
    per_family = {k: {"launches": v["launches"], "ms": v["ms"],
                      "GBps": (v["bytes"] / (v["ms"] / 1e3) / 1e9) if v["ms"] else 0.0,
                      "TFLOPs": (2 * v["macs"] / (v["ms"] / 1e3) / 1e12) if v["ms"] else 0.0}
                  for k, v in fams.items() if v["launches"]}
    props = torch.cuda.get_device_properties(local)
    dtype = {"fp64": "f64", "fp32": "f32", "bf16x3": "f32+bf16x3", "bf16x6": "f32+bf16x6"}[prec_name]
    line = {"metric": METRIC, "value": value, "unit": "lattice evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": dtype,
            "data": "synthetic: seeded uniform[-1,1) site tensors (SplitMix64); rank 0 the lattices with stored "
                    "oracle samples, other ranks fresh seeds",
            "config": {"workload": WORKLOAD, "lattices": ["12x12 D=2", "8x8 D=3"], "h": H_LARGE,
                       "outputs": "norm, every <X_k>, <Z_k>, nearest-neighbour <Z_i Z_j>, E",
                       "schedule": "auto (paper's min-bottleneck cut: quadrant (6,6) and (4,4))",
                       "l2": "working set ~23 GB >> L2; also flushed between timed steps (256 MB write)",
                       "parallelism": f"replicas x{ws}"},
            "e2e": e2e, "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roof, "kernel_families": per_family,
            "peaks_measured": {"fp64_tflops": peaks["fp64"], "fp32_tflops": peaks["fp32"],
                               "sms": props.multi_processor_count},
            "clocks": clk.summary(),
            "energies": {f"{L}x{W}_D{D}": {"E": m["E"], "E_per_site": m["E"] / (L * W), "log2_norm": m["log2_norm"]}
                         for m, (L, W, D) in zip(members, shapes)}}
    if rank == 0:
        line["vs_oracle_samples"] = golden_errors(members, shapes, seeds)
    if rank == 0 and not args.no_extras:
        line["precisions"] = other_precisions(tn, torch, ctx, stream, shapes, A, hs, members, seeds, prec_name,
                                              peaks)
        line["roofline_absorb_stream"] = absorb_stream_roofline(ctx, stream, hbm, src)
        line["batch_8x8_d2"] = batch_8x8(tn, torch, ctx, stream, args.batch)
        if args.serve_requests > 0:
            line["serving"] = serve_stream(args.serve_requests, args.calibrate, "bf16x6", seq_seconds=20.0)
        line["next_rows"] = next_rows(tn, torch, ctx)
        line["cpu_baseline"] = cpu_baseline(seeds)
        line["cpu_baseline"]["next_rows_oracle"] = next_rows_oracle()
    tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def other_precisions(tn, torch, ctx, stream, shapes, A, hs, ref_members, seeds, ref_prec, peaks):
    """Reduced precisions on the headline lattices: rate, energy errors against
    this run's FP64 results and against the stored oracle samples; the FP32
    run's absorption family as an HBM roofline."""
    out = {}
    Ls, Ws, Ds = zip(*shapes)
    for name in ("fp32", "bf16x6", "bf16x3"):
        if name == ref_prec:
            continue
        b = tn.tn_batch_create(ctx, Ls, Ws, Ds, tn.PRECISIONS[name])
        try:
            tn.tn_batch_set_tensors(b, A)
            ms = timed_runs(tn, torch, b, hs, stream, 2, 3)
            mem = split_results(tn.tn_batch_results_host(b).copy(), shapes)
            entry = {"value": len(shapes) / (ms / 1e3), "unit": "lattice evals/s", "ms_per_step": ms,
                     "per_lattice_ms": None}
            if ref_prec == "fp64":
                errs = [energy_errors(m, r, 1.0, H_LARGE) for m, r in zip(mem, ref_members)]
                entry["vs_fp64_gpu"] = {f"{L}x{W}_D{D}": e for e, (L, W, D) in zip(errs, shapes)}
            entry["vs_oracle_samples"] = golden_errors(mem, shapes, seeds)
            fams = family_stats(tn, torch, ctx, b, hs)
            entry["kernel_families_ms"] = {k: v["ms"] for k, v in fams.items() if v["launches"]}
            if name == "fp32":
                entry["roofline_absorb"] = roofline_of(fams, "absorb", "fp32", peaks)
                entry["roofline_products"] = roofline_of(fams, "gemm_simt", "fp32", peaks)
            else:
                entry["roofline_products"] = roofline_of(fams, "gemm_tc", name, peaks)
            # each lattice alone, for the per-lattice time
            per = {}
            for k, (L, W, D) in enumerate(shapes):
                b1 = tn.tn_batch_create(ctx, [L], [W], [D], tn.PRECISIONS[name])
                try:
                    off = sum(tn.tn_lattice_elems(*s) for s in shapes[:k])
                    tn.tn_batch_set_tensors(b1, A[off:off + tn.tn_lattice_elems(L, W, D)])
                    per[f"{L}x{W}_D{D}"] = timed_runs(tn, torch, b1, hs[:1], stream, 1, 3)
                finally:
                    tn.tn_batch_destroy(b1)
            entry["per_lattice_ms"] = per
            out[name] = entry
        finally:
            tn.tn_batch_destroy(b)
    return out


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
            "peak_source": f"MEASURED_PEAKS.json hbm_gbs (of {src})"}


def batch_8x8(tn, torch, ctx, stream, B: int):
    """The 8x8 D=2 batch (B lattices, h in {2.0, 3.04, 4.0}): rate per precision and
    the largest energy errors against the FP64 GPU results of the same batch."""
    import numpy as np

    from paper_1908_08553_gb300 import inputs
    hs = np.array([H_FIELDS[k % 3] for k in range(B)])
    A = np.concatenate([inputs.random_lattice(L_, W_, D_, inputs.lattice_seed(replica_seed(0), k))
                        for k in range(B)])
    shapes = [(L_, W_, D_)] * B
    out, ref = {"lattices": B, "h": list(H_FIELDS)}, None
    for name in ("fp64", "fp32", "bf16x6", "bf16x3"):
        b = tn.tn_batch_create(ctx, [L_] * B, [W_] * B, [D_] * B, tn.PRECISIONS[name])
        try:
            tn.tn_batch_set_tensors(b, A)
            ms = timed_runs(tn, torch, b, hs, stream, 3, 5)
            mem = split_results(tn.tn_batch_results_host(b).copy(), shapes)
        finally:
            tn.tn_batch_destroy(b)
        entry = {"value": B / (ms / 1e3), "unit": "lattice evals/s", "ms_per_batch": ms}
        if ref is None:
            ref = mem
        else:
            entry["vs_fp64_gpu"] = worst([energy_errors(m, r, 1.0, hs[k]) for k, (m, r) in enumerate(zip(mem, ref))])
        out[name] = entry
    return out


# ---------------------------------------------------------------- next rows --

def next_rows(tn, torch, ctx) -> dict:
    """The ranked next rows on the GPU: every pair correlator of an 8x8 D=2
    lattice in one call, a complex 8x8 D=2 energy with every <Y_k>, the
    boundary-MPS energy at chi_b = 16 against the exact one, and imaginary time
    evolution of a 6x6 lattice.  Errors are against the FP64 GPU results (the
    oracle parity of these paths is in the tests); the oracle's times on the
    same jobs are in the CPU-baseline leg (next_rows_oracle)."""
    import numpy as np

    from paper_1908_08553_gb300 import inputs

    def wall(f, reps=1):
        f()                                  # warm-up (programs, caches)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            r = f()
        torch.cuda.synchronize()
        return (time.perf_counter() - t0) / reps, r

    out = {}
    L, W, D = 8, 8, 2
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        # f2: all 2016 pairs <Z_i Z_j>, one program built and run per call
        tn.tn_set_site_tensors(lat, inputs.random_lattice(L, W, D, 8801))
        ij = np.array([(i, j) for i in range(N) for j in range(i + 1, N)], dtype=np.int32)
        pairs, ref = {"pairs": int(ij.shape[0])}, None
        for name in ("fp64", "fp32"):
            prec = tn.PRECISIONS[name]
            dt, v = wall(lambda: tn.tn_pair_correlators(lat, prec, tn.TN_OP_Z, tn.TN_OP_Z, ij[:, 0], ij[:, 1]))
            pairs[name] = {"s_per_call": dt, "pairs_per_s": ij.shape[0] / dt}
            if ref is None:
                ref = v
            else:
                pairs[name]["max_abs_diff_vs_fp64"] = float(np.abs(v - ref).max())
        out["f2_pairs_8x8_d2"] = pairs
        # f2: complex PEPS energy with every <X>, <Y>, <Z>, <ZZ>
        tn.tn_set_site_tensors_complex(lat, inputs.random_complex_lattice(L, W, D, 8802))
        cplx, ref = {}, None
        for name in ("fp64", "bf16x6"):
            prec = tn.PRECISIONS[name]

            def run():
                r, sx, zz, sz, _ = tn.tn_energy_full(lat, 1.0, 3.04, prec, tn.TN_SCHED_AUTO, L, W)
                sy = tn.tn_site_expectations(lat, prec, tn.TN_OP_Y, L, W)
                return np.concatenate([sx, sy, sz, zz])
            dt, v = wall(run)
            cplx[name] = {"s_per_eval": dt, "evals_per_s": 1.0 / dt}
            if ref is None:
                ref = v
            else:
                cplx[name]["max_abs_diff_vs_fp64"] = float(np.abs(v - ref).max())
        out["f2_complex_8x8_d2"] = cplx
        # f3: boundary MPS at chi_b = 16 against the exact FP64 energy
        tn.tn_set_site_tensors(lat, inputs.random_lattice(L, W, D, 8801))
        exact = tn.tn_energy(lat, 1.0, 3.04, tn.TN_FP64)
        bmps = {"networks": N + nb + 1}
        for name in ("fp64", "fp32"):
            dt, (r, _, _) = wall(lambda: tn.tn_bmps_energy(lat, 16, 1.0, 3.04, L, W, tn.PRECISIONS[name]))
            bmps[name] = {"s_per_energy": dt,
                          "rel_energy_err_vs_exact": abs(r.energy - exact.energy) / abs(exact.energy)}
        out["f3_bmps_8x8_d2_chi16"] = bmps
    finally:
        tn.tn_destroy_lattice(lat)
    # f4: ITE, 6x6, chi_max = 2, Gamma = 3.04, dtau = 0.05, 20 steps, energy every 10
    Li, Wi, chi, steps = 6, 6, 2, 20
    lat = tn.tn_create_lattice(ctx, Li, Wi, chi)
    try:
        def ite_run():
            tn.tn_ite_init_product(lat)
            return tn.tn_ite_run(lat, Li, Wi, 1.0, 3.04, 0.05, steps, chi, 1e-3, energy_every=10)
        dt, (en, dims, disc) = wall(ite_run)
    finally:
        tn.tn_destroy_lattice(lat)
    out["f4_ite_6x6_chi2"] = {"steps": steps, "s_per_step": dt / steps, "energy_per_site": float(en[-1]) / (Li * Wi)}
    return out


def next_rows_oracle() -> dict:
    """The oracle, as it stands, on the next rows' jobs (CPU-baseline leg):
    bounded samples scaled to each job, the sample stated."""
    import oracle
    import oracle.bmps as bm
    import oracle.complex_peps as cp
    import oracle.ite as ite
    from paper_1908_08553_gb300 import inputs

    L, W, D = 8, 8, 2
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    A = inputs.random_lattice(L, W, D, 8801)
    t0 = time.perf_counter()
    for i, j in ((0, 63), (7, 56), (27, 36)):
        oracle.pair(L, W, D, A, "z", i, "z", j)
    per_pair = (time.perf_counter() - t0) / 3
    Ac = inputs.random_complex_lattice(L, W, D, 8802)
    t0 = time.perf_counter()
    cp.value(L, W, D, Ac)
    per_contraction = time.perf_counter() - t0
    t0 = time.perf_counter()
    bm.norm(L, W, D, A, 16)
    per_network = time.perf_counter() - t0
    t0 = time.perf_counter()
    ite.evolve(6, 6, 1.0, 3.04, 0.05, 20, 2, 1e-3, energy_every=10)
    ite_s = time.perf_counter() - t0
    return {"f2_pairs_8x8_d2": {"pairs_per_s": 1.0 / per_pair, "sample": "3 pairs, one row sweep each"},
            "f2_complex_8x8_d2": {"s_per_eval": per_contraction * (3 * N + nb + 1),
                                  "sample": "one complex128 contraction x the 3N + nb + 1 contractions"},
            "f3_bmps_8x8_d2_chi16": {"s_per_energy": per_network * (N + nb + 1),
                                     "sample": "one numpy boundary-MPS network x the N + nb + 1 networks"},
            "f4_ite_6x6_chi2": {"s_per_step": ite_s / 20, "sample": "the same 20 steps (numpy)"},
            "cores": os.cpu_count()}


def run_next(args):
    import torch

    from paper_1908_08553_gb300 import tn
    torch.cuda.set_device(0)
    ctx = tn.tn_ctx_create(0, 0)
    line = {"metric": "next rows: pair correlators, complex PEPS, boundary MPS, ITE", "unit": "s",
            "higher_is_better": False, "data": "synthetic: seeded uniform[-1,1) site tensors",
            "results": next_rows(tn, torch, ctx)}
    tn.tn_ctx_destroy(ctx)
    line["cpu_baseline"] = {"kind": "oracle", "next_rows_oracle": next_rows_oracle()}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ serving --

def serve_stream(n: int, calibrate: int, precision: str, seq_seconds: float, recompute: bool = False) -> dict:
    """Serving: a Poisson stream of requests (L, W ~ U{4..12}, D ~ U{2,3},
    h ~ U[0.5, 5], seeded tensors) at 80% of the measured capacity, admitted by
    exact footprint against a 160 GB budget; p50/p99 latency and throughput,
    beside sequential FP64 solves of the same requests (the lighter ones).
    recompute: shapes whose cached-state program exceeds the budget are served
    in the recompute form (program choice bit 5 set in the tuning table)."""
    import threading

    import numpy as np
    import torch

    from paper_1908_08553_gb300 import tn

    prec = tn.PRECISIONS[precision]
    budget = int(160e9)
    rng = np.random.default_rng(3)
    reqs = [(int(rng.integers(4, 13)), int(rng.integers(4, 13)), int(rng.choice([2, 3])),
             float(rng.uniform(0.5, 5.0)), 10_000 + k) for k in range(n + calibrate)]
    ctx = tn.tn_ctx_create(torch.cuda.current_device(), budget)
    probe = tn.tn_ctx_create(-1)
    recompute_shapes = []
    if recompute:
        for (L, W, D) in sorted({r[:3] for r in reqs}):
            lat = tn.tn_create_lattice(probe, L, W, D)
            if tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY) > budget:
                tn.tn_autotune_set(L, W, D, prec, tn.TN_WORK_ENERGY, 15 | 32)
                if tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY) <= budget:
                    recompute_shapes.append((L, W, D))
                else:
                    tn.tn_autotune_set(L, W, D, prec, tn.TN_WORK_ENERGY, 15)
            tn.tn_destroy_lattice(lat)
    fits = []
    for (L, W, D, h, seed) in reqs:
        lat = tn.tn_create_lattice(probe, L, W, D)
        fits.append(tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY) <= budget)
        tn.tn_destroy_lattice(lat)
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
    pending, done, lock, shapes_of, ticket_of = {}, {}, threading.Lock(), {}, {}
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
            shapes_of[t] = (L, W, D)
        ticket_of[(L, W, D, h, sd)] = t
    stop.set()
    th.join()
    t_end = max(v[1] for v in done.values())
    lat = np.array([v[1] - v[0] for v in done.values()])
    lat_d = {d: np.array([v[1] - v[0] for t, v in done.items() if shapes_of[t][2] == d]) for d in (2, 3)}
    served = len(done)

    # sequential plain FP64 solves of the served requests in stream order, one
    # at a time, skipping those whose FP64 products exceed 5e12 multiply-adds
    # (minutes each at the GB300's FP64 rate), until seq_seconds have passed;
    # compared with the served latencies of the same requests
    probe2 = tn.tn_ctx_create(-1)

    def fp64_macs(L, W, D):
        lat_ = tn.tn_create_lattice(probe2, L, W, D)
        info = tn.tn_program_info(lat_, tn.TN_FP64)
        tn.tn_destroy_lattice(lat_)
        return info["product_macs"], info["footprint_bytes"]

    seq_times, seq_tickets, skipped = [], [], 0
    t0 = time.perf_counter()
    for r, f in stream_reqs:
        t = ticket_of.get(r)
        if not f or t is None or t not in done:
            continue
        L, W, D, h, sd = r
        macs, fp64_bytes = fp64_macs(L, W, D)
        if macs > 5e12 or fp64_bytes > budget:
            skipped += 1
            continue
        l_ = tn.tn_create_lattice(ctx, L, W, D)
        tn.tn_fill_random(l_, sd)
        torch.cuda.synchronize()
        ts_ = time.perf_counter()
        tn.tn_energy(l_, 1.0, h, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
        seq_times.append(time.perf_counter() - ts_)
        tn.tn_destroy_lattice(l_)
        seq_tickets.append(t)
        if time.perf_counter() - t0 > seq_seconds:
            break
    seq_times = np.array(seq_times)
    same = np.array([done[t][1] - done[t][0] for t in seq_tickets])
    n_seq = int(seq_times.size)
    seq_rate = n_seq / seq_times.sum() if n_seq else None
    tn.tn_ctx_destroy(probe)
    tn.tn_ctx_destroy(probe2)
    tn.tn_ctx_destroy(ctx)
    return {"metric": "served p50/p99 latency", "workload": "Poisson stream of TFIM-PEPS energy requests",
            "unit": "s", "precision": precision, "requests": n, "served": served,
            "rejected_over_budget": rejected, "budget_gb": budget / 1e9, "capacity_jobs_per_s": cap,
            "recompute_form_shapes": recompute_shapes,
            "recompute_form_served": int(sum(1 for t in done if shapes_of[t] in set(recompute_shapes))),
            "offered_rate_jobs_per_s": rate, "p50_latency_s": float(np.percentile(lat, 50)),
            "p99_latency_s": float(np.percentile(lat, 99)), "mean_latency_s": float(lat.mean()),
            "throughput_energies_per_s": served / (t_end - t_start),
            "by_D": {f"D={d}": {"served": int(v.size),
                                "p50_latency_s": float(np.percentile(v, 50)) if v.size else None,
                                "p99_latency_s": float(np.percentile(v, 99)) if v.size else None}
                     for d, v in lat_d.items()},
            "calibration": {"requests": len(calib), "what": "a burst of admissible requests from the same "
                            "distribution, submitted at once; capacity = requests / wall time"},
            "sequential_fp64": {"energies_per_s": seq_rate, "requests": n_seq, "skipped_heavy": skipped,
                                "p50_solve_s": float(np.percentile(seq_times, 50)) if n_seq else None,
                                "p99_solve_s": float(np.percentile(seq_times, 99)) if n_seq else None,
                                "served_p50_latency_s_same_requests": float(np.percentile(same, 50)) if n_seq else None,
                                "served_p99_latency_s_same_requests": float(np.percentile(same, 99)) if n_seq else None,
                                "what": "the served requests in stream order, one FP64 energy at a time (those "
                                        "with more than 5e12 FP64 product multiply-adds skipped), until the time "
                                        "cap; beside the served latencies of the same requests"},
            "distribution": "L, W ~ U{4..12}, D ~ U{2,3}, h ~ U[0.5,5], seeded uniform[-1,1) tensors"}


def run_serve(args):
    import torch
    torch.cuda.set_device(0)
    line = serve_stream(args.requests, args.calibrate, args.precision or "bf16x6", args.seq_seconds, args.recompute)
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------- 8x8 D=2 batch --

def run_8x8(args):
    """The 8x8 D=2 batch as its own line: B lattices per step, every observable,
    E at h in {2.0, 3.04, 4.0}."""
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
    prec_name = args.precision or "fp32"
    prec = tn.PRECISIONS[prec_name]
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
    tn.tn_batch_set_tensors_device(b, dev_in, n_in)
    for _ in range(max(3, args.warmup)):
        tn.tn_batch_run(b, 1.0, hs)
    torch.cuda.synchronize()
    launches_per_step = tn.tn_batch_launch_count(b)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    if ws > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    with ClockSampler(local, args.clock_log) as clk:
        for s in range(args.steps):
            with torch.cuda.stream(stream):
                flush.fill_(float(s))
            ev[s][0].record(stream)
            tn.tn_batch_run(b, 1.0, hs)
            ev[s][1].record(stream)
        torch.cuda.synchronize()
    if ws > 1:
        torch.distributed.barrier()
    t_total = max_over_ranks(sum(a.elapsed_time(e) for a, e in ev) / 1000.0, ws)
    value = job_rate(ws, B, args.steps, t_total)

    def e2e_step():
        tn.check(tn.lib().tn_batch_set_tensors(b, tn.c_void_p(host_in.data_ptr()), n_in), "set tensors")
        tn.tn_batch_run(b, 1.0, hs)
        tn.check(tn.lib().tn_batch_results_host(b, tn.c_void_p(host_out.data_ptr()), n_res), "results")

    for _ in range(2):
        e2e_step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        e2e_step()
    t_e2e = max_over_ranks(time.perf_counter() - t0, ws)
    fams = family_stats(tn, torch, ctx, b, hs, runs=3)
    hbm, bf16, sm_max, src = _peaks()
    peaks = {"hbm": hbm, "bf16": bf16, "bf16_sus": _peak_key("bf16_tflops_sustained", bf16), "src": src,
             "fp64": tn.tn_peak_probe(ctx, 0), "fp32": tn.tn_peak_probe(ctx, 1)}
    dom = max(fams, key=lambda k: fams[k]["ms"])
    line = {"metric": METRIC, "value": value, "unit": "lattice evals/s", "n_gpus": ws, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": 1000.0 * t_total / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": {"fp64": "f64", "fp32": "f32", "bf16x3": "f32+bf16x3", "bf16x6": "f32+bf16x6"}[prec_name],
            "data": "synthetic: seeded uniform[-1,1) site tensors (SplitMix64), fresh seeds per rank",
            "config": {"workload": WORKLOAD_8X8, "batch": B, "L": L_, "W": W_, "D": D_, "h": list(H_FIELDS),
                       "schedule": "auto (paper's min-bottleneck cut)",
                       "l2": "flushed between timed steps (256 MB write)", "parallelism": f"replicas x{ws}"},
            "energies_per_s": value * len(H_FIELDS),
            "e2e": {"value": job_rate(ws, B, args.steps, t_e2e), "unit": "lattice evals/s",
                    "h2d_bytes_per_step": int(n_in * 8), "d2h_bytes_per_step": int(n_res * 8)},
            "gpu_launches": int(launches_per_step * args.steps),
            "roofline": roofline_of(fams, dom, prec_name, peaks),
            "roofline_absorb": roofline_of(fams, "absorb", prec_name, peaks),
            "kernel_families_ms": {k: v["ms"] for k, v in fams.items() if v["launches"]},
            "clocks": clk.summary()}
    tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if ws > 1:
        torch.distributed.destroy_process_group()
    return 0


def run_batch(args):
    """512 independent lattices, L, W ~ U{4..10}, D ~ U{2,3}, h ~ U[0.5,5], in one
    batch group: passes of at most the pass budget (members of a pass run
    together, every wave of all members one grouped launch) sharing one arena,
    all captured into one CUDA graph, so a run is one graph launch; members
    whose footprint alone exceeds the budget are reported, not run (with
    --recompute: members whose cached-state program exceeds it run in the
    recompute form where that fits)."""
    import numpy as np
    import torch

    from paper_1908_08553_gb300 import tn

    torch.cuda.set_device(0)
    prec = tn.PRECISIONS[args.precision or "fp32"]
    budget = int(225e9)              # per pass; the passes share one arena
    rng = np.random.default_rng(2)
    n = args.members
    Ls = rng.integers(4, 11, size=n)
    Ws = rng.integers(4, 11, size=n)
    Ds = rng.choice([2, 3], size=n)
    hs = rng.uniform(0.5, 5.0, size=n)
    probe = tn.tn_ctx_create(-1)
    fp = []
    recomputed = []
    for k, (L, W, D) in enumerate(zip(Ls, Ws, Ds)):
        lat = tn.tn_create_lattice(probe, int(L), int(W), int(D))
        fp.append(tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY))
        if args.recompute and fp[-1] > budget:
            # the batch group falls back to the recompute form for such a member
            tn.tn_autotune_set(int(L), int(W), int(D), prec, tn.TN_WORK_ENERGY, 15 | 32)
            fp[-1] = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY)
            tn.tn_autotune_set(int(L), int(W), int(D), prec, tn.TN_WORK_ENERGY, 15)
            if fp[-1] <= budget:
                recomputed.append(k)
        tn.tn_destroy_lattice(lat)
    tn.tn_ctx_destroy(probe)
    tn.tn_autotune_clear()
    ok = [k for k in range(n) if fp[k] <= budget]
    excluded = [k for k in range(n) if fp[k] > budget]
    stream = torch.cuda.Stream()
    ctx = tn.tn_ctx_create(0, 0, stream)          # budget: 90% of the free device memory
    # autotune every (L, W, D) bucket whose copies fit the tuning budget (the
    # largest D = 3 shapes keep the default choices); every batch built after
    # this takes its programs from the table
    tune = None
    if not args.no_autotune:
        shapes = sorted({(int(Ls[k]), int(Ws[k]), int(Ds[k])) for k in ok})
        t0 = time.perf_counter()
        tn.tn_autotune(ctx, [s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], prec,
                       tn.TN_WORK_ENERGY, reps=3, max_bytes=int(4e9))
        tune_s = time.perf_counter() - t0
        rows = [(s, tn.tn_autotune_lookup(*s, prec)) for s in shapes]
        tuned = [(s, r) for s, r in rows if r["tuned"]]
        changed = [(s, r) for s, r in tuned if r["knobs"] != 15]
        tune = {"buckets": len(shapes), "tuned": len(tuned), "changed_from_default": len(changed),
                "seconds": tune_s,
                "changed": [{"L": s[0], "W": s[1], "D": s[2], "knobs": r["knobs"],
                             "best_ms": r["best_ms"], "default_ms": r["default_ms"]} for s, r in changed[:12]],
                "what": "per (L, W, D): every applicable program choice timed on copies of the shape "
                        "(at most 4 GB); the fastest by >= 2% kept; shapes above 4 GB keep the defaults"}
    # every admissible member in one batch group: passes of at most the budget
    # sharing one arena, all captured into one CUDA graph
    okk = np.array(ok)
    g = tn.tn_batch_group_create(ctx, Ls[okk], Ws[okk], Ds[okk], prec, budget)
    info = tn.tn_batch_group_info(g)
    tn.tn_batch_group_fill_random(g, args.batch_seed)      # member seeds from the batch seed
    hh = hs[okk].copy()
    # one timed run (minutes of device work: the graph and every kernel are
    # already loaded, so there is nothing to warm up)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    tn.tn_batch_group_run(g, 1.0, hh)                      # one graph launch
    e1.record(stream)
    torch.cuda.synchronize()
    total_ms = e0.elapsed_time(e1)
    r = tn.tn_batch_group_results_host(g)
    assert np.all(np.isfinite(r))
    tn.tn_batch_group_destroy(g)
    tn.tn_ctx_destroy(ctx)
    m = len(ok)
    line = {"metric": "batched exact TFIM-PEPS energy evals/s", "workload": "512 mixed lattices, L, W in 4..10, D in {2,3}",
            "precision": args.precision or "fp32", "members": n, "evaluated": m, "excluded_over_budget": len(excluded),
            "recompute_form_members": len(recomputed),
            "excluded_shapes": sorted({(int(Ls[k]), int(Ws[k]), int(Ds[k])) for k in excluded}),
            "graph_launches": 1, "passes": info["passes"], "kernel_launches": info["launches"],
            "shared_arena_gb": info["arena_bytes"] / 1e9, "ms": total_ms, "autotune": tune,
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
    prec = tn.PRECISIONS[args.precision or "fp32"]
    L, W, D = args.L, args.W, args.D
    if args.recompute:
        # the recompute form of the energy program (program choice bit 32)
        tn.tn_autotune_set(L, W, D, prec, work, tn.tn_autotune_lookup(L, W, D, prec, work)["knobs"] | 32)
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
    line = {"workload": f"{args.batch} x {L}x{W} D={D}", "precision": args.precision or "fp32",
            "schedule": args.schedule, "work": args.work, "recompute": bool(args.recompute), "ms_per_run": ms,
            "launches_per_run": tn.tn_batch_launch_count(b),
            "log2_norm": float(r[1]), "energy_per_site": float(r[0]) / (L * W)}
    tn.tn_batch_destroy(b)
    tn.tn_ctx_destroy(ctx)
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--batch", type=int, default=256, help="8x8 lattices per step (8x8 workload and extras)")
    ap.add_argument("--precision", default=None, choices=["fp64", "fp32", "bf16x3", "bf16x6"],
                    help="default: fp64 for the headline, fp32 for the other workloads")
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-extras", action="store_true",
                    help="headline only: skip the other precisions, the 8x8 batch, serving and the CPU baseline")
    ap.add_argument("--e2e-steps", type=int, default=3, help="steps of the end-to-end measurement")
    ap.add_argument("--serve-requests", type=int, default=48, help="headline extras: served stream length")
    ap.add_argument("--workload", default="large", choices=["large", "8x8", "serve", "batch", "case", "next"],
                    help="large: 12x12 D=2 + 8x8 D=3 energies (the headline); 8x8: the 8x8 D=2 batch; "
                         "serve: Poisson request stream; batch: 512 mixed lattices; case: --batch copies of "
                         "one L x W lattice")
    ap.add_argument("--L", type=int, default=8, help="case: rows")
    ap.add_argument("--W", type=int, default=8, help="case: columns")
    ap.add_argument("--D", type=int, default=2, help="case: bond dimension")
    ap.add_argument("--seed", type=int, default=7, help="case: tensor seed")
    ap.add_argument("--schedule", default="auto", choices=["auto", "row", "col", "quadrant"])
    ap.add_argument("--work", default="energy", choices=["energy", "norm"], help="case: work kind")
    ap.add_argument("--recompute", action="store_true",
                    help="case: the recompute form of the energy program (chain states recomputed, not cached); "
                         "batch / serve: lattices whose cached form exceeds the budget run in the recompute form")
    ap.add_argument("--clock-log", default=None, help="CSV file for the nvidia-smi clock samples")
    ap.add_argument("--members", type=int, default=512, help="batch: lattices")
    ap.add_argument("--batch-seed", type=int, default=2, help="batch: tensor seed")
    ap.add_argument("--no-autotune", action="store_true", help="batch: keep the default program choices")
    ap.add_argument("--requests", type=int, default=300, help="serve: requests in the stream")
    ap.add_argument("--calibrate", type=int, default=24, help="serve: burst size for the capacity")
    ap.add_argument("--seq-seconds", type=float, default=60.0, help="serve: time cap of the FP64 sample")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return {"large": run_headline, "8x8": run_8x8, "serve": run_serve, "batch": run_batch,
            "case": run_case, "next": run_next}[args.workload](args)


if __name__ == "__main__":
    sys.exit(main())
