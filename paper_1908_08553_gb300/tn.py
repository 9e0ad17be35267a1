"""Thin ctypes binding of libtn (include/tn.h): same names, argument marshalling only.

Every computation happens inside libtn's CUDA kernels.  If the library cannot
be loaded this module raises; there is no CPU fallback.  Device buffers may be
passed as torch CUDA tensors (their data_ptr is used) or raw integer pointers.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import POINTER, byref, c_char_p, c_double, c_int, c_int32, c_int64, c_size_t, c_uint64, c_void_p

import numpy as np

from . import build as _build

TN_OK, TN_NOT_READY = 0, 1
TN_ERR_INVALID, TN_ERR_OVER_BUDGET, TN_ERR_OOM = -1, -2, -3
TN_ERR_CUDA, TN_ERR_TIMEOUT, TN_ERR_NUMERIC, TN_ERR_NO_DEVICE = -4, -5, -6, -7
TN_FP64, TN_FP32, TN_BF16X3, TN_BF16X6 = 0, 1, 2, 3
TN_SCHED_AUTO, TN_SCHED_ROW, TN_SCHED_COL, TN_SCHED_QUADRANT = 0, 1, 2, 3
TN_WORK_NORM, TN_WORK_ENERGY = 0, 1
TN_OP_NORM, TN_OP_X, TN_OP_ZZ, TN_OP_Z, TN_OP_Y = 0, 1, 2, 3, 4

PRECISIONS = {"fp64": TN_FP64, "fp32": TN_FP32, "bf16x3": TN_BF16X3, "bf16x6": TN_BF16X6}


class tn_scalar(ctypes.Structure):
    _fields_ = [("mant", c_double), ("exp2", c_int64)]


class tn_result(ctypes.Structure):
    _fields_ = [("energy", c_double), ("energy_per_site", c_double), ("norm", tn_scalar),
                ("sx", POINTER(c_double)), ("szsz", POINTER(c_double)), ("err_bound_est", c_double),
                ("precision", c_int), ("schedule_o", c_int), ("schedule_i", c_int), ("schedule_j", c_int),
                ("sz", POINTER(c_double)), ("czz", POINTER(c_double))]


class tn_job(ctypes.Structure):
    _fields_ = [("L", c_int), ("W", c_int), ("D", c_int), ("precision", c_int), ("J", c_double),
                ("h", c_double), ("tensors", POINTER(c_double)), ("seed", c_uint64)]


class tn_ite_params(ctypes.Structure):
    _fields_ = [("J", c_double), ("gamma", c_double), ("dtau", c_double), ("steps", c_int), ("chi_max", c_int),
                ("eps", c_double), ("energy_every", c_int), ("precision", c_int)]


# name -> (restype, argtypes): the complete exported surface of include/tn.h
SIGNATURES = {
    "tn_ctx_create": (c_int, [c_int, c_size_t, c_void_p, POINTER(c_void_p)]),
    "tn_ctx_destroy": (c_int, [c_void_p]),
    "tn_ctx_memory": (c_int, [c_void_p, POINTER(c_size_t), POINTER(c_size_t)]),
    "tn_create_lattice": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_void_p)]),
    "tn_destroy_lattice": (c_int, [c_void_p]),
    "tn_lattice_elems": (c_size_t, [c_int, c_int, c_int]),
    "tn_set_site_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_fill_random": (c_int, [c_void_p, c_uint64]),
    "tn_get_site_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_footprint": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_size_t)]),
    "tn_plan": (c_int, [c_void_p, c_int, c_void_p, c_size_t, POINTER(c_size_t)]),
    "tn_plan_work": (c_int, [c_void_p, c_int, c_int, c_void_p, c_size_t, POINTER(c_size_t)]),
    "tn_contract_norm": (c_int, [c_void_p, c_int, c_int, POINTER(tn_scalar)]),
    "tn_expectation": (c_int, [c_void_p, c_int, c_int, c_int, c_int, POINTER(c_double)]),
    "tn_energy": (c_int, [c_void_p, c_double, c_double, c_int, POINTER(tn_result)]),
    "tn_program_info": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_int64), c_size_t, POINTER(c_size_t)]),
    "tn_wait_selfcheck": (c_int, [c_void_p, c_double, POINTER(c_int)]),
    "tn_bond_correlators": (c_int, [c_void_p, c_int, c_int, c_int, POINTER(c_double)]),
    "tn_energy_sched": (c_int, [c_void_p, c_double, c_double, c_int, c_int, POINTER(tn_result)]),
    "tn_batch_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int,
                                POINTER(c_void_p)]),
    "tn_batch_destroy": (c_int, [c_void_p]),
    "tn_batch_elems": (c_size_t, [c_void_p]),
    "tn_batch_set_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_batch_set_tensors_device": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_batch_fill_random": (c_int, [c_void_p, c_uint64]),
    "tn_batch_run": (c_int, [c_void_p, c_double, c_void_p]),
    "tn_batch_result_size": (c_size_t, [c_void_p]),
    "tn_batch_results_host": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_batch_results_device": (c_int, [c_void_p, POINTER(c_void_p)]),
    "tn_batch_launch_count": (c_int, [c_void_p, POINTER(c_int64)]),
    "tn_submit": (c_int, [c_void_p, POINTER(tn_job), POINTER(c_uint64)]),
    "tn_poll": (c_int, [c_void_p, c_uint64, POINTER(tn_result)]),
    "tn_wait": (c_int, [c_void_p, c_uint64, c_double, POINTER(tn_result)]),
    "tn_absorb": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64, c_void_p]),
    "tn_absorb_dot": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64, c_void_p,
                              c_void_p]),
    "tn_absorb_dot_noalloc": (c_int, [c_int, c_void_p, c_void_p, c_void_p, c_int64, c_int32, c_int32, c_int64,
                                      c_void_p, c_void_p]),
    "tn_status_string": (c_char_p, [c_int]),
    "tn_last_error": (c_char_p, []),
    "tn_ctx_set_profiling": (c_int, [c_void_p, c_int]),
    "tn_ctx_inject_wait_timeout": (c_int, [c_void_p, c_int]),
    "tn_peak_probe": (c_int, [c_void_p, c_int, POINTER(c_double)]),
    "tn_ite_init_product": (c_int, [c_void_p]),
    "tn_pair_correlators": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_void_p, c_void_p, c_void_p]),
    "tn_set_site_tensors_complex": (c_int, [c_void_p, c_void_p, c_void_p, c_size_t]),
    "tn_batch_group_create": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_size_t,
                                      POINTER(c_void_p)]),
    "tn_batch_group_destroy": (c_int, [c_void_p]),
    "tn_batch_group_info": (c_int, [c_void_p, c_void_p, c_void_p, c_void_p, c_void_p, c_void_p]),
    "tn_batch_group_set_tensors": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_batch_group_fill_random": (c_int, [c_void_p, c_uint64]),
    "tn_batch_group_run": (c_int, [c_void_p, c_double, c_void_p]),
    "tn_batch_group_results_host": (c_int, [c_void_p, c_void_p, c_size_t]),
    "tn_lattice_is_complex": (c_int, [c_void_p]),
    "tn_site_expectations": (c_int, [c_void_p, c_int, c_int, c_void_p]),
    "tn_autotune": (c_int, [c_void_p, c_int, c_void_p, c_void_p, c_void_p, c_int, c_int, c_int, c_size_t]),
    "tn_autotune_lookup": (c_int, [c_int, c_int, c_int, c_int, c_int, POINTER(c_int), POINTER(c_double),
                                   POINTER(c_double), POINTER(c_int)]),
    "tn_autotune_set": (c_int, [c_int, c_int, c_int, c_int, c_int, c_int]),
    "tn_autotune_clear": (c_int, []),
    "tn_autotune_save": (c_int, [c_char_p]),
    "tn_autotune_load": (c_int, [c_char_p]),
    "tn_bmps_norm": (c_int, [c_void_p, c_int, c_int, POINTER(tn_scalar)]),
    "tn_bmps_expectation": (c_int, [c_void_p, c_int, c_int, c_int, c_int, c_int, c_int, POINTER(c_double)]),
    "tn_bmps_energy": (c_int, [c_void_p, c_int, c_int, c_double, c_double, POINTER(tn_result)]),
    "tn_ite_run": (c_int, [c_void_p, POINTER(tn_ite_params), c_void_p, c_void_p, POINTER(c_double)]),
    "tn_ctx_kernel_stats": (c_int, [c_void_p, c_int, POINTER(c_int64), POINTER(c_double), POINTER(c_double),
                                    POINTER(c_double)]),
}

_lib = None


def lib(build_if_needed: bool = True):
    """Load libtn (building it first if stale).  Raises if it cannot be loaded."""
    global _lib
    if _lib is None:
        path = _build.build() if build_if_needed else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"libtn not built at {path}")
        # bind every symbol at load: a missing definition fails here, not mid-run
        _lib = ctypes.CDLL(path, mode=os.RTLD_NOW | os.RTLD_LOCAL)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(_lib, name)
            f.restype = res
            f.argtypes = args
    return _lib


class TNError(RuntimeError):
    def __init__(self, status: int, where: str):
        msg = lib().tn_last_error().decode() or lib().tn_status_string(status).decode()
        super().__init__(f"{where}: {lib().tn_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def check(status: int, where: str):
    if status not in (TN_OK,):
        raise TNError(status, where)


def _ptr(x):
    """Device or host pointer from a torch tensor, numpy array or int."""
    if x is None:
        return None
    if isinstance(x, int):
        return c_void_p(x)
    if isinstance(x, np.ndarray):
        return x.ctypes.data_as(c_void_p)
    if hasattr(x, "data_ptr"):
        return c_void_p(x.data_ptr())
    raise TypeError(type(x))


# -------------------------------------------------------------- wrappers

def tn_ctx_create(device: int = 0, budget: int = 0, stream=None):
    h = c_void_p()
    st = None
    if stream is not None:
        st = c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(lib().tn_ctx_create(device, budget, st, byref(h)), "tn_ctx_create")
    return h


def tn_ctx_destroy(ctx):
    check(lib().tn_ctx_destroy(ctx), "tn_ctx_destroy")


def tn_ctx_memory(ctx):
    u, b = c_size_t(), c_size_t()
    check(lib().tn_ctx_memory(ctx, byref(u), byref(b)), "tn_ctx_memory")
    return u.value, b.value


def tn_create_lattice(ctx, L: int, W: int, D: int):
    h = c_void_p()
    check(lib().tn_create_lattice(ctx, L, W, D, byref(h)), "tn_create_lattice")
    return h


def tn_destroy_lattice(lat):
    check(lib().tn_destroy_lattice(lat), "tn_destroy_lattice")


def tn_lattice_elems(L: int, W: int, D: int) -> int:
    return int(lib().tn_lattice_elems(L, W, D))


def tn_set_site_tensors(lat, host: np.ndarray):
    host = np.ascontiguousarray(host, dtype=np.float64)
    check(lib().tn_set_site_tensors(lat, _ptr(host), host.size), "tn_set_site_tensors")


def tn_get_site_tensors(lat, n: int) -> np.ndarray:
    out = np.empty(n)
    check(lib().tn_get_site_tensors(lat, _ptr(out), n), "tn_get_site_tensors")
    return out


def tn_fill_random(lat, seed: int):
    check(lib().tn_fill_random(lat, c_uint64(seed)), "tn_fill_random")


def tn_footprint(lat, sched: int, prec: int, work: int) -> int:
    n = c_size_t()
    check(lib().tn_footprint(lat, sched, prec, work, byref(n)), "tn_footprint")
    return n.value


def tn_plan(lat, sched: int = TN_SCHED_AUTO) -> np.ndarray:
    n = c_size_t()
    check(lib().tn_plan(lat, sched, None, 0, byref(n)), "tn_plan")
    out = np.zeros(n.value, dtype=np.int64)
    check(lib().tn_plan(lat, sched, _ptr(out), out.size, byref(n)), "tn_plan")
    return out


def tn_plan_work(lat, sched: int = TN_SCHED_AUTO, work: int = TN_WORK_ENERGY) -> np.ndarray:
    n = c_size_t()
    check(lib().tn_plan_work(lat, sched, work, None, 0, byref(n)), "tn_plan_work")
    out = np.zeros(n.value, dtype=np.int64)
    check(lib().tn_plan_work(lat, sched, work, _ptr(out), out.size, byref(n)), "tn_plan_work")
    return out


def tn_contract_norm(lat, prec: int = TN_FP64, sched: int = TN_SCHED_AUTO):
    s = tn_scalar()
    check(lib().tn_contract_norm(lat, prec, sched, byref(s)), "tn_contract_norm")
    return s.mant, s.exp2


def tn_expectation(lat, prec: int, op: int, i: int, j: int = 0) -> float:
    v = c_double()
    check(lib().tn_expectation(lat, prec, op, i, j, byref(v)), "tn_expectation")
    return v.value


def tn_program_info(lat, prec: int, sched: int = TN_SCHED_AUTO, work: int = TN_WORK_ENERGY) -> dict:
    """Build and check the lattice's contraction program (host only)."""
    out = np.zeros(7, dtype=np.int64)
    n = c_size_t()
    check(lib().tn_program_info(lat, prec, sched, work, out.ctypes.data_as(POINTER(c_int64)), out.size, byref(n)),
          "tn_program_info")
    keys = ["ops", "waves", "arena_bytes", "footprint_bytes", "absorb_bytes", "fused_pairs", "product_macs"]
    return dict(zip(keys, (int(v) for v in out)))


def tn_wait_selfcheck(ctx, limit_ms: float) -> bool:
    """True when a bounded device wait on a flag nothing sets expired cleanly."""
    v = c_int()
    check(lib().tn_wait_selfcheck(ctx, limit_ms, byref(v)), "tn_wait_selfcheck")
    return bool(v.value)


def tn_bond_correlators(lat, prec: int, op_a: int, op_b: int, L: int, W: int) -> np.ndarray:
    """<A_i B_j> on every nearest-neighbour bond, A, B in {TN_OP_X, TN_OP_Z}."""
    nb = L * (W - 1) + W * (L - 1)
    out = np.zeros(max(nb, 1))
    check(lib().tn_bond_correlators(lat, prec, op_a, op_b, out.ctypes.data_as(POINTER(c_double))),
          "tn_bond_correlators")
    return out[:nb]


def tn_energy_full(lat, J: float, h: float, prec: int, sched: int, L: int, W: int):
    """(tn_result, sx, szsz, sz, czz): every observable of the energy evaluation."""
    r, sx, zz, nb = _result_arrays(L, W)
    sz, czz = np.zeros(L * W), np.zeros(max(nb, 1))
    r.sz = sz.ctypes.data_as(POINTER(c_double))
    r.czz = czz.ctypes.data_as(POINTER(c_double))
    check(lib().tn_energy_sched(lat, J, h, prec, sched, byref(r)), "tn_energy")
    return r, sx, zz[:nb], sz, czz[:nb]


def tn_energy(lat, J: float, h: float, prec: int = TN_FP64, sched: int = TN_SCHED_AUTO,
              L: int | None = None, W: int | None = None):
    """Returns (tn_result, sx array, szsz array) when L, W are given, else the result only."""
    r = tn_result()
    sx = zz = None
    if L is not None:
        nb = L * (W - 1) + W * (L - 1)
        sx, zz = np.zeros(L * W), np.zeros(max(nb, 1))
        r.sx = sx.ctypes.data_as(POINTER(c_double))
        r.szsz = zz.ctypes.data_as(POINTER(c_double))
    check(lib().tn_energy_sched(lat, J, h, prec, sched, byref(r)), "tn_energy")
    if L is None:
        return r
    return r, sx, zz[:L * (W - 1) + W * (L - 1)]


def tn_batch_create(ctx, Ls, Ws, Ds, prec: int, sched: int = TN_SCHED_AUTO, work: int = TN_WORK_ENERGY):
    Ls, Ws, Ds = (np.ascontiguousarray(v, dtype=np.int32) for v in (Ls, Ws, Ds))
    h = c_void_p()
    check(lib().tn_batch_create(ctx, Ls.size, _ptr(Ls), _ptr(Ws), _ptr(Ds), prec, sched, work, byref(h)),
          "tn_batch_create")
    return h


def tn_batch_destroy(b):
    check(lib().tn_batch_destroy(b), "tn_batch_destroy")


def tn_batch_elems(b) -> int:
    return int(lib().tn_batch_elems(b))


def tn_batch_set_tensors(b, host: np.ndarray):
    check(lib().tn_batch_set_tensors(b, _ptr(host), host.size), "tn_batch_set_tensors")


def tn_batch_set_tensors_device(b, dev, n: int):
    check(lib().tn_batch_set_tensors_device(b, _ptr(dev), n), "tn_batch_set_tensors_device")


def tn_batch_fill_random(b, seed: int):
    check(lib().tn_batch_fill_random(b, c_uint64(seed)), "tn_batch_fill_random")


def tn_batch_run(b, J: float, h: np.ndarray):
    h = np.ascontiguousarray(h, dtype=np.float64)
    check(lib().tn_batch_run(b, J, _ptr(h)), "tn_batch_run")


def tn_batch_result_size(b) -> int:
    return int(lib().tn_batch_result_size(b))


def tn_batch_results_host(b, out: np.ndarray | None = None) -> np.ndarray:
    n = tn_batch_result_size(b)
    if out is None:
        out = np.empty(n)
    check(lib().tn_batch_results_host(b, _ptr(out), n), "tn_batch_results_host")
    return out


def tn_batch_results_device(b) -> int:
    p = c_void_p()
    check(lib().tn_batch_results_device(b, byref(p)), "tn_batch_results_device")
    return p.value


def tn_batch_launch_count(b) -> int:
    n = c_int64()
    check(lib().tn_batch_launch_count(b, byref(n)), "tn_batch_launch_count")
    return n.value


def tn_submit(ctx, L, W, D, prec, J, h, tensors: np.ndarray | None = None, seed: int = 0):
    job = tn_job(L, W, D, prec, J, h, None, seed)
    keep = None
    if tensors is not None:
        keep = np.ascontiguousarray(tensors, dtype=np.float64)
        job.tensors = keep.ctypes.data_as(POINTER(c_double))
    t = c_uint64()
    st = lib().tn_submit(ctx, byref(job), byref(t))
    check(st, "tn_submit")
    return t.value


def _result_arrays(L, W):
    nb = L * (W - 1) + W * (L - 1)
    r = tn_result()
    sx, zz = np.zeros(L * W), np.zeros(max(nb, 1))
    r.sx = sx.ctypes.data_as(POINTER(c_double))
    r.szsz = zz.ctypes.data_as(POINTER(c_double))
    return r, sx, zz, nb


def tn_poll(ctx, ticket: int, L: int, W: int):
    """None while not ready, else (tn_result, sx, szsz)."""
    r, sx, zz, nb = _result_arrays(L, W)
    st = lib().tn_poll(ctx, c_uint64(ticket), byref(r))
    if st == TN_NOT_READY:
        return None
    check(st, "tn_poll")
    return r, sx, zz[:nb]


def tn_wait(ctx, ticket: int, timeout_s: float, L: int, W: int):
    r, sx, zz, nb = _result_arrays(L, W)
    check(lib().tn_wait(ctx, c_uint64(ticket), timeout_s, byref(r)), "tn_wait")
    return r, sx, zz[:nb]


def tn_absorb(dtype: int, x_in, E, out, P: int, K: int, N: int, S: int, stream=None):
    st = None if stream is None else c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(lib().tn_absorb(dtype, _ptr(x_in), _ptr(E), _ptr(out), P, K, N, S, st), "tn_absorb")


def tn_absorb_dot(dtype: int, x_in, E, adj, P: int, K: int, N: int, S: int, result, stream=None):
    st = None if stream is None else c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(lib().tn_absorb_dot(dtype, _ptr(x_in), _ptr(E), _ptr(adj), P, K, N, S, _ptr(result), st),
          "tn_absorb_dot")


def tn_absorb_dot_noalloc(dtype: int, x_in, E, adj, P: int, K: int, N: int, S: int, result, stream=None):
    """tn_absorb_dot with its scratch in a fixed array inside the library (no allocation)."""
    st = None if stream is None else c_void_p(stream if isinstance(stream, int) else stream.cuda_stream)
    check(lib().tn_absorb_dot_noalloc(dtype, _ptr(x_in), _ptr(E), _ptr(adj), P, K, N, S, _ptr(result), st),
          "tn_absorb_dot_noalloc")


def tn_ctx_set_profiling(ctx, on: bool):
    check(lib().tn_ctx_set_profiling(ctx, 1 if on else 0), "tn_ctx_set_profiling")


def tn_batch_group_create(ctx, Ls, Ws, Ds, prec: int, pass_budget: int, sched: int = TN_SCHED_AUTO,
                          work: int = TN_WORK_ENERGY):
    """Lattices of any number and sizes, split into passes of at most pass_budget
    bytes sharing one arena, run as one CUDA graph."""
    Ls, Ws, Ds = (np.ascontiguousarray(v, dtype=np.int32) for v in (Ls, Ws, Ds))
    g = c_void_p()
    check(lib().tn_batch_group_create(ctx, Ls.size, _ptr(Ls), _ptr(Ws), _ptr(Ds), prec, sched, work,
                                      c_size_t(int(pass_budget)), byref(g)), "tn_batch_group_create")
    return g


def tn_batch_group_destroy(g):
    check(lib().tn_batch_group_destroy(g), "tn_batch_group_destroy")


def tn_batch_group_info(g) -> dict:
    p, a, ne, nr, nl = c_int(), c_size_t(), c_size_t(), c_size_t(), c_int64()
    check(lib().tn_batch_group_info(g, byref(p), byref(a), byref(ne), byref(nr), byref(nl)), "tn_batch_group_info")
    return {"passes": p.value, "arena_bytes": a.value, "n_elems": ne.value, "n_results": nr.value,
            "launches": nl.value}


def tn_batch_group_set_tensors(g, A):
    A = np.ascontiguousarray(A, dtype=np.float64)
    check(lib().tn_batch_group_set_tensors(g, _ptr(A), A.size), "tn_batch_group_set_tensors")


def tn_batch_group_fill_random(g, seed: int):
    check(lib().tn_batch_group_fill_random(g, c_uint64(seed)), "tn_batch_group_fill_random")


def tn_batch_group_run(g, J: float, hs):
    hs = np.ascontiguousarray(hs, dtype=np.float64)
    check(lib().tn_batch_group_run(g, J, _ptr(hs)), "tn_batch_group_run")


def tn_batch_group_results_host(g) -> np.ndarray:
    out = np.zeros(tn_batch_group_info(g)["n_results"])
    check(lib().tn_batch_group_results_host(g, _ptr(out), out.size), "tn_batch_group_results_host")
    return out


def tn_set_site_tensors_complex(lat, A) -> None:
    """Complex site tensors (one complex array in the real layout)."""
    A = np.asarray(A, dtype=np.complex128)
    re = np.ascontiguousarray(A.real)
    im = np.ascontiguousarray(A.imag)
    check(lib().tn_set_site_tensors_complex(lat, _ptr(re), _ptr(im), re.size), "tn_set_site_tensors_complex")


def tn_lattice_is_complex(lat) -> bool:
    return bool(lib().tn_lattice_is_complex(lat))


def tn_site_expectations(lat, prec: int, op: int, L: int, W: int) -> np.ndarray:
    """<O_k> for every site, O = TN_OP_X, TN_OP_Y or TN_OP_Z."""
    out = np.zeros(L * W)
    check(lib().tn_site_expectations(lat, prec, op, _ptr(out)), "tn_site_expectations")
    return out


def tn_pair_correlators(lat, prec: int, op_a: int, op_b: int, i, j) -> np.ndarray:
    """<A_i B_j> for arbitrary pairs of distinct sites (row-major), exactly."""
    i = np.ascontiguousarray(i, dtype=np.int32)
    j = np.ascontiguousarray(j, dtype=np.int32)
    out = np.zeros(max(i.size, 1))
    check(lib().tn_pair_correlators(lat, prec, op_a, op_b, i.size, _ptr(i), _ptr(j), _ptr(out)),
          "tn_pair_correlators")
    return out[:i.size]


def tn_autotune(ctx, Ls, Ws, Ds, prec: int, work: int = TN_WORK_ENERGY, reps: int = 3, max_bytes: int = 0):
    """Time the program choices of every distinct shape and keep the fastest (see tn.h)."""
    Ls, Ws, Ds = (np.ascontiguousarray(v, dtype=np.int32) for v in (Ls, Ws, Ds))
    check(lib().tn_autotune(ctx, Ls.size, _ptr(Ls), _ptr(Ws), _ptr(Ds), prec, work, reps, max_bytes),
          "tn_autotune")


def tn_autotune_lookup(L: int, W: int, D: int, prec: int, work: int = TN_WORK_ENERGY) -> dict:
    k, b, d, t = c_int(), c_double(), c_double(), c_int()
    check(lib().tn_autotune_lookup(L, W, D, prec, work, byref(k), byref(b), byref(d), byref(t)),
          "tn_autotune_lookup")
    return {"knobs": k.value, "best_ms": b.value, "default_ms": d.value, "tuned": bool(t.value)}


def tn_autotune_set(L: int, W: int, D: int, prec: int, work: int, knobs: int):
    check(lib().tn_autotune_set(L, W, D, prec, work, knobs), "tn_autotune_set")


def tn_autotune_clear():
    check(lib().tn_autotune_clear(), "tn_autotune_clear")


def tn_autotune_save(path: str):
    check(lib().tn_autotune_save(path.encode()), "tn_autotune_save")


def tn_autotune_load(path: str):
    check(lib().tn_autotune_load(path.encode()), "tn_autotune_load")


def tn_bmps_norm(lat, chi: int, prec: int = TN_FP64):
    """<Psi|Psi> by the boundary MPS of bond chi: (mantissa, exponent)."""
    out = tn_scalar()
    check(lib().tn_bmps_norm(lat, chi, prec, byref(out)), "tn_bmps_norm")
    return out.mant, out.exp2


def tn_bmps_expectation(lat, chi: int, op_i: int, i: int, op_j: int = 0, j: int = -1, prec: int = TN_FP64) -> float:
    v = c_double()
    check(lib().tn_bmps_expectation(lat, chi, prec, op_i, i, op_j, j, byref(v)), "tn_bmps_expectation")
    return v.value


def tn_bmps_energy(lat, chi: int, J: float, h: float, L: int, W: int, prec: int = TN_FP64):
    """(tn_result, sx, szsz) by the boundary MPS of bond chi."""
    r, sx, zz, nb = _result_arrays(L, W)
    check(lib().tn_bmps_energy(lat, chi, prec, J, h, byref(r)), "tn_bmps_energy")
    return r, sx, zz[:nb]


def tn_ite_init_product(lat):
    check(lib().tn_ite_init_product(lat), "tn_ite_init_product")


def tn_ite_run(lat, L: int, W: int, J: float, gamma: float, dtau: float, steps: int, chi_max: int, eps: float,
               energy_every: int = 2, prec: int = TN_FP64):
    """Imaginary time evolution in place; returns (energies, bond_dims, max_discarded)."""
    p = tn_ite_params(J, gamma, dtau, steps, chi_max, eps, energy_every, prec)
    ne = steps // energy_every if energy_every > 0 else 0
    en = np.zeros(max(ne, 1))
    nb = L * (W - 1) + W * (L - 1)
    dims = np.zeros(max(nb, 1), dtype=np.int32)
    disc = c_double()
    check(lib().tn_ite_run(lat, byref(p), _ptr(en), _ptr(dims), byref(disc)), "tn_ite_run")
    return en[:ne], dims[:nb], disc.value


def tn_peak_probe(ctx, dtype: int) -> float:
    """Measured FMA rate of the device in TFLOP/s (dtype 0 FP64, 1 FP32)."""
    v = c_double()
    check(lib().tn_peak_probe(ctx, dtype, byref(v)), "tn_peak_probe")
    return v.value


def tn_ctx_inject_wait_timeout(ctx, count: int):
    """Mark the next `count` batch runs as if a bounded device wait had run out."""
    check(lib().tn_ctx_inject_wait_timeout(ctx, count), "tn_ctx_inject_wait_timeout")


def tn_ctx_kernel_stats(ctx, family: int):
    n, ms, by, mac = c_int64(), c_double(), c_double(), c_double()
    check(lib().tn_ctx_kernel_stats(ctx, family, byref(n), byref(ms), byref(by), byref(mac)),
          "tn_ctx_kernel_stats")
    return dict(launches=n.value, ms=ms.value, bytes=by.value, macs=mac.value)


def plan_steps(words: np.ndarray):
    """Decode tn_plan's words into (header dict, steps array [n, 9])."""
    hdr = dict(fmt=int(words[0]), o=int(words[1]), i=int(words[2]), j=int(words[3]),
               n_steps=int(words[4]), peak=int(words[5]), mac=int(words[6]))
    steps = words[7:7 + 9 * hdr["n_steps"]].reshape(-1, 9)
    return hdr, steps
