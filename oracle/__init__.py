"""FP64 CPU oracle for the exact PEPS contraction -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  It shares no code with the CUDA library
(``paper_1908_08553_gb300``) and never imports it; the two meet only through
the seeded inputs of ``paper_1908_08553_gb300.inputs``.

Parts:
  * ``tn_oracle.c``  -- row-by-row boundary sweep in FP64 (Sec. 4 row order),
                        observables of Sec. 3, classical Ising enumeration.
  * ``brute.py``     -- 2^N state vector and explicit Hamiltonian (numpy/scipy).
  * ``planner.py``   -- the paper's minimum-bottleneck partition choice (Sec. 4),
                        written independently of the library's planner.
  * ``complex_peps.py`` -- complex site tensors: the double layer with the bra
                        conjugated, contracted row by row in complex128.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tn_oracle.c")
_OUT = os.path.join(_HERE, "_build", "libtn_oracle.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile the C oracle with gcc (OpenMP) into oracle/_build/."""
    os.makedirs(os.path.dirname(_OUT), exist_ok=True)
    if force or not os.path.exists(_OUT) or os.path.getmtime(_OUT) < os.path.getmtime(_SRC):
        tmp = _OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _OUT)
    return _OUT


def lib():
    global _lib
    if _lib is None:
        _lib = ctypes.CDLL(build())
        d, i64, i32 = ctypes.c_double, ctypes.c_int64, ctypes.c_int
        P = ctypes.c_void_p
        _lib.or_grid_contract.argtypes = [i32, i32, P, P, P, P]
        _lib.or_peps_norm.argtypes = [i32, i32, i32, P, P, P]
        _lib.or_peps_sweep_rows.argtypes = [i32, i32, i32, P, i32, i32, P, P]
        _lib.or_peps_sweep_rows.restype = i32
        _lib.or_peps_norm_all_cuts.argtypes = [i32, i32, i32, P, P, P]
        _lib.or_peps_observables.argtypes = [i32, i32, i32, P, P, P, P, P]
        _lib.or_peps_expect_one.argtypes = [i32, i32, i32, P, i32, i32, i32, P, P, P]
        _lib.or_ising_enumerate.argtypes = [i32, i32, d, P, P, P]
        _lib.or_peps_sz.argtypes = [i32, i32, i32, P, P]
        _lib.or_peps_bond_ops.argtypes = [i32, i32, i32, P, i32, i32, P]
        _lib.or_peps_bond_ops.restype = i32
        _lib.or_peps_pair.argtypes = [i32, i32, i32, P, i32, i32, i32, i32, P]
        _lib.or_peps_pair.restype = i32
        for f in (_lib.or_grid_contract, _lib.or_peps_norm, _lib.or_peps_norm_all_cuts,
                  _lib.or_peps_observables, _lib.or_peps_expect_one,
                  _lib.or_ising_enumerate, _lib.or_num_threads, _lib.or_peps_sz):
            f.restype = i32
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def _check_sites(L, W, D, A):
    from paper_1908_08553_gb300.inputs import n_elems  # input layout only
    A = np.ascontiguousarray(A, dtype=np.float64)
    if A.size != n_elems(L, W, D):
        raise ValueError(f"expected {n_elems(L, W, D)} entries, got {A.size}")
    return A


def num_threads() -> int:
    return int(lib().or_num_threads())


def grid_contract(L: int, W: int, dims: np.ndarray, tensors) -> tuple[float, int]:
    """Contract a generic grid of rank-4 tensors T[u][l][dn][rt] (row sweep)."""
    dims = np.ascontiguousarray(dims, dtype=np.int32).reshape(L * W, 4)
    flat = np.ascontiguousarray(np.concatenate([np.asarray(t, np.float64).ravel() for t in tensors]))
    m, e = np.zeros(1), np.zeros(1, np.int64)
    lib().or_grid_contract(L, W, _ptr(dims), _ptr(flat), _ptr(m), _ptr(e))
    return float(m[0]), int(e[0])


def norm(L: int, W: int, D: int, A: np.ndarray) -> tuple[float, int]:
    """<Psi|Psi> as (mantissa, exponent): value = mantissa * 2**exponent."""
    A = _check_sites(L, W, D, A)
    m, e = np.zeros(1), np.zeros(1, np.int64)
    lib().or_peps_norm(L, W, D, _ptr(A), _ptr(m), _ptr(e))
    return float(m[0]), int(e[0])


def sweep_rows(L: int, W: int, D: int, A: np.ndarray, nrows: int, ncols: int = 0) -> tuple[float, int]:
    """The first nrows rows of the row sweep, then the first ncols sites of the
    next row (a bounded timing sample)."""
    A = _check_sites(L, W, D, A)
    m, e = np.zeros(1), np.zeros(1, np.int64)
    if lib().or_peps_sweep_rows(L, W, D, _ptr(A), nrows, ncols, _ptr(m), _ptr(e)) != 0:
        raise ValueError("nrows / ncols out of range")
    return float(m[0]), int(e[0])


def sweep_macs(L: int, W: int, D: int, nrows: int, ncols: int = 0) -> int:
    """Multiply-adds of sweep_rows(L, W, D, A, nrows, ncols): a site absorption
    of the row sweep maps [P, h, u, S] to [P, dn, rt, S] with P * S * (h u)(dn rt)
    multiply-adds (double-layer dimensions, each leg D^2 or 1 on the edge)."""
    d = D * D

    def leg(on_edge):
        return 1 if on_edge else d

    total = 0
    for r in range(min(nrows + 1, L)):
        cols = W if r < nrows else ncols
        for c in range(cols):
            P = 1
            for k in range(c):
                P *= leg(r == L - 1)                 # dn legs of the sites already absorbed
            S = 1
            for k in range(c + 1, W):
                S *= leg(r == 0)                     # u legs of the sites still to come
            h, u = leg(c == 0), leg(r == 0)
            dn, rt = leg(r == L - 1), leg(c == W - 1)
            total += P * S * h * u * dn * rt
    return total


def energy_macs(L: int, W: int, D: int) -> int:
    """Multiply-adds of observables(): the cached top and bottom sweeps, one row
    per site and per horizontal bond, two rows per vertical bond, each row
    absorbed into the cached boundary above it (its cost is sweep_macs of that
    row; the bottom sweep mirrors the top one)."""
    row = [sweep_macs(L, W, D, r + 1) - sweep_macs(L, W, D, r) for r in range(L)]
    total = 2 * sum(row)
    total += sum(W * row[r] for r in range(L))              # sites
    total += sum((W - 1) * row[r] for r in range(L))        # horizontal bonds
    total += sum(W * (row[r] + row[r + 1]) for r in range(L - 1))   # vertical bonds
    return total


def norm_all_cuts(L: int, W: int, D: int, A: np.ndarray):
    """<T_r, B_r> for r = 0..L (the same norm through every row cut)."""
    A = _check_sites(L, W, D, A)
    m, e = np.zeros(L + 1), np.zeros(L + 1, np.int64)
    lib().or_peps_norm_all_cuts(L, W, D, _ptr(A), _ptr(m), _ptr(e))
    return m, e


@dataclass
class Observables:
    norm_m: float
    norm_e: int
    sx: np.ndarray
    szsz: np.ndarray
    sz: np.ndarray | None = None     # <Z_k>, filled by observables(..., with_z=True)

    def connected(self, L: int, W: int) -> np.ndarray:
        """c_ij = <Z_i Z_j> - <Z_i><Z_j> per bond (Eq. cij), bond order of szsz."""
        from paper_1908_08553_gb300.inputs import bonds
        i = np.array([a[0] * W + a[1] for a, _ in bonds(L, W)], dtype=np.int64)
        j = np.array([b[0] * W + b[1] for _, b in bonds(L, W)], dtype=np.int64)
        return self.szsz - self.sz[i] * self.sz[j]

    def energy(self, J: float, h: float) -> float:
        """E = -J sum <zz> - h sum <x> (Eqs. Hamiltonian and Etot)."""
        return float(-J * self.szsz.sum() - h * self.sx.sum())

    @property
    def log2_norm(self) -> float:
        return float(np.log2(abs(self.norm_m)) + self.norm_e)


def observables(L: int, W: int, D: int, A: np.ndarray, with_z: bool = False) -> Observables:
    A = _check_sites(L, W, D, A)
    nb = L * (W - 1) + W * (L - 1)
    m, e = np.zeros(1), np.zeros(1, np.int64)
    sx, szsz = np.zeros(L * W), np.zeros(max(nb, 1))
    lib().or_peps_observables(L, W, D, _ptr(A), _ptr(m), _ptr(e), _ptr(sx), _ptr(szsz))
    sz = None
    if with_z:
        sz = np.zeros(L * W)
        lib().or_peps_sz(L, W, D, _ptr(A), _ptr(sz))
    return Observables(float(m[0]), int(e[0]), sx, szsz[:nb], sz)


def bond_correlators(L: int, W: int, D: int, A: np.ndarray, op_a: str, op_b: str) -> np.ndarray:
    """<A_i B_j> on every nearest-neighbour bond (szsz order, i the left or upper
    site), A and B in {'x', 'z'}."""
    A = _check_sites(L, W, D, A)
    nb = L * (W - 1) + W * (L - 1)
    out = np.zeros(max(nb, 1))
    code = {"x": 1, "z": 2}
    lib().or_peps_bond_ops(L, W, D, _ptr(A), code[op_a], code[op_b], _ptr(out))
    return out[:nb]


def pair(L: int, W: int, D: int, A: np.ndarray, op_a: str, i: int, op_b: str, j: int) -> float:
    """<A_i B_j> for any distinct sites (row-major), A, B in {'x', 'z', 'y'}, one full
    contraction per observable.  A real state has <X_i Y_j> = <Z_i Y_j> = 0
    exactly; <Y_i Y_j> is -<R_i R_j> with the real antisymmetric R, Y = i R."""
    A = _check_sites(L, W, D, A)
    ya, yb = op_a == "y", op_b == "y"
    if ya != yb:
        if i == j:
            raise ValueError("sites must differ")
        return 0.0
    code = {"x": 1, "z": 2, "y": 4}
    v = np.zeros(1)
    if lib().or_peps_pair(L, W, D, _ptr(A), code[op_a], i, code[op_b], j, _ptr(v)) != 0:
        raise ValueError("bad sites or operators")
    return -float(v[0]) if ya else float(v[0])


def expect_one(L: int, W: int, D: int, A: np.ndarray, op: str, i: int = 0, j: int = 0):
    """One observable with only two cached boundaries: op in {'norm', 'x', 'zz', 'z'}.

    Returns (ratio, norm_mantissa, norm_exponent)."""
    A = _check_sites(L, W, D, A)
    code = {"norm": 0, "x": 1, "zz": 2, "z": 3}[op]
    v, m, e = np.zeros(1), np.zeros(1), np.zeros(1, np.int64)
    rc = lib().or_peps_expect_one(L, W, D, _ptr(A), code, i, j, _ptr(v), _ptr(m), _ptr(e))
    if rc != 0:
        raise ValueError("sites are not nearest neighbours in (i, j) order")
    return float(v[0]), float(m[0]), int(e[0])


def ising_enumerate(L: int, W: int, K: float):
    """Classical Ising by enumeration: (log Z, <s_i s_j> per bond, <exp(-K s_k h_k)>)."""
    N = L * W
    nb = L * (W - 1) + W * (L - 1)
    logZ = np.zeros(1)
    corr, xf = np.zeros(max(nb, 1)), np.zeros(N)
    rc = lib().or_ising_enumerate(L, W, K, _ptr(logZ), _ptr(corr), _ptr(xf))
    if rc != 0:
        raise ValueError("too many sites to enumerate")
    return float(logZ[0]), corr[:nb], xf
