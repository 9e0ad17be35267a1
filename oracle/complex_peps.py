"""Exact contraction of a complex PEPS, plainly -- TEST INFRASTRUCTURE ONLY.

The state of Eq. Psi with complex site tensors A[p][u][l][dn][rt] (same layout
as the real ones).  Every quantity of Sec. 3 is a ratio of two contractions of
the double-layer network (Sec. 5) whose site tensors are

    T_O[(u u')(l l')(dn dn')(rt rt')] = sum_{p,q} conj(A[p,u,l,dn,rt]) O[p,q] A[q,u',l',dn',rt']

(bra layer conjugated, O = I away from the inserted operators):

    <O_i ... >  =  contraction with T_O at the inserted sites / contraction with T_I.

The network is contracted row by row, site by site, with the boundary over the
legs cut between the finished and the open part of the lattice (the row order
of Sec. 4), in complex128, the boundary rescaled by a power of two after every
site and the factors kept as an integer exponent.

Operators are 2 x 2 matrices on the physical index p, p = 0 <-> sigma = -1 and
p = 1 <-> sigma = +1: X = [[0, 1], [1, 0]], Z = diag(-1, 1) and
Y = [[0, i], [-i, 0]] (the standard sigma_y with its rows and columns taken in
the order (sigma = -1, sigma = +1)).
"""
from __future__ import annotations

import math

import numpy as np

PAULI = {
    "i": np.eye(2, dtype=complex),
    "x": np.array([[0, 1], [1, 0]], dtype=complex),
    "y": np.array([[0, 1j], [-1j, 0]], dtype=complex),
    "z": np.array([[-1, 0], [0, 1]], dtype=complex),
}


def sites_of(L: int, W: int, D: int, A: np.ndarray):
    from paper_1908_08553_gb300.inputs import split_sites   # input layout only
    return split_sites(np.asarray(A, dtype=complex), L, W, D)


def double_layer(A: np.ndarray, O: np.ndarray) -> np.ndarray:
    """T_O with every leg pair (bra, ket) merged, bra index major."""
    T = np.einsum("pabcd,pq,qefgh->aebfcgdh", A.conj(), O, A)
    _, u, l, n, r = A.shape
    return T.reshape(u * u, l * l, n * n, r * r)


def _rescale(B: np.ndarray):
    m = float(np.max(np.abs(B))) if B.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return B, 0
    e = math.frexp(m)[1]
    return B * 2.0 ** (-e), e


def contract(L: int, W: int, grid) -> tuple[complex, int]:
    """Value of the network of rank-4 tensors grid[r*W+c][u][l][dn][rt] as (m, e), value = m 2^e.

    Before site (r, c) the boundary's axes are: dn of columns 0..c-1 of row r,
    the rt leg of site (r, c-1) (dimension 1 at c = 0), and dn of columns
    c..W-1 of row r-1 (dimension 1 for r = 0)."""
    B = np.ones([1] * (W + 1), dtype=complex)
    e_tot = 0
    for r in range(L):
        for c in range(W):
            T = grid[r * W + c]
            # contract the carried rt leg (axis c) with l and the dn leg of (r-1, c) (axis c+1) with u
            R = np.tensordot(B, T, axes=([c, c + 1], [1, 0]))
            # R axes: the other W-1 boundary axes in order, then dn, rt
            n = R.ndim
            order = list(range(c)) + [n - 2, n - 1] + list(range(c, n - 2))
            B, e = _rescale(np.transpose(R, order))
            e_tot += e
        # the last site's rt leg has dimension 1: it becomes the next row's carried leg
        B = np.moveaxis(B, W, 0)
    v = complex(B.reshape(-1)[0])
    if v == 0:
        return 0j, 0
    m, e = math.frexp(abs(v))
    return v / abs(v) * m, e_tot + e


def value(L: int, W: int, D: int, A: np.ndarray, ops: dict | None = None) -> tuple[complex, int]:
    """<Psi| prod_k O_k |Psi> (ops: site -> 2 x 2 matrix) as (mantissa, exponent)."""
    ops = ops or {}
    grid = [double_layer(S, ops.get(k, PAULI["i"])) for k, S in enumerate(sites_of(L, W, D, A))]
    return contract(L, W, grid)


def norm(L: int, W: int, D: int, A: np.ndarray) -> tuple[float, int]:
    """<Psi|Psi> as (mantissa, exponent), mantissa in [0.5, 1)."""
    m, e = value(L, W, D, A)
    return float(m.real), e


def expect(L: int, W: int, D: int, A: np.ndarray, ops: dict) -> complex:
    """<Psi| prod_k O_k |Psi> / <Psi|Psi>."""
    m1, e1 = value(L, W, D, A, ops)
    m0, e0 = value(L, W, D, A)
    return m1 / m0 * 2.0 ** (e1 - e0)


def site(L: int, W: int, D: int, A: np.ndarray, op: str, k: int) -> float:
    """<O_k> (Eq. mx and Eq. mz; Y likewise), real for a Hermitian O."""
    return float(expect(L, W, D, A, {k: PAULI[op]}).real)


def pair(L: int, W: int, D: int, A: np.ndarray, op_a: str, i: int, op_b: str, j: int) -> float:
    """<A_i B_j> for two distinct sites (Eq. cij for any pair)."""
    if i == j:
        raise ValueError("sites must differ")
    return float(expect(L, W, D, A, {i: PAULI[op_a], j: PAULI[op_b]}).real)


def observables(L: int, W: int, D: int, A: np.ndarray):
    """(log2 norm, <X_k>, <Y_k>, <Z_k>, <Z_i Z_j> per nearest-neighbour bond)."""
    from paper_1908_08553_gb300.inputs import bonds
    m0, e0 = norm(L, W, D, A)
    N = L * W
    sx = np.array([site(L, W, D, A, "x", k) for k in range(N)])
    sy = np.array([site(L, W, D, A, "y", k) for k in range(N)])
    sz = np.array([site(L, W, D, A, "z", k) for k in range(N)])
    zz = np.array([pair(L, W, D, A, "z", ri * W + ci, "z", rj * W + cj) for (ri, ci), (rj, cj) in bonds(L, W)])
    return math.log2(m0) + e0, sx, sy, sz, zz


def energy(sx: np.ndarray, zz: np.ndarray, J: float, h: float) -> float:
    """E = -J sum <Z_i Z_j> - h sum <X_k> (Eq. Etot)."""
    return float(-J * np.sum(zz) - h * np.sum(sx))
