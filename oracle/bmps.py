"""Boundary-MPS approximate contraction, plainly -- TEST INFRASTRUCTURE ONLY.

The paper's exact method is limited by memory and names an environment
approximation as the missing piece for larger and more entangled lattices
(Sec. 7).  The standard one is the boundary MPS: the top row of the network is
a matrix product state (its down legs the physical ones), every further row is
applied to it as a matrix product operator, and the grown state is compressed
back to bond dimension chi_b before the next row:
  * right-to-left, each tensor is made right-orthonormal (QR of its
    transpose), the R factor pushed into the left neighbour;
  * left-to-right, each bond is cut by an SVD of its left tensor, keeping the
    chi_b largest singular values (U stays, S V^T is pushed into the right
    neighbour).
The last row closes the state into a scalar.  With chi_b at least the exact
boundary rank (d^floor(W/2) for a row of W legs of dimension d) nothing is
dropped and the result is the exact contraction.

Networks are grids of rank-4 tensors T[u][l][dn][rt] (legs of dimension 1 at
the lattice edge); a PEPS norm uses the double-layer tensors
T[(u u')(l l')(dn dn')(rt rt')] = sum_p A[p,u,l,dn,rt] A[p,u',l',dn',rt'].
Every tensor of the boundary is rescaled to max |entry| = 1 after each row,
the factors kept as a power-of-two exponent.
"""
from __future__ import annotations

import math

import numpy as np


def double_layer(A: np.ndarray, O: np.ndarray | None = None) -> np.ndarray:
    """sum_{p,q} A[p] O[p,q] A[q] with each leg pair (ket, bra) merged, ket major."""
    if O is None:
        O = np.eye(2)
    T = np.einsum("pabcd,pq,qefgh->aebfcgdh", A, O, A)
    u, l, n, r = A.shape[1:]
    return T.reshape(u * u, l * l, n * n, r * r)


def peps_grid(L: int, W: int, D: int, flat: np.ndarray, ops: dict | None = None):
    """Double-layer grid of a PEPS (ops: site -> 2x2 operator inserted there)."""
    from paper_1908_08553_gb300.inputs import split_sites   # input layout only
    sites = split_sites(np.asarray(flat, np.float64), L, W, D)
    ops = ops or {}
    return [double_layer(np.asarray(A), ops.get(k)) for k, A in enumerate(sites)]


def _rescale(t: np.ndarray):
    m = float(np.max(np.abs(t))) if t.size else 0.0
    if m == 0.0 or not math.isfinite(m):
        return t, 0
    e = math.frexp(m)[1]
    return t * 2.0 ** (-e), e


def compress(mps, chi: int):
    """Right-orthonormalise right to left, then truncate each bond left to right."""
    W = len(mps)
    mps = [m.copy() for m in mps]
    for c in range(W - 1, 0, -1):
        a, p, b = mps[c].shape
        Q, R = np.linalg.qr(mps[c].reshape(a, p * b).T)      # M^T = Q R -> M = R^T Q^T
        k = Q.shape[1]
        mps[c] = Q.T.reshape(k, p, b)
        mps[c - 1] = np.einsum("xpa,ka->xpk", mps[c - 1], R)  # times R^T on the right bond
    for c in range(W - 1):
        a, p, b = mps[c].shape
        U, s, Vt = np.linalg.svd(mps[c].reshape(a * p, b), full_matrices=False)
        k = min(chi, s.size)
        mps[c] = U[:, :k].reshape(a, p, k)
        mps[c + 1] = np.einsum("kb,bpy->kpy", s[:k, None] * Vt[:k], mps[c + 1])
    return mps


def contract(L: int, W: int, grid, chi: int):
    """Approximate value of the grid network as (mantissa, exponent): value = m 2^e."""
    e_tot = 0
    # top row: M_c[a = l][p = dn][b = rt] (u legs have dimension 1)
    mps = []
    for c in range(W):
        T = grid[c]
        mps.append(T.reshape(T.shape[1], T.shape[2], T.shape[3]))
    for r in range(1, L):
        new = []
        for c in range(W):
            T = grid[r * W + c]
            M = mps[c]
            a, _, b = M.shape
            N = np.einsum("aub,ulnr->alnbr", M, T)
            new.append(N.reshape(a * T.shape[1], T.shape[2], b * T.shape[3]))
        mps = compress(new, chi) if r < L - 1 else new
        scaled = []
        for M in mps:
            M, e = _rescale(M)
            e_tot += e
            scaled.append(M)
        mps = scaled
    # close: every physical leg now has dimension 1
    v = np.ones(1)
    for M in mps:
        v = v @ M[:, 0, :]
        v, e = _rescale(v)
        e_tot += e
    val = float(v[0])
    if val == 0.0:
        return 0.0, 0
    m, e = math.frexp(val)
    return m, e_tot + e


def norm(L: int, W: int, D: int, flat: np.ndarray, chi: int):
    """<Psi|Psi> of a PEPS by the boundary MPS with bond chi: (mantissa, exponent)."""
    return contract(L, W, peps_grid(L, W, D, flat), chi)


def expectation(L: int, W: int, D: int, flat: np.ndarray, chi: int, ops: dict) -> float:
    """<Psi| prod_k O_k |Psi> / <Psi|Psi> with both contracted by the boundary MPS."""
    m1, e1 = contract(L, W, peps_grid(L, W, D, flat, ops), chi)
    m0, e0 = contract(L, W, peps_grid(L, W, D, flat), chi)
    return m1 / m0 * 2.0 ** (e1 - e0)


def exact_rank(W: int, d: int) -> int:
    """Bond dimension that makes the boundary exact for a row of W legs of dimension d."""
    return d ** (W // 2)
