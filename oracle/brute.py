"""Brute-force 2^N state vector for small lattices -- TEST INFRASTRUCTURE ONLY.

The amplitudes A(sigma) of Eq. Psi are built as a full state vector by
absorbing the single-layer site tensors one at a time while keeping every
physical leg open (never forming a double layer), then every quantity of
Sec. 3 is evaluated directly on the vector:

  norm        = sum_sigma A(sigma)^2                        (Eq. norm)
  <X_k>       = sum_sigma A(sigma) A(sigma with k flipped) / norm   (Eq. mx)
  <Z_i Z_j>   = sum_sigma A(sigma)^2 sigma_i sigma_j / norm (Eq. cij, 1st term)
  E           = <Psi|H|Psi> / norm with H built as a sparse matrix from
                Kronecker products (Eqs. Hamiltonian, Etot), and the exact
                ground energy E_0 of that H by Lanczos (scipy eigsh).

Basis convention: site k (row-major) is bit k of the basis index, bit = p, and
p = 1 means sigma = +1 (x = (sigma + 1) / 2, Sec. 3).
"""
from __future__ import annotations

import numpy as np


def state_vector(L: int, W: int, D: int, flat: np.ndarray) -> np.ndarray:
    """psi[index] with bit k of index = p of site k (row-major)."""
    from paper_1908_08553_gb300.inputs import split_sites  # input layout only
    flat = np.asarray(flat)
    if not np.iscomplexobj(flat):
        flat = flat.astype(np.float64)
    sites = split_sites(flat, L, W, D)
    # T axes: [phys bits 0..k-1 (2 each, site 0 first)] + boundary legs
    # boundary before site (r, c): dn_0..dn_{c-1} of row r, h, u_c..u_{W-1}
    T = np.ones([1] * (W + 1), dtype=flat.dtype)  # h + W u-legs of row 0, all of dimension 1
    nphys = 0
    for r in range(L):
        for c in range(W):
            A = sites[r * W + c]  # [p][u][l][dn][rt]
            # boundary axes start after nphys; position of h is nphys + c,
            # position of u_c is nphys + c + 1
            ah, au = nphys + c, nphys + c + 1
            # contract h with l and u_c with u -> result axes: rest of T + (p, dn, rt)
            R = np.tensordot(T, A, axes=([ah, au], [2, 1]))
            # R axes: T axes without (ah, au) in order, then p, dn, rt
            nT = T.ndim - 2
            p_ax, dn_ax, rt_ax = nT, nT + 1, nT + 2
            # move p to position nphys (after the previous physical bits),
            # dn to position nphys + 1 + c, rt right after it
            order = list(range(nT))
            phys = order[:nphys]
            rest = order[nphys:]
            new = phys + [p_ax] + rest[:c] + [dn_ax, rt_ax] + rest[c:]
            T = np.transpose(R, new)
            nphys += 1
        # end of the row: the trailing h' (rt of the last column) has dim 1;
        # re-insert a fresh dim-1 h before the dn legs for the next row
        T = T.reshape(T.shape[:nphys] + T.shape[nphys:nphys + W] + (1,))
        T = np.moveaxis(T, -1, nphys)
    psi = T.reshape(T.shape[:nphys])
    # psi axes: site 0 .. N-1; index bit k must be p of site k -> site k is the
    # k-th least significant bit, so reverse the axis order before flattening
    psi = np.transpose(psi, list(range(nphys))[::-1]).reshape(-1)
    return psi


def observables(L: int, W: int, D: int, flat: np.ndarray):
    """(norm, <X_k>[N], <Z_i Z_j>[nb]) straight from the state vector."""
    from paper_1908_08553_gb300.inputs import bonds
    psi = state_vector(L, W, D, flat)
    N = L * W
    idx = np.arange(psi.size)
    norm = float(psi @ psi)
    sx = np.empty(N)
    for k in range(N):
        sx[k] = float(psi @ psi[idx ^ (1 << k)]) / norm
    sig = [np.where((idx >> k) & 1, 1.0, -1.0) for k in range(N)]
    zz = []
    for (ri, ci), (rj, cj) in bonds(L, W):
        i, j = ri * W + ci, rj * W + cj
        zz.append(float(np.sum(psi * psi * sig[i] * sig[j])) / norm)
    return norm, sx, np.array(zz)


def sz(L: int, W: int, D: int, flat: np.ndarray) -> np.ndarray:
    """<Z_k>[N] straight from the state vector (p = 1 <-> sigma = +1)."""
    psi = state_vector(L, W, D, flat)
    idx = np.arange(psi.size)
    w = psi * psi
    return np.array([float(np.sum(w * np.where((idx >> k) & 1, 1.0, -1.0))) for k in range(L * W)]) / float(w.sum())


def bond_correlators(L: int, W: int, D: int, flat: np.ndarray, op_a: str, op_b: str) -> np.ndarray:
    """<A_i B_j> per nearest-neighbour bond from the state vector (X flips the
    site's bit, Z multiplies by its sign)."""
    from paper_1908_08553_gb300.inputs import bonds
    psi = state_vector(L, W, D, flat)
    idx = np.arange(psi.size)

    def apply(op, k, v):
        if op == "x":
            return v[idx ^ (1 << k)]
        return v * np.where((idx >> k) & 1, 1.0, -1.0)

    out = []
    for (ri, ci), (rj, cj) in bonds(L, W):
        i, j = ri * W + ci, rj * W + cj
        out.append(float(psi @ apply(op_a, i, apply(op_b, j, psi))))
    return np.array(out) / float(psi @ psi)


def hamiltonian(L: int, W: int, J: float, h: float):
    """Sparse TFIM Hamiltonian -J sum Z_i Z_j - h sum X_k on the 2^N basis."""
    import scipy.sparse as sp
    from paper_1908_08553_gb300.inputs import bonds
    N = L * W
    dim = 1 << N
    idx = np.arange(dim)
    diag = np.zeros(dim)
    for (ri, ci), (rj, cj) in bonds(L, W):
        i, j = ri * W + ci, rj * W + cj
        si = np.where((idx >> i) & 1, 1.0, -1.0)
        sj = np.where((idx >> j) & 1, 1.0, -1.0)
        diag -= J * si * sj
    rows, cols, vals = [idx], [idx], [diag]
    for k in range(N):
        rows.append(idx)
        cols.append(idx ^ (1 << k))
        vals.append(np.full(dim, -h))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                         shape=(dim, dim))


def energy(L: int, W: int, D: int, flat: np.ndarray, J: float, h: float) -> float:
    psi = state_vector(L, W, D, flat)
    H = hamiltonian(L, W, J, h)
    return float(psi @ (H @ psi)) / float(psi @ psi)


def ground_energy(L: int, W: int, J: float, h: float) -> float:
    from scipy.sparse.linalg import eigsh
    H = hamiltonian(L, W, J, h)
    w = eigsh(H, k=1, which="SA", return_eigenvectors=False, tol=1e-10)
    return float(w[0])


def _pauli_p(name: str) -> np.ndarray:
    """Pauli matrix on the p basis: the standard one on (sigma = +1, sigma = -1)
    with rows and columns reversed (p = 1 - position)."""
    std = {"x": np.array([[0, 1], [1, 0]], complex), "y": np.array([[0, -1j], [1j, 0]]),
           "z": np.array([[1, 0], [0, -1]], complex)}
    return std[name][::-1, ::-1]


def _apply(M: np.ndarray, k: int, v: np.ndarray) -> np.ndarray:
    """(M acting on site k) v: (M v)[s] = M[s_k, s_k] v[s] + M[s_k, 1 - s_k] v[s with k flipped]."""
    idx = np.arange(v.size)
    bit = (idx >> k) & 1
    return M[bit, bit] * v + M[bit, 1 - bit] * v[idx ^ (1 << k)]


def _ratio(psi: np.ndarray, w: np.ndarray):
    val = np.vdot(psi, w) / np.vdot(psi, psi)
    return float(val.real) if abs(val.imag) < 1e-12 * max(1.0, abs(val)) else complex(val)


def pair_correlator(L: int, W: int, D: int, flat: np.ndarray, op_a: str, i: int, op_b: str, j: int) -> float:
    """<A_i B_j> = psi^dagger A_i B_j psi / psi^dagger psi for any sites i != j,
    A, B in {'x', 'y', 'z'} as complex 2 x 2 Pauli matrices on the basis
    (p = 0 <-> sigma = -1, p = 1 <-> sigma = +1), applied to the state vector
    (real or complex site tensors)."""
    psi = state_vector(L, W, D, flat).astype(np.complex128)
    N = L * W
    assert 0 <= i < N and 0 <= j < N and i != j
    return _ratio(psi, _apply(_pauli_p(op_a), i, _apply(_pauli_p(op_b), j, psi)))


def site_expectation(L: int, W: int, D: int, flat: np.ndarray, op: str, k: int) -> float:
    """<O_k> = psi^dagger O_k psi / psi^dagger psi, O in {'x', 'y', 'z'}."""
    psi = state_vector(L, W, D, flat).astype(np.complex128)
    return _ratio(psi, _apply(_pauli_p(op), k, psi))


def complex_energy(L: int, W: int, D: int, flat: np.ndarray, J: float, h: float) -> float:
    """psi^dagger H psi / psi^dagger psi with the sparse TFIM Hamiltonian."""
    psi = state_vector(L, W, D, flat).astype(np.complex128)
    H = hamiltonian(L, W, J, h)
    return float((np.vdot(psi, H @ psi) / np.vdot(psi, psi)).real)
