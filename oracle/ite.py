"""Imaginary time evolution of the PEPS, plainly -- TEST INFRASTRUCTURE ONLY.

Sec. 5 (QMB Ground State Computation) evolves the initial state
|Psi> = prod_k (|+1> + |-1>)/sqrt 2 (every bond of dimension 1) by m steps of
  U(dtau) = U^Gamma(dtau/2) U^J(dtau) U^Gamma(dtau/2),
  U^Gamma(t) = exp(-H_Gamma t) = prod_k exp(Gamma t X_k),
  U^J(t)     = exp(-H_J t)     = prod_<ij> exp(J t Z_i Z_j),
(second-order Trotter-Suzuki split of H = -J sum Z Z - Gamma sum X, Eq.
Hamiltonian), normalising the state after every set of operators, and
evaluating the energy every two steps:
  * a one-body operator is contracted into the site's physical index;
  * a two-body operator is contracted with the two site tensors over their
    physical indices and the bond between them; the result is matricised
    (rows: the first site's physical index and other legs, columns: the
    second's), decomposed by SVD, and the sites are replaced by U sqrt(lambda)
    and sqrt(lambda) V^T (Fig. 3), keeping the singular values with
    lambda_k / lambda_1 >= eps (Sec. 6) and at most chi_max of them.

Readings where the paper is silent (stated here and in the design doc):
  * the bonds of one U^J set are updated in four classes of disjoint bonds:
    horizontal bonds whose left site has an even column, then odd, then
    vertical bonds whose upper site has an even row, then odd (the gates
    commute; the order only matters through truncation);
  * normalisation divides every site tensor by N^(1/(2 n_sites)), N the norm
    from the full contraction, which divides the state by sqrt(N);
  * the energy is evaluated after steps 2, 4, ... on the state at that point.

Bond dimensions vary from bond to bond here.  To contract, the state is zero-
padded to a uniform bond dimension (padded indices carry zeros, so the network
is unchanged) and handed to the exact FP64 row-sweep oracle.
"""
from __future__ import annotations

import math

import numpy as np


def product_plus(L: int, W: int):
    """The uniform superposition of Sec. 5 as L x W site tensors A[p][u][l][dn][rt] (chi = 1)."""
    A = []
    for _ in range(L * W):
        t = np.zeros((2, 1, 1, 1, 1))
        t[:, 0, 0, 0, 0] = 1.0 / math.sqrt(2.0)
        A.append(t)
    return A


def one_body_gate(gamma: float, t: float) -> np.ndarray:
    """exp(Gamma t X) = cosh(Gamma t) I + sinh(Gamma t) X."""
    c, s = math.cosh(gamma * t), math.sinh(gamma * t)
    return np.array([[c, s], [s, c]])


def two_body_gate(J: float, t: float) -> np.ndarray:
    """exp(J t Z_i Z_j) as g[p_i][p_j] (diagonal); Z = diag(-1, +1) on p = 0, 1."""
    z = np.array([-1.0, 1.0])
    return np.exp(J * t * np.outer(z, z))


def _keep(s: np.ndarray, chi_max: int, eps: float) -> int:
    if s.size == 0 or s[0] <= 0.0:
        return 1
    k = int(np.count_nonzero(s / s[0] >= eps))
    return max(1, min(k, chi_max))


def update_bond(Ai: np.ndarray, Aj: np.ndarray, g: np.ndarray, horizontal: bool, chi_max: int, eps: float):
    """Fig. 3 on one bond: returns (Ai', Aj', kept singular values, first discarded / largest)."""
    if horizontal:      # Ai [p,u,l,dn,b], Aj [q,v,b,m,r]
        th = np.einsum("pulnb,qvbmr->pulnqvmr", Ai, Aj)
        th = th * g[:, None, None, None, :, None, None, None]
        p, u, l, n = Ai.shape[:4]
        q, v, _, m, r = Aj.shape
        rows, cols = p * u * l * n, q * v * m * r
    else:               # Ai [p,u,l,b,r], Aj [q,b,x,n,y]
        th = np.einsum("pulbr,qbxny->pulrqxny", Ai, Aj)
        th = th * g[:, None, None, None, :, None, None, None]
        p, u, l, _, r = Ai.shape
        q, _, x, n, y = Aj.shape
        rows, cols = p * u * l * r, q * x * n * y
    U, s, Vt = np.linalg.svd(th.reshape(rows, cols), full_matrices=False)
    k = _keep(s, chi_max, eps)
    disc = float(s[k] / s[0]) if k < s.size and s[0] > 0 else 0.0
    sq = np.sqrt(s[:k])
    a = U[:, :k] * sq
    b = (sq[:, None] * Vt[:k]).reshape((k,) + th.shape[4:])
    if horizontal:
        Ai2 = a.reshape(p, u, l, n, k)
        Aj2 = np.transpose(b, (1, 2, 0, 3, 4))            # k,q,v,m,r -> q,v,k,m,r
    else:
        Ai2 = np.transpose(a.reshape(p, u, l, r, k), (0, 1, 2, 4, 3))   # -> p,u,l,k,r
        Aj2 = np.transpose(b, (1, 0, 2, 3, 4))            # k,q,x,n,y -> q,k,x,n,y
    return Ai2, Aj2, s[:k].copy(), disc


def bond_classes(L: int, W: int):
    """The four classes of disjoint bonds, in update order: (i, j, horizontal)."""
    out = []
    for par in (0, 1):
        out.append([(r * W + c, r * W + c + 1, True) for r in range(L) for c in range(par, W - 1, 2)])
    for par in (0, 1):
        out.append([(r * W + c, (r + 1) * W + c, False) for r in range(par, L - 1, 2) for c in range(W)])
    return out


def pad(A, L: int, W: int, D: int) -> np.ndarray:
    """Zero-pad every bond to dimension D (edge legs stay 1) in the flat input layout."""
    flat = []
    for r in range(L):
        for c in range(W):
            t = A[r * W + c]
            dims = (2, 1 if r == 0 else D, 1 if c == 0 else D, 1 if r == L - 1 else D, 1 if c == W - 1 else D)
            if any(a > b for a, b in zip(t.shape, dims)):
                raise ValueError(f"site {(r, c)} has a bond above {D}: {t.shape}")
            z = np.zeros(dims)
            z[tuple(slice(0, s) for s in t.shape)] = t
            flat.append(z.ravel())
    return np.concatenate(flat)


def unpad(flat: np.ndarray, L: int, W: int, D: int):
    """Flat uniform layout -> list of site tensors (bond dimension D)."""
    from paper_1908_08553_gb300.inputs import split_sites   # input layout only
    return [np.array(t) for t in split_sites(flat, L, W, D)]


def normalise(A, L: int, W: int, D: int):
    """Divide the state by sqrt(<Psi|Psi>) (full contraction by the FP64 oracle)."""
    import oracle
    m, e = oracle.norm(L, W, D, pad(A, L, W, D))
    log2n = math.log2(abs(m)) + e
    f = 2.0 ** (-log2n / (2 * L * W))
    return [t * f for t in A]


def evolve(L: int, W: int, J: float, gamma: float, dtau: float, steps: int, chi_max: int, eps: float,
           energy_every: int = 2, A=None):
    """Run the ITE; returns dict(energies=[(step, E)], flat=padded final state,
    bond_dims=[per bond, bond order of inputs.bonds], max_discarded=largest
    lambda_k / lambda_1 dropped, A=site tensors)."""
    import oracle
    from paper_1908_08553_gb300.inputs import bonds
    D = chi_max
    A = product_plus(L, W) if A is None else [np.array(t) for t in A]
    g1 = one_body_gate(gamma, dtau / 2.0)
    g2 = two_body_gate(J, dtau)
    classes = bond_classes(L, W)
    energies, max_disc = [], 0.0
    for step in range(1, steps + 1):
        A = [np.einsum("pq,qulnr->pulnr", g1, t) for t in A]
        A = normalise(A, L, W, D)
        for cls in classes:
            for i, j, hz in cls:
                A[i], A[j], _, disc = update_bond(A[i], A[j], g2, hz, chi_max, eps)
                max_disc = max(max_disc, disc)
        A = normalise(A, L, W, D)
        A = [np.einsum("pq,qulnr->pulnr", g1, t) for t in A]
        A = normalise(A, L, W, D)
        if energy_every and step % energy_every == 0:
            ob = oracle.observables(L, W, D, pad(A, L, W, D))
            energies.append((step, ob.energy(J, gamma)))
    dims = []
    for (ri, ci), (rj, cj) in bonds(L, W):
        t = A[ri * W + ci]
        dims.append(t.shape[4] if ri == rj else t.shape[3])
    return {"energies": energies, "flat": pad(A, L, W, D), "bond_dims": dims, "max_discarded": max_disc, "A": A}
