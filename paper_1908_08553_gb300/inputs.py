"""Seeded synthetic inputs shared by the CUDA path's tests/bench and the CPU oracle.

This module holds only input construction: the lattice leg dimensions, the
counter-based random generator and a few structured states used as pins.  It
holds none of the contraction arithmetic and imports neither the CUDA library
nor the oracle.

Site tensor layout (Sec. 5, the rank-5 PEPS tensor of one spin): for site
(r, c) of an L x W open-boundary lattice, ``A[p][u][l][dn][rt]`` in C order,
with the physical index p in {0, 1} (p = 1 is sigma = +1, Eq. Psi and the
binary map x = (sigma + 1) / 2) and bond legs of dimension D, or 1 where the
leg would leave the lattice (the paper's rank-3 edge and rank-2 corner tensors,
Sec. 4, written as rank 5 with unit legs).  Sites are stored one after another
in row-major site order.

Random generator: SplitMix64 (Steele, Lea & Flood, OOPSLA 2014) used as a
counter-based generator.  Element k of a lattice with seed s is
``mix64(s + (k + 1) * 0x9E3779B97F4A7C15)`` mapped to ``2 * (z >> 11) * 2**-53 - 1``,
uniform on [-1, 1).  Lattice k of a batch with seed b gets seed
``mix64(b + (k + 1) * 0x9E3779B97F4A7C15)``.  The C library's ``tn_fill_random``
implements the same definition and is checked against this one.
"""
from __future__ import annotations

import numpy as np

GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


def site_dims(L: int, W: int, D: int, r: int, c: int):
    """Bond dimensions (u, l, dn, rt) of site (r, c); 1 on the lattice edge."""
    return (1 if r == 0 else D, 1 if c == 0 else D,
            1 if r == L - 1 else D, 1 if c == W - 1 else D)


def site_sizes(L: int, W: int, D: int):
    """Number of FP64 entries of every site tensor, in row-major site order."""
    out = []
    for r in range(L):
        for c in range(W):
            u, l, dn, rt = site_dims(L, W, D, r, c)
            out.append(2 * u * l * dn * rt)
    return out


def n_elems(L: int, W: int, D: int) -> int:
    return int(sum(site_sizes(L, W, D)))


def _mix64(z: np.ndarray) -> np.ndarray:
    z = z.copy()
    z ^= z >> np.uint64(30)
    z *= _M1
    z ^= z >> np.uint64(27)
    z *= _M2
    z ^= z >> np.uint64(31)
    return z


def splitmix_u64(seed: int, count: int, start: int = 0) -> np.ndarray:
    """Outputs start..start+count-1 of the counter-based SplitMix64 stream."""
    k = np.arange(start + 1, start + count + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & 0xFFFFFFFFFFFFFFFF) + k * GAMMA
        return _mix64(z)


def uniform_pm1(seed: int, count: int) -> np.ndarray:
    """``count`` doubles uniform on [-1, 1) from ``seed``."""
    z = splitmix_u64(seed, count)
    u = (z >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)
    return 2.0 * u - 1.0


def lattice_seed(batch_seed: int, k: int) -> int:
    """Seed of lattice k of a batch drawn from ``batch_seed``."""
    return int(splitmix_u64(batch_seed, 1, start=k)[0])


def random_lattice(L: int, W: int, D: int, seed: int) -> np.ndarray:
    """Flat FP64 site tensors, i.i.d. uniform[-1, 1) from ``seed``."""
    return uniform_pm1(seed, n_elems(L, W, D))


def random_complex_lattice(L: int, W: int, D: int, seed: int) -> np.ndarray:
    """Flat complex site tensors: real parts the first n_elems draws of ``seed``,
    imaginary parts the next n_elems, each uniform[-1, 1)."""
    n = n_elems(L, W, D)
    u = uniform_pm1(seed, 2 * n)
    return u[:n] + 1j * u[n:]


def ones_lattice(L: int, W: int, D: int) -> np.ndarray:
    """Every entry 1: the workload of the paper's timing figures (Sec. 6)."""
    return np.ones(n_elems(L, W, D), dtype=np.float64)


def product_lattice(L: int, W: int, a0: np.ndarray, a1: np.ndarray) -> np.ndarray:
    """D = 1 product state: site k has amplitudes (a0[k], a1[k]) for p = 0, 1."""
    out = np.empty(2 * L * W)
    out[0::2] = np.asarray(a0, dtype=np.float64).ravel()
    out[1::2] = np.asarray(a1, dtype=np.float64).ravel()
    return out


def product_lattice_bonds(L: int, W: int, D: int, a0: np.ndarray, a1: np.ndarray, seed: int,
                          with_bonds: bool = False):
    """A product state written with bond dimension D: site k is
    (a0[k], a1[k]) on p times one seeded uniform[-1, 1) vector per bond,
    the same vector on both ends of the bond (edge legs: [1]).  Every bond
    contracts to the scalar |v|^2, so the amplitudes are those of the D = 1
    product state times a positive constant.  with_bonds: also return the
    horizontal and vertical bond vectors, shapes (L, W-1, D) and (L-1, W, D)."""
    rng = np.random.default_rng(seed)
    hv = rng.uniform(-1.0, 1.0, (L, max(W - 1, 0), D))   # bond (r, c)-(r, c+1)
    vv = rng.uniform(-1.0, 1.0, (max(L - 1, 0), W, D))   # bond (r, c)-(r+1, c)
    one = np.ones(1)
    a0 = np.asarray(a0, dtype=np.float64).ravel()
    a1 = np.asarray(a1, dtype=np.float64).ravel()
    sites = []
    for r in range(L):
        for c in range(W):
            u = vv[r - 1, c] if r > 0 else one
            l = hv[r, c - 1] if c > 0 else one
            dn = vv[r, c] if r < L - 1 else one
            rt = hv[r, c] if c < W - 1 else one
            p = np.array([a0[r * W + c], a1[r * W + c]])
            sites.append(np.einsum("p,u,l,d,r->puldr", p, u, l, dn, rt))
    return (join_sites(sites), hv, vv) if with_bonds else join_sites(sites)


def split_sites(flat: np.ndarray, L: int, W: int, D: int):
    """View the flat array as a list of rank-5 site tensors [p][u][l][dn][rt]."""
    out, off = [], 0
    for r in range(L):
        for c in range(W):
            u, l, dn, rt = site_dims(L, W, D, r, c)
            n = 2 * u * l * dn * rt
            out.append(flat[off:off + n].reshape(2, u, l, dn, rt))
            off += n
    return out


def join_sites(sites) -> np.ndarray:
    return np.concatenate([np.asarray(s, dtype=np.float64).ravel() for s in sites])


def ising_peps_lattice(L: int, W: int, K: float) -> np.ndarray:
    """D = 2 PEPS whose amplitude is prod over bonds of exp(K s_i s_j / 2), K >= 0.

    The bond weight w(s, s') = exp(K s s' / 2) is factored as Q Q^T with
    Q = V diag(sqrt(lambda)), V the eigenvectors of the 2x2 weight; each site
    tensor is prod over its present legs of Q[s(p), leg].  Its norm is the
    classical Ising partition function Z(K) and its correlators are classical
    averages, which the tests compute by enumeration.
    """
    if K < 0:
        raise ValueError("K >= 0 required for a real square-root factor")
    a, b = np.exp(K / 2), np.exp(-K / 2)
    Q = np.array([[np.sqrt((a + b) / 2), np.sqrt((a - b) / 2)],
                  [np.sqrt((a + b) / 2), -np.sqrt((a - b) / 2)]])
    # rows of Q are indexed by the spin: row 0 is s = -1, row 1 is s = +1; the
    # weight is symmetric in (s, s') and w(+,+) = w(-,-) = a, w(+,-) = b.
    sites = []
    for r in range(L):
        for c in range(W):
            u, l, dn, rt = site_dims(L, W, 2, r, c)
            A = np.zeros((2, u, l, dn, rt))
            for p in range(2):
                qu = Q[p, :u] if u > 1 else np.ones(1)
                ql = Q[p, :l] if l > 1 else np.ones(1)
                qd = Q[p, :dn] if dn > 1 else np.ones(1)
                qr = Q[p, :rt] if rt > 1 else np.ones(1)
                A[p] = np.einsum("a,b,c,d->abcd", qu, ql, qd, qr)
            sites.append(A)
    return join_sites(sites)


def bonds(L: int, W: int):
    """Nearest-neighbour bonds: horizontal row-major, then vertical row-major."""
    out = [((r, c), (r, c + 1)) for r in range(L) for c in range(W - 1)]
    out += [((r, c), (r + 1, c)) for r in range(L - 1) for c in range(W)]
    return out
