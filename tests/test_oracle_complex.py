"""Pins of the complex-PEPS oracle (oracle/complex_peps.py) against things other
than itself: the complex 2^N state vector (Eq. Psi evaluated amplitude by
amplitude, no double layer), the real C oracle on real inputs, the D = 1
product-state closed forms (the Bloch vector of each spin), and three exact
invariances of Eqs. mx, mz and cij: a phase on one site tensor, a complex
gauge transformation G G^-1 on one bond, and complex conjugation of every
tensor (which leaves <X>, <Z>, <Z Z>, <Y Y> and flips <Y>)."""
import cmath

import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.complex_peps as cp
from paper_1908_08553_gb300 import inputs


@pytest.mark.parametrize("L,W,D,seed", [(3, 3, 2, 1), (2, 4, 3, 2), (4, 4, 2, 3), (1, 5, 2, 4)])
def test_against_state_vector(L, W, D, seed):
    A = inputs.random_complex_lattice(L, W, D, seed)
    lg, sx, sy, sz, zz = cp.observables(L, W, D, A)
    psi = brute.state_vector(L, W, D, A)
    assert abs(lg - np.log2(np.vdot(psi, psi).real)) < 1e-12
    N = L * W
    for k in range(N):
        assert abs(sx[k] - brute.site_expectation(L, W, D, A, "x", k)) < 1e-12
        assert abs(sy[k] - brute.site_expectation(L, W, D, A, "y", k)) < 1e-12
        assert abs(sz[k] - brute.site_expectation(L, W, D, A, "z", k)) < 1e-12
    assert np.abs(sy).max() > 1e-3          # a complex state has <Y> != 0
    for b, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W)):
        ref = brute.pair_correlator(L, W, D, A, "z", ri * W + ci, "z", rj * W + cj)
        assert abs(zz[b] - ref) < 1e-12
    rng = np.random.default_rng(seed)
    for _ in range(6):
        i, j = rng.choice(N, size=2, replace=False)
        for a, b in (("x", "y"), ("y", "y"), ("z", "x"), ("y", "z")):
            assert abs(cp.pair(L, W, D, A, a, int(i), b, int(j)) -
                       brute.pair_correlator(L, W, D, A, a, int(i), b, int(j))) < 1e-12
    e = cp.energy(sx, zz, 1.0, 3.04)
    assert abs(e - brute.complex_energy(L, W, D, A, 1.0, 3.04)) < 1e-11 * max(1.0, abs(e))


@pytest.mark.parametrize("L,W,D", [(3, 4, 2), (3, 3, 3)])
def test_real_input_matches_real_oracle(L, W, D):
    A = inputs.random_lattice(L, W, D, 40 + L + W + D)
    ref = oracle.observables(L, W, D, A, with_z=True)
    lg, sx, sy, sz, zz = cp.observables(L, W, D, A.astype(complex))
    assert abs(lg - ref.log2_norm) < 1e-12
    np.testing.assert_allclose(sx, ref.sx, rtol=0, atol=1e-13)
    np.testing.assert_allclose(sz, ref.sz, rtol=0, atol=1e-13)
    np.testing.assert_allclose(zz, ref.szsz, rtol=0, atol=1e-13)
    assert np.abs(sy).max() < 1e-14          # real amplitudes: <Y> = 0


def test_product_state_bloch_vector():
    # D = 1: site k is a0 |p=0> + a1 |p=1>; <X> = 2 Re(a0* a1) / n,
    # <Y> = -2 Im(a0* a1) / n, <Z> = (|a1|^2 - |a0|^2) / n, n = |a0|^2 + |a1|^2,
    # and every pair factorises
    L, W = 2, 3
    rng = np.random.default_rng(5)
    a = rng.uniform(-1, 1, (L * W, 2)) + 1j * rng.uniform(-1, 1, (L * W, 2))
    A = np.empty(2 * L * W, dtype=complex)
    A[0::2], A[1::2] = a[:, 0], a[:, 1]
    n = np.abs(a[:, 0]) ** 2 + np.abs(a[:, 1]) ** 2
    c = np.conj(a[:, 0]) * a[:, 1]
    bloch = {"x": 2 * c.real / n, "y": -2 * c.imag / n, "z": (np.abs(a[:, 1]) ** 2 - np.abs(a[:, 0]) ** 2) / n}
    for op, v in bloch.items():
        got = np.array([cp.site(L, W, 1, A, op, k) for k in range(L * W)])
        np.testing.assert_allclose(got, v, rtol=0, atol=1e-14)
    for (i, j) in ((0, 5), (1, 3), (4, 2)):
        for p, q in (("x", "y"), ("y", "y"), ("z", "y")):
            assert abs(cp.pair(L, W, 1, A, p, i, q, j) - bloch[p][i] * bloch[q][j]) < 1e-14


def _all(L, W, D, A):
    lg, sx, sy, sz, zz = cp.observables(L, W, D, A)
    return sx, sy, sz, zz, cp.pair(L, W, D, A, "y", 0, "y", L * W - 1)


def test_phase_and_gauge_invariance_and_conjugation():
    L, W, D = 3, 3, 2
    A = inputs.random_complex_lattice(L, W, D, 77)
    base = _all(L, W, D, A)
    sites = [s.copy() for s in inputs.split_sites(A, L, W, D)]
    # a phase on site 4
    ph = [s.copy() for s in sites]
    ph[4] = ph[4] * cmath.exp(0.7j)
    # a complex gauge on the horizontal bond (1,0)-(1,1) and the vertical bond (0,2)-(1,2)
    rng = np.random.default_rng(3)
    G = rng.uniform(-1, 1, (D, D)) + 1j * rng.uniform(-1, 1, (D, D)) + 2 * np.eye(D)
    Gi = np.linalg.inv(G)
    ga = [s.copy() for s in sites]
    ga[3] = np.einsum("pulda,ab->puldb", ga[3], G)       # rt leg of (1,0)
    ga[4] = np.einsum("ab,pubdr->puadr", Gi, ga[4])      # l leg of (1,1)
    ga[2] = np.einsum("pulad,ab->pulbd", ga[2], G)       # dn leg of (0,2)
    ga[5] = np.einsum("ab,pbldr->paldr", Gi, ga[5])      # u leg of (1,2)
    for variant in (ph, ga):
        B = np.concatenate([s.ravel() for s in variant])
        for x, y in zip(base, _all(L, W, D, B)):
            np.testing.assert_allclose(y, x, rtol=0, atol=1e-12)
    sx, sy, sz, zz, yy = _all(L, W, D, np.conj(A))
    np.testing.assert_allclose(sx, base[0], rtol=0, atol=1e-13)
    np.testing.assert_allclose(sy, -base[1], rtol=0, atol=1e-13)
    np.testing.assert_allclose(sz, base[2], rtol=0, atol=1e-13)
    np.testing.assert_allclose(zz, base[3], rtol=0, atol=1e-13)
    assert abs(yy - base[4]) < 1e-13
