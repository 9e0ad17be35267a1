"""Pins of the oracle's boundary-MPS contraction (oracle/bmps.py), CPU only.

* With chi_b at least the exact boundary rank d^floor(W/2), the compression
  drops nothing: the norm equals the exact row-sweep norm, and expectation
  values equal the exact ones.
* On the single-layer classical Ising network (bond 2), the same holds against
  exact enumeration of Z(K); chi_b = 1 gives a different (approximate) value.
* The truncation error is small where it should be: chi_b = 8 on a 6x6 D = 2
  random PEPS (exact rank 64) is within 1% of the exact log norm.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.bmps as bm
from paper_1908_08553_gb300 import inputs
from test_oracle_pins import _ising_grid


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (5, 4, 2), (3, 6, 2), (4, 3, 3), (1, 5, 2), (5, 1, 2)])
def test_exact_rank_gives_the_exact_norm(L, W, D):
    A = inputs.random_lattice(L, W, D, 40 + L + W + D)
    m, e = oracle.norm(L, W, D, A)
    mb, eb = bm.norm(L, W, D, A, bm.exact_rank(W, D * D))
    assert abs((math.log2(abs(mb)) + eb) - (math.log2(abs(m)) + e)) < 1e-12 * max(1.0, abs(math.log2(abs(m)) + e))


def test_exact_rank_gives_exact_observables():
    L, W, D = 4, 4, 2
    A = inputs.random_lattice(L, W, D, 7)
    ob = oracle.observables(L, W, D, A)
    X, Z = np.array([[0.0, 1.0], [1.0, 0.0]]), np.diag([-1.0, 1.0])
    chi = bm.exact_rank(W, D * D)
    for k in (0, 5, 15):
        assert abs(bm.expectation(L, W, D, A, chi, {k: X}) - ob.sx[k]) < 1e-11
    bonds = inputs.bonds(L, W)
    for bi in (0, 7, 20):
        (ri, ci), (rj, cj) = bonds[bi]
        v = bm.expectation(L, W, D, A, chi, {ri * W + ci: Z, rj * W + cj: Z})
        assert abs(v - ob.szsz[bi]) < 1e-11


@pytest.mark.parametrize("L,W,K", [(4, 4, 0.4), (5, 5, 0.3), (3, 6, 0.8)])
def test_ising_partition_function(L, W, K):
    dims, ts = _ising_grid(L, W, K)
    grid = [np.asarray(t).reshape(tuple(d)) for t, d in zip(ts, dims)]
    logz, _, _ = oracle.ising_enumerate(L, W, K)
    m, e = bm.contract(L, W, grid, 2 ** (W // 2))
    assert abs(math.log(m) + e * math.log(2) - logz) < 1e-11 * logz
    m1, e1 = bm.contract(L, W, grid, 1)
    assert abs(math.log(m1) + e1 * math.log(2) - logz) > 1e-6


def test_truncation_error_is_small_at_moderate_chi():
    L, W, D = 6, 6, 2
    A = inputs.random_lattice(L, W, D, 77)
    m, e = oracle.norm(L, W, D, A)
    exact = math.log2(abs(m)) + e
    mb, eb = bm.norm(L, W, D, A, 8)
    assert abs(math.log2(abs(mb)) + eb - exact) < 0.01 * abs(exact)
    mb, eb = bm.norm(L, W, D, A, 64)
    assert abs(math.log2(abs(mb)) + eb - exact) < 1e-12 * abs(exact)
