"""Boundary-MPS approximate contraction on the GPU (tn_bmps_*) against the oracle.

* chi at the exact boundary rank: the GPU result is the exact contraction
  (the FP64 row-sweep oracle), norm and observables.
* Truncating chi: the GPU follows the oracle's boundary MPS (oracle/bmps.py,
  numpy QR and SVD) to rounding: the same compression keeps the same singular
  values, whatever the factorisation's gauge.
* The Ising PEPS norm is the enumerated partition function at the exact rank.
* FP32 (every tensor and SVD): the same results within 1e-5 relative (norm) and
  1e-4 absolute (observables), the truncation decisions unchanged.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.bmps as bm
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

X, Z = np.array([[0.0, 1.0], [1.0, 0.0]]), np.diag([-1.0, 1.0])


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _lat(ctx, L, W, D, A):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    tn.tn_set_site_tensors(lat, A)
    return lat


def _log2(m, e):
    return math.log2(abs(m)) + e


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (3, 5, 2), (4, 3, 3), (5, 2, 2), (1, 6, 2), (6, 1, 2)])
def test_exact_rank_is_exact(ctx, L, W, D):
    A = inputs.random_lattice(L, W, D, 300 + L * W + D)
    lat = _lat(ctx, L, W, D, A)
    try:
        chi = bm.exact_rank(W, D * D)
        m, e = tn.tn_bmps_norm(lat, chi)
        m0, e0 = oracle.norm(L, W, D, A)
        assert abs(_log2(m, e) - _log2(m0, e0)) < 1e-12 * max(1.0, abs(_log2(m0, e0)))
        r, sx, zz = tn.tn_bmps_energy(lat, chi, 1.0, 3.04, L, W)
        ob = oracle.observables(L, W, D, A)
        np.testing.assert_allclose(sx, ob.sx, atol=1e-10)
        np.testing.assert_allclose(zz, ob.szsz, atol=1e-10)
        assert abs(r.energy - ob.energy(1.0, 3.04)) <= 1e-10 * abs(ob.energy(1.0, 3.04))
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,D,chi", [(6, 6, 2, 4), (6, 6, 2, 8), (5, 7, 2, 6), (4, 4, 3, 12)])
def test_truncated_follows_the_oracle(ctx, L, W, D, chi):
    A = inputs.random_lattice(L, W, D, 900 + L + W + chi)
    lat = _lat(ctx, L, W, D, A)
    try:
        m, e = tn.tn_bmps_norm(lat, chi)
        mr, er = bm.norm(L, W, D, A, chi)
        assert abs(_log2(m, e) - _log2(mr, er)) < 1e-10 * abs(_log2(mr, er))
        for k in (0, W + 1, L * W - 1):
            v = tn.tn_bmps_expectation(lat, chi, tn.TN_OP_X, k)
            assert abs(v - bm.expectation(L, W, D, A, chi, {k: X})) < 1e-9
        # a longer-range pair, across the lattice
        i, j = 0, L * W - 1
        v = tn.tn_bmps_expectation(lat, chi, tn.TN_OP_Z, i, tn.TN_OP_Z, j)
        assert abs(v - bm.expectation(L, W, D, A, chi, {i: Z, j: Z})) < 1e-9
    finally:
        tn.tn_destroy_lattice(lat)


def test_energy_at_truncating_chi(ctx):
    L, W, D, chi = 4, 5, 2, 4
    A = inputs.random_lattice(L, W, D, 4545)
    lat = _lat(ctx, L, W, D, A)
    try:
        r, sx, zz = tn.tn_bmps_energy(lat, chi, 1.0, 2.0, L, W)
    finally:
        tn.tn_destroy_lattice(lat)
    for k in range(L * W):
        assert abs(sx[k] - bm.expectation(L, W, D, A, chi, {k: X})) < 1e-9
    for bi, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W)):
        assert abs(zz[bi] - bm.expectation(L, W, D, A, chi, {ri * W + ci: Z, rj * W + cj: Z})) < 1e-9
    assert abs(r.energy - (-zz.sum() - 2.0 * sx.sum())) < 1e-12 * max(1.0, abs(r.energy))


def test_ising_peps_partition_function(ctx):
    L, W, K = 5, 4, 0.35
    A = inputs.ising_peps_lattice(L, W, K)
    lat = _lat(ctx, L, W, 2, A)
    try:
        m, e = tn.tn_bmps_norm(lat, bm.exact_rank(W, 4))
    finally:
        tn.tn_destroy_lattice(lat)
    logz, _, _ = oracle.ising_enumerate(L, W, K)
    assert abs(_log2(m, e) * math.log(2) - logz) < 1e-11 * logz


@pytest.mark.parametrize("L,W,D,chi", [(4, 4, 2, 16), (4, 3, 3, 9), (6, 6, 2, 8), (5, 7, 2, 6)])
def test_fp32_follows_fp64(ctx, L, W, D, chi):
    A = inputs.random_lattice(L, W, D, 3200 + L + W + chi)
    lat = _lat(ctx, L, W, D, A)
    try:
        m, e = tn.tn_bmps_norm(lat, chi, tn.TN_FP32)
        mr, er = bm.norm(L, W, D, A, chi)
        assert abs(_log2(m, e) - _log2(mr, er)) < 1e-5 * max(1.0, abs(_log2(mr, er)))
        r32, sx32, zz32 = tn.tn_bmps_energy(lat, chi, 1.0, 3.04, L, W, tn.TN_FP32)
        r64, sx64, zz64 = tn.tn_bmps_energy(lat, chi, 1.0, 3.04, L, W, tn.TN_FP64)
        np.testing.assert_allclose(sx32, sx64, rtol=0, atol=1e-4)
        np.testing.assert_allclose(zz32, zz64, rtol=0, atol=1e-4)
        assert r32.precision == tn.TN_FP32
        v = tn.tn_bmps_expectation(lat, chi, tn.TN_OP_Z, 0, tn.TN_OP_Z, L * W - 1, tn.TN_FP32)
        assert abs(v - bm.expectation(L, W, D, A, chi, {0: Z, L * W - 1: Z})) < 1e-4
    finally:
        tn.tn_destroy_lattice(lat)
