"""GPU parity for complex PEPS (complex site tensors, bra layer conjugated)
against the complex FP64 oracle (oracle/complex_peps.py) and, at 16 sites, the
complex state vector: norm, every <X_k>, <Y_k>, <Z_k>, every bond <Z_i Z_j>, E,
and arbitrary pairs <A_i B_j> with A, B in {X, Y, Z}.  Tolerances as for the
real path: observables |d| <= tol * max(1, |value|) (FP64 1e-10, FP32 and
BF16x6 1e-6, BF16x3 1e-5); E by the precision's bound (energy_tol)."""
import itertools
import math

import numpy as np
import pytest

import oracle.brute as brute
import oracle.complex_peps as cp
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}
OPS = {"x": tn.TN_OP_X, "y": tn.TN_OP_Y, "z": tn.TN_OP_Z}
H = 3.04


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _gpu_all(ctx, L, W, D, A, prec):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors_complex(lat, A)
        assert tn.tn_lattice_is_complex(lat)
        r, sx, zz, sz, _ = tn.tn_energy_full(lat, 1.0, H, prec, tn.TN_SCHED_AUTO, L, W)
        sy = tn.tn_site_expectations(lat, prec, tn.TN_OP_Y, L, W)
        y0 = tn.tn_expectation(lat, prec, tn.TN_OP_Y, L * W - 1)
        assert y0 == sy[-1]
        return math.log2(r.norm.mant) + r.norm.exp2, r.energy, sx, sy, sz, zz
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (3, 5, 2), (3, 3, 3), (4, 4, 3), (1, 6, 2)])
def test_complex_fp64(ctx, L, W, D):
    A = inputs.random_complex_lattice(L, W, D, 900 + 13 * L + W + D)
    lg, e, sx, sy, sz, zz = _gpu_all(ctx, L, W, D, A, tn.TN_FP64)
    rlg, rsx, rsy, rsz, rzz = cp.observables(L, W, D, A)
    assert abs(lg - rlg) < 1e-10
    for got, ref in ((sx, rsx), (sy, rsy), (sz, rsz), (zz, rzz)):
        np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    assert np.abs(rsy).max() > 1e-3
    check_energy(e, cp.energy(rsx, rzz, 1.0, H), rsx, rzz, 1.0, H, tn.TN_FP64)
    if L * W <= 16:
        assert abs(e - brute.complex_energy(L, W, D, A, 1.0, H)) <= 1e-10 * abs(e)


@pytest.mark.parametrize("prec", [tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6])
@pytest.mark.parametrize("L,W,D", [(6, 6, 2), (4, 4, 3)])
def test_complex_reduced(ctx, prec, L, W, D):
    A = inputs.random_complex_lattice(L, W, D, 910 + L + D)
    lg, e, sx, sy, sz, zz = _gpu_all(ctx, L, W, D, A, prec)
    rlg, rsx, rsy, rsz, rzz = cp.observables(L, W, D, A)
    tol = TOL_OBS[prec]
    assert abs(lg - rlg) < 1e-4
    for got, ref in ((sx, rsx), (sy, rsy), (sz, rsz), (zz, rzz)):
        np.testing.assert_allclose(got, ref, rtol=0, atol=tol * max(1.0, float(np.abs(ref).max())))
    check_energy(e, cp.energy(rsx, rzz, 1.0, H), rsx, rzz, 1.0, H, prec)


@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_BF16X6])
def test_complex_pairs(ctx, prec):
    L, W, D = 4, 4, 3
    A = inputs.random_complex_lattice(L, W, D, 944)
    rng = np.random.default_rng(44)
    ij = np.array([rng.choice(L * W, 2, replace=False) for _ in range(12)], dtype=np.int32)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors_complex(lat, A)
        for a, b in itertools.product("xyz", repeat=2):
            got = tn.tn_pair_correlators(lat, prec, OPS[a], OPS[b], ij[:, 0], ij[:, 1])
            ref = np.array([cp.pair(L, W, D, A, a, int(i), b, int(j)) for i, j in ij])
            np.testing.assert_allclose(got, ref, rtol=0, atol=TOL_OBS[prec] * max(1.0, float(np.abs(ref).max())))
        bc = tn.tn_bond_correlators(lat, prec, tn.TN_OP_Y, tn.TN_OP_X, L, W)
        ref = np.array([cp.pair(L, W, D, A, "y", ri * W + ci, "x", rj * W + cj)
                        for (ri, ci), (rj, cj) in inputs.bonds(L, W)])
        np.testing.assert_allclose(bc, ref, rtol=0, atol=TOL_OBS[prec])
    finally:
        tn.tn_destroy_lattice(lat)


def test_state_vector_pairs_4x4(ctx):
    L, W, D = 4, 4, 2
    A = inputs.random_complex_lattice(L, W, D, 4416)
    ij = np.array([(i, j) for i in range(16) for j in range(16) if i != j], dtype=np.int32)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors_complex(lat, A)
        for a, b in (("y", "y"), ("x", "y"), ("y", "z")):
            got = tn.tn_pair_correlators(lat, tn.TN_FP64, OPS[a], OPS[b], ij[:, 0], ij[:, 1])
            ref = np.array([brute.pair_correlator(L, W, D, A, a, int(i), b, int(j)) for i, j in ij])
            np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    finally:
        tn.tn_destroy_lattice(lat)


def test_real_tensors_through_the_complex_path(ctx):
    # a real state given as complex: the Hermitian-basis site matrices give the
    # real path's results, and <Y_k> = 0
    L, W, D = 5, 5, 2
    A = inputs.random_lattice(L, W, D, 5525)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        r0, sx0, zz0, sz0, _ = tn.tn_energy_full(lat, 1.0, H, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
        tn.tn_set_site_tensors_complex(lat, A.astype(complex))
        r1, sx1, zz1, sz1, _ = tn.tn_energy_full(lat, 1.0, H, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
        sy = tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_Y, L, W)
        tn.tn_set_site_tensors(lat, A)               # back to real
        assert not tn.tn_lattice_is_complex(lat)
        r2 = tn.tn_energy(lat, 1.0, H, tn.TN_FP64)
    finally:
        tn.tn_destroy_lattice(lat)
    assert abs(r1.energy - r0.energy) <= 1e-12 * abs(r0.energy)
    for a, b in ((sx0, sx1), (zz0, zz1), (sz0, sz1)):
        np.testing.assert_allclose(b, a, rtol=0, atol=1e-12)
    assert np.abs(sy).max() < 1e-12
    assert r2.energy == r0.energy


def test_conjugate_state_flips_y(ctx):
    L, W, D = 4, 5, 2
    A = inputs.random_complex_lattice(L, W, D, 4520)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors_complex(lat, A)
        y = tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_Y, L, W)
        x = tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_X, L, W)
        tn.tn_set_site_tensors_complex(lat, np.conj(A))
        yc = tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_Y, L, W)
        xc = tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_X, L, W)
    finally:
        tn.tn_destroy_lattice(lat)
    np.testing.assert_allclose(yc, -y, rtol=0, atol=1e-12)
    np.testing.assert_allclose(xc, x, rtol=0, atol=1e-12)
