"""GPU parity for the nearest-neighbour two-site correlators <A_i B_j>,
A, B in {X, Z}, against the FP64 oracle element by element.  Tolerances as for
the other observables: |gpu - ref| <= tol * max(1, |ref|), FP64 1e-10, FP32
and BF16x6 1e-6, BF16x3 1e-5."""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}
OPS = {"x": tn.TN_OP_X, "z": tn.TN_OP_Z}
PAIRS = [("x", "x"), ("x", "z"), ("z", "x"), ("z", "z")]


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _bonds(ctx, L, W, D, A, prec, a, b):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_bond_correlators(lat, prec, OPS[a], OPS[b], L, W)
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("a,b", PAIRS)
@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (3, 5, 2), (3, 3, 3), (1, 6, 2)])
def test_bonds_fp64(ctx, L, W, D, a, b):
    A = inputs.random_lattice(L, W, D, 300 + 7 * L + W + D)
    got = _bonds(ctx, L, W, D, A, tn.TN_FP64, a, b)
    np.testing.assert_allclose(got, oracle.bond_correlators(L, W, D, A, a, b), rtol=0, atol=1e-10)
    if L * W <= 16:
        np.testing.assert_allclose(got, brute.bond_correlators(L, W, D, A, a, b), rtol=0, atol=1e-10)


@pytest.mark.parametrize("a,b", PAIRS)
@pytest.mark.parametrize("prec", [tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6])
def test_bonds_8x8_reduced(ctx, prec, a, b):
    L, W, D = 8, 8, 2
    A = inputs.random_lattice(L, W, D, 808)
    ref = oracle.bond_correlators(L, W, D, A, a, b)
    got = _bonds(ctx, L, W, D, A, prec, a, b)
    np.testing.assert_allclose(got, ref, rtol=0, atol=TOL_OBS[prec] * max(1.0, float(np.abs(ref).max())))


def test_zz_equals_energy_path(ctx):
    L, W, D = 5, 6, 2
    A = inputs.random_lattice(L, W, D, 56)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        zz = tn.tn_bond_correlators(lat, tn.TN_FP64, tn.TN_OP_Z, tn.TN_OP_Z, L, W)
        _, _, zz_e = tn.tn_energy(lat, 1.0, 3.04, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
    finally:
        tn.tn_destroy_lattice(lat)
    np.testing.assert_allclose(zz, zz_e, rtol=0, atol=1e-12)


def test_all_ones_xx_is_one(ctx):
    L, W = 6, 6
    got = _bonds(ctx, L, W, 2, inputs.ones_lattice(L, W, 2), tn.TN_FP32, "x", "x")
    assert np.all(got == 1.0)


def test_bad_operator_rejected(ctx):
    lat = tn.tn_create_lattice(ctx, 3, 3, 2)
    try:
        with pytest.raises(tn.TNError):
            tn.tn_bond_correlators(lat, tn.TN_FP64, tn.TN_OP_ZZ, tn.TN_OP_X, 3, 3)
    finally:
        tn.tn_destroy_lattice(lat)
