"""GPU parity for the single-site <Z_k> and the connected correlators
c_ij = <Z_i Z_j> - <Z_i><Z_j> (Sec. 3, Eqs. mz and cij) against the FP64
oracle, element by element.  Tolerances as for the other observables:
|gpu - ref| <= tol * max(1, |ref|), FP64 1e-10, FP32 and BF16x6 1e-6,
BF16x3 1e-5."""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _full(ctx, L, W, D, A, prec, sched=tn.TN_SCHED_AUTO):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_energy_full(lat, 1.0, 3.04, prec, sched, L, W)
    finally:
        tn.tn_destroy_lattice(lat)


def _close(a, b, tol):
    np.testing.assert_allclose(a, b, rtol=0, atol=tol * max(1.0, float(np.abs(b).max()) if b.size else 1.0))


@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6])
def test_c1_4x4_sz_all_precisions(ctx, prec):
    L, W, D = 4, 4, 2
    A = inputs.random_lattice(L, W, D, 1)
    ref = oracle.observables(L, W, D, A, with_z=True)
    r, sx, zz, sz, czz = _full(ctx, L, W, D, A, prec)
    _close(sz, ref.sz, TOL_OBS[prec])
    _close(czz, ref.connected(L, W), 2 * TOL_OBS[prec])
    if prec == tn.TN_FP64:
        _close(sz, brute.sz(L, W, D, A), 1e-10)


@pytest.mark.parametrize("L,W,D", [(1, 1, 2), (1, 5, 2), (3, 3, 3), (2, 5, 2), (5, 5, 2), (3, 4, 1)])
@pytest.mark.parametrize("sched", [tn.TN_SCHED_AUTO, tn.TN_SCHED_ROW, tn.TN_SCHED_COL, tn.TN_SCHED_QUADRANT])
def test_sz_shapes_fp64_all_schedules(ctx, L, W, D, sched):
    A = inputs.random_lattice(L, W, D, 900 + 13 * L + W + D)
    ref = oracle.observables(L, W, D, A, with_z=True)
    r, sx, zz, sz, czz = _full(ctx, L, W, D, A, tn.TN_FP64, sched)
    _close(sz, ref.sz, 1e-10)
    if czz.size:
        _close(czz, ref.connected(L, W), 1e-10)


@pytest.mark.parametrize("prec", [tn.TN_FP32, tn.TN_BF16X3])
def test_c2_8x8_sz(ctx, prec):
    L, W, D = 8, 8, 2
    A = inputs.random_lattice(L, W, D, 88)
    ref = oracle.observables(L, W, D, A, with_z=True)
    r, sx, zz, sz, czz = _full(ctx, L, W, D, A, prec)
    _close(sz, ref.sz, TOL_OBS[prec])
    _close(czz, ref.connected(L, W), 2 * TOL_OBS[prec])


def test_sz_zero_for_ising_peps(ctx):
    """psi(s) = psi(-s): every <Z_k> vanishes; c_ij equals the classical <s_i s_j>."""
    L, W, K = 4, 4, 0.6
    A = inputs.ising_peps_lattice(L, W, K)
    _, corr, _ = oracle.ising_enumerate(L, W, K)
    r, sx, zz, sz, czz = _full(ctx, L, W, 2, A, tn.TN_FP64)
    assert np.max(np.abs(sz)) <= 1e-12
    _close(czz, corr, 1e-10)


def test_expectation_z_entry_point(ctx):
    L, W, D = 3, 4, 2
    A = inputs.random_lattice(L, W, D, 12)
    ref = oracle.observables(L, W, D, A, with_z=True)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        for k in (0, 5, 11):
            v = tn.tn_expectation(lat, tn.TN_FP64, tn.TN_OP_Z, k)
            assert abs(v - ref.sz[k]) <= 1e-10
    finally:
        tn.tn_destroy_lattice(lat)
