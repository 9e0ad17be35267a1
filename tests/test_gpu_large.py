"""Large single instances (12x12 D=2, 8x8 D=3): parity at full size.

12x12 D=2: the FP32 and BF16x3 paths against the FP64 oracle on sampled
outputs it computes one by one (norm, sites, bonds, each with two cached
boundaries); every output of the reduced precisions against the FP64 GPU path;
the all-ones lattice exactly (norm 2^672, beyond the FP32 range, so the
power-of-two bookkeeping is exercised).
8x8 D=3 (the oracle would need hours): the FP64 GPU path is pinned at smaller
D=3 sizes in test_gpu_parity; here the all-ones closed form, order invariance
of the FP64 norm over the row, column and quadrant schemes, and the reduced
precisions against FP64 on every output.
"""
import math

import numpy as np
import pytest

import oracle
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _run(ctx, L, W, D, A, prec, sched=tn.TN_SCHED_AUTO, h=3.04):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_energy(lat, 1.0, h, prec, sched, L, W)
    finally:
        tn.tn_destroy_lattice(lat)


def _log2(r):
    return math.log2(abs(r.norm.mant)) + r.norm.exp2


def test_12x12_d2_sampled_oracle_and_fp64(ctx):
    L, W, D = 12, 12, 2
    A = inputs.random_lattice(L, W, D, 1212)
    r64, sx64, zz64 = _run(ctx, L, W, D, A, tn.TN_FP64)
    for prec, tol_obs in ((tn.TN_FP32, 1e-6), (tn.TN_BF16X3, 1e-5)):
        r, sx, zz = _run(ctx, L, W, D, A, prec)
        assert abs(r.energy - r64.energy) / (L * W) <= 1e-6 * max(1.0, abs(r64.energy) / (L * W))
        assert np.max(np.abs(sx - sx64)) <= tol_obs and np.max(np.abs(zz - zz64)) <= tol_obs
        assert abs(_log2(r) - _log2(r64)) <= 1e-6 * abs(_log2(r64))
    bonds = inputs.bonds(L, W)
    samples = [("x", 0, 0), ("x", 5 * W + 6, 0), ("zz", bonds[70][0][0] * W + bonds[70][0][1],
                                                     bonds[70][1][0] * W + bonds[70][1][1]),
               ("zz", bonds[200][0][0] * W + bonds[200][0][1], bonds[200][1][0] * W + bonds[200][1][1])]
    for op, i, j in samples:
        v, nm, ne = oracle.expect_one(L, W, D, A, op, i, j)
        got = sx64[i] if op == "x" else zz64[[(a[0] * W + a[1], b[0] * W + b[1]) for a, b in bonds].index((i, j))]
        assert abs(got - v) <= 1e-10, (op, i, j, got, v)
    assert abs(_log2(r64) - (math.log2(abs(nm)) + ne)) <= 1e-12 * abs(_log2(r64))


def test_12x12_d2_all_ones_exact(ctx):
    L, W = 12, 12
    A = inputs.ones_lattice(L, W, 2)
    for prec in (tn.TN_FP32, tn.TN_BF16X3):
        r, sx, zz = _run(ctx, L, W, 2, A, prec)
        N, nb = L * W, L * (W - 1) + W * (L - 1)
        assert r.norm.mant == 0.5 and r.norm.exp2 == N + 2 * nb + 1 == 673
        assert np.all(sx == 1.0) and np.all(zz == 0.0)


def test_8x8_d3_all_ones_closed_form(ctx):
    L, W, D = 8, 8, 3
    A = inputs.ones_lattice(L, W, D)
    r, sx, zz = _run(ctx, L, W, D, A, tn.TN_FP32)
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    assert abs(_log2(r) - (N + 2 * nb * math.log2(3))) <= 1e-6 * (N + 2 * nb * 2)
    np.testing.assert_allclose(sx, 1.0, atol=1e-6)
    np.testing.assert_allclose(zz, 0.0, atol=1e-6)


def test_8x8_d3_order_invariance_and_precisions(ctx):
    L, W, D = 8, 8, 3
    A = inputs.random_lattice(L, W, D, 883)
    c = ctx
    lat = tn.tn_create_lattice(c, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        logs = []
        for sched in (tn.TN_SCHED_AUTO, tn.TN_SCHED_ROW, tn.TN_SCHED_COL, tn.TN_SCHED_QUADRANT):
            m, e = tn.tn_contract_norm(lat, tn.TN_FP64, sched)
            logs.append(math.log2(abs(m)) + e)
        assert max(logs) - min(logs) <= 1e-12 * abs(logs[0])
    finally:
        tn.tn_destroy_lattice(lat)
    r64, sx64, zz64 = _run(c, L, W, D, A, tn.TN_FP64)
    assert abs(_log2(r64) - logs[0]) <= 1e-12 * abs(logs[0])
    for prec, tol_obs in ((tn.TN_FP32, 1e-6), (tn.TN_BF16X6, 1e-6), (tn.TN_BF16X3, 1e-5)):
        r, sx, zz = _run(c, L, W, D, A, prec)
        assert abs(r.energy - r64.energy) / (L * W) <= 1e-6 * max(1.0, abs(r64.energy) / (L * W))
        assert np.max(np.abs(sx - sx64)) <= tol_obs and np.max(np.abs(zz - zz64)) <= tol_obs
