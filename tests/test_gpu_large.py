"""Large single instances (12x12 D=2, 8x8 D=3): parity at full size.

Against the FP64 oracle: tests/golden/large_samples.json holds oracle values
computed one by one (norm, a site <X_k>, <Z_i Z_j> on bonds inside a corner and
across both cuts of the quadrant partition), written by
tests/golden/make_large.py, which calls only the oracle.  Every precision's
norm and sampled observables are compared with them; the FP64 GPU path, pinned
there at 1e-10, then serves as the reference for every other output and for E
(the whole observable set of the 8x8 D=3 lattice would take the oracle hours).
Also: the all-ones lattices exactly (12x12: norm 2^672, beyond the FP32
range, so the power-of-two bookkeeping is exercised), order invariance of the
8x8 D=3 FP64 norm over four schedules.
"""
import json
import math
import os

import numpy as np
import pytest

from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden", "large_samples.json")
TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X6: 1e-6, tn.TN_BF16X3: 1e-5}


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


def _golden(L, W, D):
    with open(GOLDEN) as f:
        for c in json.load(f)["cases"]:
            if (c["L"], c["W"], c["D"]) == (L, W, D):
                return c
    raise AssertionError(f"no golden samples for {L}x{W} D={D}")


def _sampled(case, sx, zz, W):
    """(golden value, our value, what) for every sample of the case."""
    L = case["L"]
    bonds = [(a[0] * W + a[1], b[0] * W + b[1]) for a, b in inputs.bonds(L, W)]
    out = []
    for s in case["samples"]:
        got = sx[s["i"]] if s["op"] == "x" else zz[bonds.index((s["i"], s["j"]))]
        out.append((s["value"], got, s["what"]))
    return out


@pytest.mark.parametrize("L,W,D", [(12, 12, 2), (8, 8, 3)])
def test_large_against_oracle_samples(ctx, L, W, D):
    case = _golden(L, W, D)
    A = inputs.random_lattice(L, W, D, case["seed"])
    lg_ref = math.log2(abs(case["samples"][0]["norm_mant"])) + case["samples"][0]["norm_exp2"]
    r64, sx64, zz64 = _run(ctx, L, W, D, A, tn.TN_FP64)
    assert abs(_log2(r64) - lg_ref) <= 1e-12 * abs(lg_ref)
    for v_ref, got, what in _sampled(case, sx64, zz64, W):
        assert abs(got - v_ref) <= 1e-10 * max(1.0, abs(v_ref)), (what, got, v_ref)
    for prec in (tn.TN_FP32, tn.TN_BF16X6, tn.TN_BF16X3):
        r, sx, zz = _run(ctx, L, W, D, A, prec)
        tol = TOL_OBS[prec]
        assert abs(_log2(r) - lg_ref) <= 1e-6 * abs(lg_ref), prec
        for v_ref, got, what in _sampled(case, sx, zz, W):
            assert abs(got - v_ref) <= tol * max(1.0, abs(v_ref)), (prec, what, got, v_ref)
        # every other output and E against the FP64 path pinned above
        assert np.max(np.abs(sx - sx64)) <= tol and np.max(np.abs(zz - zz64)) <= tol, prec
        check_energy(r.energy, r64.energy, sx64, zz64, 1.0, 3.04, prec)


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


def test_8x8_d3_order_invariance(ctx):
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
