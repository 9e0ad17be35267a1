"""Edge cases of the GPU path: the largest lattices the C-ABI accepts (16 x 16)
as D = 1 product states against their closed form, long chains (1 x 16,
16 x 1) and thin strips against the oracle, and the degenerate all-zero state
(a zero norm is reported as TN_ERR_NUMERIC, not as numbers)."""
import math

import numpy as np
import pytest

import oracle
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

PRECS = [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6]
TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _run(ctx, L, W, D, A, prec, h=3.04):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_energy_full(lat, 1.0, h, prec, tn.TN_SCHED_AUTO, L, W)
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("prec", PRECS)
def test_16x16_product_state_closed_form(ctx, prec):
    # D = 1: psi = prod_k (a0_k |0> + a1_k |1>); <X_k> = 2 a0 a1 / n_k,
    # <Z_k> = (a1^2 - a0^2) / n_k, <Z_i Z_j> = <Z_i><Z_j>, norm = prod n_k
    L = W = 16
    rng = np.random.default_rng(1616)
    a0, a1 = rng.uniform(-1, 1, L * W), rng.uniform(-1, 1, L * W)
    A = inputs.product_lattice(L, W, a0, a1)
    nk = a0 ** 2 + a1 ** 2
    sx_ref, sz_ref = 2 * a0 * a1 / nk, (a1 ** 2 - a0 ** 2) / nk
    zz_ref = np.array([sz_ref[ri * W + ci] * sz_ref[rj * W + cj] for (ri, ci), (rj, cj) in inputs.bonds(L, W)])
    r, sx, zz, sz, czz = _run(ctx, L, W, 1, A, prec)
    tol = TOL_OBS[prec]
    np.testing.assert_allclose(sx, sx_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(sz, sz_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(zz, zz_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(czz, 0.0, rtol=0, atol=2 * tol)
    log2n = float(np.sum(np.log2(nk)))
    assert abs(math.log2(r.norm.mant) + r.norm.exp2 - log2n) <= (1e-12 if prec == tn.TN_FP64 else 1e-5) * abs(log2n)
    e_ref = -float(np.sum(zz_ref)) - 3.04 * float(np.sum(sx_ref))
    check_energy(r.energy, e_ref, sx_ref, zz_ref, 1.0, 3.04, prec)


# (the oracle sweeps rows, so its boundary grows as d^W: strips are tall, not wide)
@pytest.mark.parametrize("L,W,D", [(1, 16, 2), (16, 1, 3), (1, 16, 4), (16, 2, 2), (16, 3, 2)])
def test_chains_and_strips_vs_oracle(ctx, L, W, D):
    A = inputs.random_lattice(L, W, D, 1600 + L + W + D)
    ref = oracle.observables(L, W, D, A, with_z=True)
    for prec in (tn.TN_FP64, tn.TN_FP32):
        r, sx, zz, sz, _ = _run(ctx, L, W, D, A, prec)
        tol = TOL_OBS[prec]
        np.testing.assert_allclose(sx, ref.sx, rtol=0, atol=tol)
        np.testing.assert_allclose(zz, ref.szsz, rtol=0, atol=tol)
        np.testing.assert_allclose(sz, ref.sz, rtol=0, atol=tol)
        check_energy(r.energy, ref.energy(1.0, 3.04), ref.sx, ref.szsz, 1.0, 3.04, prec)


@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32])
def test_zero_state_is_reported_not_computed(ctx, prec):
    L, W, D = 4, 4, 2
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, np.zeros(tn.tn_lattice_elems(L, W, D)))
        with pytest.raises(tn.TNError) as e:
            tn.tn_energy(lat, 1.0, 3.04, prec)
        assert e.value.status == tn.TN_ERR_NUMERIC
        with pytest.raises(tn.TNError) as e:
            tn.tn_contract_norm(lat, prec)
        assert e.value.status == tn.TN_ERR_NUMERIC
        # the context stays usable
        tn.tn_set_site_tensors(lat, inputs.random_lattice(L, W, D, 5))
        r = tn.tn_energy(lat, 1.0, 3.04, prec)
        assert math.isfinite(r.energy)
    finally:
        tn.tn_destroy_lattice(lat)
