"""The recompute form of the energy program (program choice bit 32): the
forward chains keep only the states that start a frame row, and every other
state is absorbed again from the checkpoint before it where an observable
needs it.  The ops and their inputs are those of the cached form, so every
result equals the cached form's bit for bit, in every precision, for the
energy, arbitrary pairs, the bond work kinds and complex tensors.  The lattice
API and batch groups fall back to it when the cached chain states exceed the
budget.  At the full sizes (9 x 9 and 10 x 10, D = 3), where no oracle runs,
the forms are compared with each other and with a product state's closed
form."""
import math

import numpy as np
import pytest

import oracle
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

RECOMPUTE = 32
E = tn.TN_WORK_ENERGY
PRECS = [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6]
SHAPES = [(4, 4, 2), (5, 5, 2), (6, 6, 2), (8, 8, 2), (3, 7, 2), (5, 7, 3), (6, 6, 3), (4, 9, 3), (2, 6, 3),
          (1, 7, 2), (5, 4, 4)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


@pytest.fixture(autouse=True)
def clean_table():
    tn.tn_autotune_clear()
    yield
    tn.tn_autotune_clear()


def _energy(ctx, L, W, D, A, prec, knobs=None, h=3.04, cplx=False):
    if knobs is not None:
        tn.tn_autotune_set(L, W, D, prec, E, knobs)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        if cplx:
            tn.tn_set_site_tensors_complex(lat, A)
        else:
            tn.tn_set_site_tensors(lat, A)
        r, sx, zz, sz, czz = tn.tn_energy_full(lat, 1.0, h, prec, tn.TN_SCHED_AUTO, L, W)
        sy = tn.tn_site_expectations(lat, prec, tn.TN_OP_Y, L, W) if cplx else None
        return (r.energy, r.norm.mant, r.norm.exp2), sx.copy(), zz.copy(), sz.copy(), sy
    finally:
        tn.tn_destroy_lattice(lat)


def _same(a, b):
    for x, y in zip(a, b):
        if x is None:
            assert y is None
        elif isinstance(x, tuple):
            assert x == y
        else:
            assert np.array_equal(x, y)


@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L,W,D", SHAPES)
def test_recompute_equals_cached(ctx, L, W, D, prec):
    A = inputs.random_lattice(L, W, D, 9100 + 17 * L + W + D)
    cached = _energy(ctx, L, W, D, A, prec, 15)
    rec = _energy(ctx, L, W, D, A, prec, 15 | RECOMPUTE)
    _same(cached, rec)
    if (L, W, D) in ((5, 5, 2), (5, 7, 3)) and prec in (tn.TN_FP64, tn.TN_FP32):
        ref = oracle.observables(L, W, D, A, with_z=True)
        check_energy(rec[0][0], ref.energy(1.0, 3.04), ref.sx, ref.szsz, 1.0, 3.04, prec)


@pytest.mark.parametrize("knobs", [0, 11, 23, 31])
def test_recompute_with_other_choices(ctx, knobs):
    # the recompute bit combined with the other program choices
    for (L, W, D, prec) in [(6, 6, 2, tn.TN_FP32), (5, 5, 3, tn.TN_BF16X6)]:
        A = inputs.random_lattice(L, W, D, 9200 + knobs)
        _same(_energy(ctx, L, W, D, A, prec, knobs), _energy(ctx, L, W, D, A, prec, knobs | RECOMPUTE))


@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X6])
def test_recompute_pairs(ctx, prec):
    # arbitrary pairs: inside one corner, adjacent corners and diagonal corners
    for (L, W, D) in [(6, 6, 2), (5, 6, 3)]:
        A = inputs.random_lattice(L, W, D, 9300 + L + W + D)
        rng = np.random.default_rng(93)
        N = L * W
        i = rng.integers(0, N, 60)
        j = (i + rng.integers(1, N, 60)) % N
        out = []
        for knobs in (15, 15 | RECOMPUTE):
            tn.tn_autotune_set(L, W, D, prec, E, knobs)
            lat = tn.tn_create_lattice(ctx, L, W, D)
            try:
                tn.tn_set_site_tensors(lat, A)
                out.append(tn.tn_pair_correlators(lat, prec, tn.TN_OP_Z, tn.TN_OP_X, i, j).copy())
            finally:
                tn.tn_destroy_lattice(lat)
        assert np.array_equal(out[0], out[1])


def test_recompute_complex(ctx):
    L, W, D = 5, 5, 2
    A = inputs.random_complex_lattice(L, W, D, 9400)
    for prec in (tn.TN_FP64, tn.TN_BF16X6):
        _same(_energy(ctx, L, W, D, A, prec, 15, cplx=True),
              _energy(ctx, L, W, D, A, prec, 15 | RECOMPUTE, cplx=True))


def _footprint(L, W, D, prec, work=E, knobs=None):
    probe = tn.tn_ctx_create(-1)
    lat = tn.tn_create_lattice(probe, L, W, D)
    try:
        if knobs is not None:
            tn.tn_autotune_set(L, W, D, prec, E, knobs)
        return tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, work)
    finally:
        if knobs is not None:
            tn.tn_autotune_clear()
        tn.tn_destroy_lattice(lat)
        tn.tn_ctx_destroy(probe)


def test_lattice_falls_back_when_the_cache_does_not_fit(ctx):
    L, W, D, prec = 7, 7, 3, tn.TN_FP32
    A = inputs.random_lattice(L, W, D, 9500)
    f_cached = _footprint(L, W, D, prec)
    f_rec = _footprint(L, W, D, prec, knobs=15 | RECOMPUTE)
    assert f_rec < f_cached / 2
    ref = _energy(ctx, L, W, D, A, prec)
    small = tn.tn_ctx_create(0, (f_rec + f_cached) // 2)
    try:
        _same(_energy(small, L, W, D, A, prec), ref)
        # the bond work kinds take the same fallback
        lat = tn.tn_create_lattice(small, L, W, D)
        big = tn.tn_create_lattice(ctx, L, W, D)
        try:
            tn.tn_set_site_tensors(lat, A)
            tn.tn_set_site_tensors(big, A)
            xx_small = tn.tn_bond_correlators(lat, prec, tn.TN_OP_X, tn.TN_OP_X, L, W)
            xx_big = tn.tn_bond_correlators(big, prec, tn.TN_OP_X, tn.TN_OP_X, L, W)
            assert np.array_equal(xx_small, xx_big)
        finally:
            tn.tn_destroy_lattice(lat)
            tn.tn_destroy_lattice(big)
        # below the recompute form's footprint the call is refused
        tiny = tn.tn_ctx_create(0, f_rec // 2)
        try:
            lat = tn.tn_create_lattice(tiny, L, W, D)
            try:
                tn.tn_set_site_tensors(lat, A)
                with pytest.raises(tn.TNError) as e:
                    tn.tn_energy(lat, 1.0, 3.04, prec)
                assert e.value.status == tn.TN_ERR_OVER_BUDGET
            finally:
                tn.tn_destroy_lattice(lat)
        finally:
            tn.tn_ctx_destroy(tiny)
    finally:
        tn.tn_ctx_destroy(small)


def test_group_member_falls_back(ctx):
    shapes = [(4, 4, 2), (7, 7, 3), (5, 5, 2)]
    prec = tn.TN_FP32
    f_cached = _footprint(7, 7, 3, prec)
    f_rec = _footprint(7, 7, 3, prec, knobs=15 | RECOMPUTE)
    budget = (f_rec + f_cached) // 2
    Ls, Ws, Ds = zip(*shapes)
    g = tn.tn_batch_group_create(ctx, Ls, Ws, Ds, prec, budget)
    try:
        tn.tn_batch_group_fill_random(g, 9600)
        hs = np.array([1.0, 3.04, 4.0])
        tn.tn_batch_group_run(g, 1.0, hs)
        res = tn.tn_batch_group_results_host(g).copy()
    finally:
        tn.tn_batch_group_destroy(g)
    off = 0
    for k, (L, W, D) in enumerate(shapes):
        n = 6 + 2 * L * W + L * (W - 1) + W * (L - 1)
        A = inputs.random_lattice(L, W, D, inputs.lattice_seed(9600, k))
        b = tn.tn_batch_create(ctx, [L], [W], [D], prec)
        try:
            tn.tn_batch_set_tensors(b, A)
            tn.tn_batch_run(b, 1.0, np.array([hs[k]]))
            assert np.array_equal(res[off:off + n], tn.tn_batch_results_host(b)), (L, W, D)
        finally:
            tn.tn_batch_destroy(b)
        off += n


def _product_closed_form(L, W, a0, a1, h):
    nk = a0 ** 2 + a1 ** 2
    sx, sz = 2 * a0 * a1 / nk, (a1 ** 2 - a0 ** 2) / nk
    zz = np.array([sz[ri * W + ci] * sz[rj * W + cj] for (ri, ci), (rj, cj) in inputs.bonds(L, W)])
    return sx, sz, zz, -float(np.sum(zz)) - h * float(np.sum(sx))


def test_9x9_d3_recompute_equals_cached_bf16x6(ctx):
    # the largest D = 3 square whose cached form fits one GB300: both forms, same bits
    L, W, D, prec = 9, 9, 3, tn.TN_BF16X6
    A = inputs.random_lattice(L, W, D, 9900)
    cached = _energy(ctx, L, W, D, A, prec, 15)
    rec = _energy(ctx, L, W, D, A, prec, 15 | RECOMPUTE)
    _same(cached, rec)
    assert np.all(np.abs(rec[1]) <= 1 + 1e-6) and np.all(np.abs(rec[2]) <= 1 + 1e-6)


def test_10x10_d3_product_state_closed_form_bf16x6(ctx):
    # 10 x 10, D = 3: only the recompute form fits (the cached one needs ~0.7 TB);
    # a product state written with bond dimension 3 has a closed form
    L, W, D, prec, h = 10, 10, 3, tn.TN_BF16X6, 3.04
    rng = np.random.default_rng(1010)
    a0, a1 = rng.uniform(-1, 1, L * W), rng.uniform(-1, 1, L * W)
    A, hv, vv = inputs.product_lattice_bonds(L, W, D, a0, a1, 1011, with_bonds=True)
    (e, mant, exp2), sx, zz, sz, _ = _energy(ctx, L, W, D, A, prec)
    sx_ref, sz_ref, zz_ref, e_ref = _product_closed_form(L, W, a0, a1, h)
    tol = 1e-6
    np.testing.assert_allclose(sx, sx_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(sz, sz_ref, rtol=0, atol=tol)
    np.testing.assert_allclose(zz, zz_ref, rtol=0, atol=tol)
    check_energy(e, e_ref, sx_ref, zz_ref, 1.0, h, prec)
    # norm: prod_k n_k times |v_b|^4 per bond (|v_b|^2 from each layer)
    log2n = float(np.sum(np.log2(a0 ** 2 + a1 ** 2)))
    log2n += 2.0 * float(np.sum(np.log2(np.sum(hv ** 2, axis=-1))) + np.sum(np.log2(np.sum(vv ** 2, axis=-1))))
    assert abs(math.log2(abs(mant)) + exp2 - log2n) <= 1e-5 * abs(log2n)


def test_pairs_fall_back_when_the_cache_does_not_fit(ctx):
    L, W, D, prec = 7, 7, 3, tn.TN_FP32
    A = inputs.random_lattice(L, W, D, 9700)
    rng = np.random.default_rng(97)
    i = rng.integers(0, L * W, 40)
    j = (i + rng.integers(1, L * W, 40)) % (L * W)
    f_cached = _footprint(L, W, D, prec)
    f_rec = _footprint(L, W, D, prec, knobs=15 | RECOMPUTE)
    out = []
    small = tn.tn_ctx_create(0, (f_rec + f_cached) // 2)
    try:
        for c in (ctx, small):
            lat = tn.tn_create_lattice(c, L, W, D)
            try:
                tn.tn_set_site_tensors(lat, A)
                out.append(tn.tn_pair_correlators(lat, prec, tn.TN_OP_X, tn.TN_OP_Z, i, j).copy())
            finally:
                tn.tn_destroy_lattice(lat)
    finally:
        tn.tn_ctx_destroy(small)
    assert np.array_equal(out[0], out[1])


def test_served_in_the_recompute_form(ctx):
    # the server takes the table's choice: with bit 5 set for the shape, a job
    # whose cached form exceeds the budget is admitted and equals the lattice alone
    L, W, D, prec = 7, 7, 3, tn.TN_FP32
    f_cached = _footprint(L, W, D, prec)
    f_rec = _footprint(L, W, D, prec, knobs=15 | RECOMPUTE)
    srv = tn.tn_ctx_create(0, (f_rec + f_cached) // 2)
    try:
        with pytest.raises(tn.TNError) as e:
            tn.tn_submit(srv, L, W, D, prec, 1.0, 3.04, seed=9800)
        assert e.value.status == tn.TN_ERR_OVER_BUDGET
        tn.tn_autotune_set(L, W, D, prec, E, 15 | RECOMPUTE)
        t = tn.tn_submit(srv, L, W, D, prec, 1.0, 3.04, seed=9800)
        r, sx, zz = tn.tn_wait(srv, t, 300.0, L, W)
        served = (r.energy, r.norm.mant, r.norm.exp2)
    finally:
        tn.tn_ctx_destroy(srv)
    tn.tn_autotune_clear()
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_fill_random(lat, 9800)
        r2, sx2, zz2 = tn.tn_energy(lat, 1.0, 3.04, prec, tn.TN_SCHED_AUTO, L, W)
    finally:
        tn.tn_destroy_lattice(lat)
    assert served == (r2.energy, r2.norm.mant, r2.norm.exp2)
    assert np.array_equal(sx, sx2) and np.array_equal(zz, zz2)
