"""The autotuner (tn_autotune): every program choice it times is exact, the
table's choice reaches every later contraction of the shape, and a lattice
still gives the same bits alone and inside a batch."""
import numpy as np
import pytest

import oracle
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X6: 1e-6, tn.TN_BF16X3: 1e-5}
# knob combinations that change each shape's program (bits: 1 pairs, 2 triple dot, 4 D=3 factors,
# 8 tensor-core products of >= 2^26 multiply-adds, 16 smaller ones too)
CASES = [((6, 6, 2), tn.TN_FP32, [15, 14, 13, 12]), ((4, 4, 3), tn.TN_FP32, [15, 11]),
         ((4, 4, 3), tn.TN_FP64, [15, 11]), ((8, 8, 2), tn.TN_BF16X6, [15, 31, 30, 29]),
         ((5, 5, 3), tn.TN_BF16X6, [15, 11, 7, 3]), ((5, 5, 3), tn.TN_BF16X3, [15, 11])]


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)
    tn.tn_autotune_clear()


@pytest.mark.parametrize("shape,prec,codes", CASES)
def test_every_choice_is_exact(ctx, shape, prec, codes):
    L, W, D = shape
    A = inputs.random_lattice(L, W, D, 61 + L + D)
    ref = oracle.observables(L, W, D, A)
    try:
        for code in codes:
            tn.tn_autotune_set(L, W, D, prec, tn.TN_WORK_ENERGY, code)
            lat = tn.tn_create_lattice(ctx, L, W, D)
            try:
                tn.tn_set_site_tensors(lat, A)
                r, sx, zz = tn.tn_energy(lat, 1.0, 3.04, prec, tn.TN_SCHED_AUTO, L, W)
            finally:
                tn.tn_destroy_lattice(lat)
            check_energy(r.energy, ref.energy(1.0, 3.04), ref.sx, ref.szsz, 1.0, 3.04, prec)
            assert np.max(np.abs(sx - ref.sx)) <= TOL_OBS[prec], code
            assert np.max(np.abs(zz - ref.szsz)) <= TOL_OBS[prec], code
    finally:
        tn.tn_autotune_clear()


def test_tuned_choice_is_used_alone_and_in_batches(ctx):
    shapes = [(5, 5, 2), (4, 4, 3)]
    try:
        tn.tn_autotune(ctx, [s[0] for s in shapes], [s[1] for s in shapes], [s[2] for s in shapes], tn.TN_FP32,
                       reps=3, max_bytes=1 << 28)
        for L, W, D in shapes:
            e = tn.tn_autotune_lookup(L, W, D, tn.TN_FP32)
            assert e["tuned"] and 0 < e["best_ms"] <= e["default_ms"] * 1.0000001
        Ls, Ws, Ds = zip(*shapes)
        b = tn.tn_batch_create(ctx, Ls, Ws, Ds, tn.TN_FP32)
        try:
            tn.tn_batch_fill_random(b, 99)
            tn.tn_batch_run(b, 1.0, np.array([3.04, 2.0]))
            res = tn.tn_batch_results_host(b).copy()
        finally:
            tn.tn_batch_destroy(b)
        off = 0
        for k, (L, W, D) in enumerate(shapes):
            nres = 6 + 2 * L * W + L * (W - 1) + W * (L - 1)
            b1 = tn.tn_batch_create(ctx, [L], [W], [D], tn.TN_FP32)
            try:
                tn.tn_batch_set_tensors(b1, inputs.random_lattice(L, W, D, inputs.lattice_seed(99, k)))
                tn.tn_batch_run(b1, 1.0, np.array([[3.04, 2.0][k]]))
                alone = tn.tn_batch_results_host(b1)
            finally:
                tn.tn_batch_destroy(b1)
            assert np.array_equal(res[off:off + nres], alone)
            off += nres
    finally:
        tn.tn_autotune_clear()
