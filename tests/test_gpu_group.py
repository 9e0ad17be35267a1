"""Batch groups: lattices of uneven sizes split into passes that share one
arena and run as one CUDA graph.  Every member's result row equals the same
lattice in an ordinary batch of its own, bit for bit, whatever pass it lands
in; the energies agree with the oracle."""
import numpy as np
import pytest

import oracle
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

SHAPES = [(4, 4, 2), (5, 6, 2), (4, 4, 3), (6, 6, 2), (3, 5, 3), (7, 4, 2), (5, 5, 3), (8, 8, 2),
          (4, 7, 2), (6, 4, 3), (2, 9, 2)]


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _footprint(L, W, D, prec):
    probe = tn.tn_ctx_create(-1)
    lat = tn.tn_create_lattice(probe, L, W, D)
    try:
        return tn.tn_footprint(lat, tn.TN_SCHED_AUTO, prec, tn.TN_WORK_ENERGY)
    finally:
        tn.tn_destroy_lattice(lat)
        tn.tn_ctx_destroy(probe)


def _row_len(L, W):
    return 6 + 2 * L * W + L * (W - 1) + W * (L - 1)


@pytest.mark.parametrize("prec", [tn.TN_FP32, tn.TN_FP64, tn.TN_BF16X6])
def test_group_equals_members_alone(ctx, prec):
    Ls, Ws, Ds = zip(*SHAPES)
    # just above the largest member: three passes in every precision
    budget = int(1.05 * max(_footprint(*s, prec) for s in SHAPES))
    g = tn.tn_batch_group_create(ctx, Ls, Ws, Ds, prec, budget)
    try:
        info = tn.tn_batch_group_info(g)
        assert info["passes"] >= 3 and info["launches"] > 0
        tn.tn_batch_group_fill_random(g, 4242)
        hs = np.linspace(0.5, 5.0, len(SHAPES))
        tn.tn_batch_group_run(g, 1.0, hs)
        res = tn.tn_batch_group_results_host(g).copy()
        tn.tn_batch_group_run(g, 1.0, hs)              # replay: the same bits
        assert np.array_equal(tn.tn_batch_group_results_host(g), res)
    finally:
        tn.tn_batch_group_destroy(g)
    off = 0
    for k, (L, W, D) in enumerate(SHAPES):
        n = _row_len(L, W)
        row = res[off:off + n]
        off += n
        A = inputs.random_lattice(L, W, D, inputs.lattice_seed(4242, k))
        b = tn.tn_batch_create(ctx, [L], [W], [D], prec)
        try:
            tn.tn_batch_set_tensors(b, A)
            tn.tn_batch_run(b, 1.0, np.array([hs[k]]))
            alone = tn.tn_batch_results_host(b)
        finally:
            tn.tn_batch_destroy(b)
        assert np.array_equal(row, alone), (k, L, W, D)
        if k in (0, 2):
            ref = oracle.observables(L, W, D, A)
            check_energy(row[0], ref.energy(1.0, hs[k]), ref.sx, ref.szsz, 1.0, hs[k], prec)
    assert off == res.size


def test_group_of_one_pass_and_refusals(ctx):
    prec = tn.TN_FP32
    Ls, Ws, Ds = zip(*SHAPES[:4])
    g = tn.tn_batch_group_create(ctx, Ls, Ws, Ds, prec, 1 << 40)
    try:
        assert tn.tn_batch_group_info(g)["passes"] == 1
    finally:
        tn.tn_batch_group_destroy(g)
    with pytest.raises(tn.TNError) as e:        # a member larger than the pass budget
        tn.tn_batch_group_create(ctx, [6], [6], [3], prec, 1024)
    assert e.value.status == tn.TN_ERR_OVER_BUDGET
