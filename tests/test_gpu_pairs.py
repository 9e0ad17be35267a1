"""GPU parity for arbitrary-range two-site correlators <A_i B_j> (Eq. cij for any
pair of distinct sites), A, B in {X, Y, Z}, against the FP64 oracle's full
contraction per pair and, on lattices of at most 16 sites, against the complex
state vector.  Pairs cover every combination of corners the schedule uses: one
corner, two adjacent corners and the two diagonal ones.  Tolerances as for the
other observables: |gpu - ref| <= tol * max(1, |ref|), FP64 1e-10, FP32 and
BF16x6 1e-6, BF16x3 1e-5."""
import itertools

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}
OPS = {"x": tn.TN_OP_X, "y": tn.TN_OP_Y, "z": tn.TN_OP_Z}


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _pairs(ctx, L, W, D, A, prec, a, b, i, j):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_pair_correlators(lat, prec, OPS[a], OPS[b], i, j)
    finally:
        tn.tn_destroy_lattice(lat)


def _corner_of(ctx, L, W, D):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        p = tn.tn_plan_work(lat, tn.TN_SCHED_AUTO, tn.TN_WORK_ENERGY)
    finally:
        tn.tn_destroy_lattice(lat)
    ns = int(p[4])
    steps = p[7:7 + 9 * ns].reshape(ns, 9)
    return {int(s[3]) * W + int(s[4]): int(s[0]) for s in steps}


def _sample_pairs(ctx, L, W, D, per_class, seed):
    """per_class pairs (i, j), i != j, for every unordered pair of corners in use."""
    corner = _corner_of(ctx, L, W, D)
    rng = np.random.default_rng(seed)
    classes = {}
    for i, j in itertools.permutations(range(L * W), 2):
        classes.setdefault(tuple(sorted((corner[i], corner[j]))), []).append((i, j))
    out = []
    for key in sorted(classes):
        lst = classes[key]
        for k in rng.choice(len(lst), size=min(per_class, len(lst)), replace=False):
            out.append(lst[k])
    return np.array(out, dtype=np.int32), set(classes)


@pytest.mark.parametrize("a,b", list(itertools.product("xyz", repeat=2)))
def test_all_pairs_4x4_fp64_vs_state_vector(ctx, a, b):
    L, W, D = 4, 4, 2
    A = inputs.random_lattice(L, W, D, 4402)
    ij = np.array([(i, j) for i in range(16) for j in range(16) if i != j], dtype=np.int32)
    got = _pairs(ctx, L, W, D, A, tn.TN_FP64, a, b, ij[:, 0], ij[:, 1])
    ref = np.array([brute.pair_correlator(L, W, D, A, a, int(i), b, int(j)) for i, j in ij])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    if (a == "y") != (b == "y"):
        assert np.all(got == 0.0)


@pytest.mark.parametrize("L,W,D", [(3, 4, 2), (5, 5, 2), (3, 3, 3), (4, 4, 3)])
@pytest.mark.parametrize("a,b", [("z", "z"), ("x", "z"), ("y", "y")])
def test_sampled_pairs_fp64(ctx, L, W, D, a, b):
    A = inputs.random_lattice(L, W, D, 500 + 11 * L + W + D)
    ij, classes = _sample_pairs(ctx, L, W, D, 6, L * W * D)
    assert {(0, 3), (1, 2)} <= classes          # both diagonal corner classes occur
    got = _pairs(ctx, L, W, D, A, tn.TN_FP64, a, b, ij[:, 0], ij[:, 1])
    ref = np.array([oracle.pair(L, W, D, A, a, int(i), b, int(j)) for i, j in ij])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10 * max(1.0, float(np.abs(ref).max())))


@pytest.mark.parametrize("prec", [tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6])
@pytest.mark.parametrize("a,b", [("z", "z"), ("x", "x"), ("y", "y"), ("z", "x")])
def test_sampled_pairs_8x8_reduced(ctx, prec, a, b):
    L, W, D = 8, 8, 2
    A = inputs.random_lattice(L, W, D, 8802)
    ij, _ = _sample_pairs(ctx, L, W, D, 3, 88)
    ref = np.array([oracle.pair(L, W, D, A, a, int(i), b, int(j)) for i, j in ij])
    got = _pairs(ctx, L, W, D, A, prec, a, b, ij[:, 0], ij[:, 1])
    np.testing.assert_allclose(got, ref, rtol=0, atol=TOL_OBS[prec] * max(1.0, float(np.abs(ref).max())))


def test_nearest_neighbour_pairs_equal_bond_correlators(ctx):
    L, W, D = 5, 6, 2
    A = inputs.random_lattice(L, W, D, 5602)
    bonds = [(r * W + c, r * W + c + 1) for r in range(L) for c in range(W - 1)]
    bonds += [(r * W + c, (r + 1) * W + c) for r in range(L - 1) for c in range(W)]
    ij = np.array(bonds, dtype=np.int32)
    for a, b in (("z", "z"), ("x", "z"), ("y", "y")):
        lat = tn.tn_create_lattice(ctx, L, W, D)
        try:
            tn.tn_set_site_tensors(lat, A)
            bc = tn.tn_bond_correlators(lat, tn.TN_FP64, OPS[a], OPS[b], L, W)
            pc = tn.tn_pair_correlators(lat, tn.TN_FP64, OPS[a], OPS[b], ij[:, 0], ij[:, 1])
        finally:
            tn.tn_destroy_lattice(lat)
        np.testing.assert_allclose(pc, bc, rtol=0, atol=1e-12)


def test_swapped_pair_swaps_operators(ctx):
    L, W, D = 4, 4, 3
    A = inputs.random_lattice(L, W, D, 4403)
    ij, _ = _sample_pairs(ctx, L, W, D, 4, 7)
    xz = _pairs(ctx, L, W, D, A, tn.TN_FP64, "x", "z", ij[:, 0], ij[:, 1])
    zx = _pairs(ctx, L, W, D, A, tn.TN_FP64, "z", "x", ij[:, 1], ij[:, 0])
    np.testing.assert_allclose(xz, zx, rtol=0, atol=1e-12)


def test_single_row_and_product_state(ctx):
    # one corner only (a 1 x W lattice), and the product state of all-ones
    # tensors, |+>^N: <X_i X_j> = 1, <Z_i Z_j> = <Y_i Y_j> = 0 exactly
    L, W, D = 1, 7, 2
    A = inputs.random_lattice(L, W, D, 1702)
    ij = np.array([(i, j) for i in range(W) for j in range(W) if i != j], dtype=np.int32)
    got = _pairs(ctx, L, W, D, A, tn.TN_FP64, "z", "y", ij[:, 0], ij[:, 1])
    assert np.all(got == 0.0)
    got = _pairs(ctx, L, W, D, A, tn.TN_FP64, "y", "y", ij[:, 0], ij[:, 1])
    ref = np.array([brute.pair_correlator(L, W, D, A, "y", int(i), "y", int(j)) for i, j in ij])
    np.testing.assert_allclose(got, ref, rtol=0, atol=1e-10)
    L, W = 6, 6
    ones = inputs.ones_lattice(L, W, 2)
    ij = np.array([(0, 35), (5, 30), (3, 20), (14, 15)], dtype=np.int32)
    assert np.all(_pairs(ctx, L, W, 2, ones, tn.TN_FP32, "x", "x", ij[:, 0], ij[:, 1]) == 1.0)
    assert np.all(_pairs(ctx, L, W, 2, ones, tn.TN_FP64, "z", "z", ij[:, 0], ij[:, 1]) == 0.0)
    assert np.all(_pairs(ctx, L, W, 2, ones, tn.TN_FP64, "y", "y", ij[:, 0], ij[:, 1]) == 0.0)


def test_bad_pairs_rejected(ctx):
    lat = tn.tn_create_lattice(ctx, 3, 3, 2)
    try:
        tn.tn_set_site_tensors(lat, inputs.random_lattice(3, 3, 2, 1))
        for i, j in ((2, 2), (-1, 3), (0, 9)):
            with pytest.raises(tn.TNError) as e:
                tn.tn_pair_correlators(lat, tn.TN_FP64, tn.TN_OP_Z, tn.TN_OP_Z, [i], [j])
            assert e.value.status == tn.TN_ERR_INVALID
        assert tn.tn_pair_correlators(lat, tn.TN_FP64, tn.TN_OP_Z, tn.TN_OP_Z, [], []).size == 0
    finally:
        tn.tn_destroy_lattice(lat)
