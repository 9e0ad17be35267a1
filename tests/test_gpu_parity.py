"""GPU parity: libtn's CUDA path against the FP64 CPU oracle, element by element.

Tolerances (written per test):
  energy E (energy_tol.check_energy): FP64 |dE| <= 1e-10 |E|; FP32, BF16x3 and
  BF16x6 |dE| <= 1e-6 S with S = |J| sum |<ZZ>| + |h| sum |<X>| (and <= 1e-6 |E|
  wherever S <= 10 |E|);
  every <X_k> and <Z_i Z_j>, as |gpu - ref| <= tol * max(1, |ref|) (O(1)
  quantities that can be ~0): FP64 1e-10; FP32 and BF16x6 1e-6; BF16x3 1e-5
  (three split products keep about 16 mantissa bits; with D = 3 the absorption
  itself runs on them).
Exact cases (all-ones, D = 2) are compared with ==.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

TOL = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-6, tn.TN_BF16X6: 1e-6}      # E (energy_tol)
TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X3: 1e-5, tn.TN_BF16X6: 1e-6}  # <X>, <ZZ>
PRECS = [tn.TN_FP64, tn.TN_FP32]
SCHEDS = [tn.TN_SCHED_AUTO, tn.TN_SCHED_ROW, tn.TN_SCHED_COL, tn.TN_SCHED_QUADRANT]


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _energy(ctx, L, W, D, A, prec, sched, J=1.0, h=3.04):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        r, sx, zz = tn.tn_energy(lat, J, h, prec, sched, L, W)
        return r, sx, zz
    finally:
        tn.tn_destroy_lattice(lat)


def _check(r, sx, zz, ref, prec, J=1.0, h=3.04):
    tol, tol_obs = TOL[prec], TOL_OBS[prec]
    check_energy(r.energy, ref.energy(J, h), ref.sx, ref.szsz, J, h, prec)
    assert abs(r.energy_per_site * sx.size - r.energy) <= 1e-15 * abs(r.energy) * sx.size
    np.testing.assert_allclose(sx, ref.sx, rtol=0, atol=tol_obs * max(1.0, np.abs(ref.sx).max()))
    if zz.size:
        np.testing.assert_allclose(zz, ref.szsz, rtol=0, atol=tol_obs * max(1.0, np.abs(ref.szsz).max()))
    lg = math.log2(abs(r.norm.mant)) + r.norm.exp2
    assert abs(lg - ref.log2_norm) <= max(tol, 1e-12) * 64 * max(1.0, abs(ref.log2_norm))


# ------------------------------------------------------------------ C1

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("sched", SCHEDS)
def test_c1_4x4_d2_vs_oracle_and_brute_force(ctx, prec, sched):
    L, W, D = 4, 4, 2
    A = inputs.random_lattice(L, W, D, 2024)
    ref = oracle.observables(L, W, D, A)
    r, sx, zz = _energy(ctx, L, W, D, A, prec, sched)
    _check(r, sx, zz, ref, prec)
    n, bsx, bzz = brute.observables(L, W, D, A)
    tol = TOL[prec]
    np.testing.assert_allclose(sx, bsx, atol=tol)
    np.testing.assert_allclose(zz, bzz, atol=tol)


SHAPES = [(1, 1, 2), (1, 4, 2), (4, 1, 2), (2, 2, 1), (2, 3, 2), (3, 3, 2), (3, 2, 3), (3, 5, 2),
          (5, 3, 2), (4, 4, 3), (5, 5, 2), (2, 6, 2), (6, 2, 3), (3, 4, 4)]


@pytest.mark.parametrize("L,W,D", SHAPES)
def test_shapes_fp64_every_schedule(ctx, L, W, D):
    A = inputs.random_lattice(L, W, D, 100 + 7 * L + W + 31 * D)
    ref = oracle.observables(L, W, D, A)
    for sched in SCHEDS:
        r, sx, zz = _energy(ctx, L, W, D, A, tn.TN_FP64, sched)
        _check(r, sx, zz, ref, tn.TN_FP64)


@pytest.mark.parametrize("L,W,D", [(3, 4, 2), (4, 4, 3), (5, 6, 2)])
def test_shapes_fp32(ctx, L, W, D):
    A = inputs.random_lattice(L, W, D, 9 + L + W + D)
    ref = oracle.observables(L, W, D, A)
    for sched in (tn.TN_SCHED_AUTO, tn.TN_SCHED_ROW):
        r, sx, zz = _energy(ctx, L, W, D, A, tn.TN_FP32, sched)
        _check(r, sx, zz, ref, tn.TN_FP32)


# ------------------------------------------------------- exact workloads

@pytest.mark.parametrize("prec", PRECS)
@pytest.mark.parametrize("L,W", [(4, 4), (6, 6), (8, 8), (5, 7)])
def test_all_ones_exact(ctx, prec, L, W):
    """Sec. 6 workload: norm = 2^N 2^(2 nb), <X> = 1, <ZZ> = 0 exactly (D = 2)."""
    D = 2
    A = inputs.ones_lattice(L, W, D)
    r, sx, zz = _energy(ctx, L, W, D, A, prec, tn.TN_SCHED_AUTO)
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    assert r.norm.mant == 0.5 and r.norm.exp2 == N + 2 * nb + 1
    assert np.all(sx == 1.0) and np.all(zz == 0.0)
    assert r.energy == -3.04 * N


@pytest.mark.parametrize("L,W,K", [(3, 3, 0.3), (4, 4, 0.5), (4, 5, 0.9)])
def test_ising_peps_vs_enumeration(ctx, L, W, K):
    A = inputs.ising_peps_lattice(L, W, K)
    logz, corr, xf = oracle.ising_enumerate(L, W, K)
    r, sx, zz = _energy(ctx, L, W, 2, A, tn.TN_FP64, tn.TN_SCHED_AUTO)
    lg = (math.log2(abs(r.norm.mant)) + r.norm.exp2) * math.log(2)
    assert abs(lg - logz) < 1e-10 * max(1, logz)
    np.testing.assert_allclose(zz, corr, atol=1e-10)
    np.testing.assert_allclose(sx, xf, atol=1e-10)


# ------------------------------------------------------------------ C2

@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32])
def test_c2_8x8_d2_three_fields(ctx, prec):
    L, W, D = 8, 8, 2
    A = inputs.random_lattice(L, W, D, 88)
    ref = oracle.observables(L, W, D, A)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        for h in (2.0, 3.04, 4.0):
            r, sx, zz = tn.tn_energy(lat, 1.0, h, prec, tn.TN_SCHED_AUTO, L, W)
            _check(r, sx, zz, ref, prec, 1.0, h)
    finally:
        tn.tn_destroy_lattice(lat)


def test_norm_and_expectation_entry_points(ctx):
    L, W, D = 4, 5, 2
    A = inputs.random_lattice(L, W, D, 5)
    ref = oracle.observables(L, W, D, A)
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        m, e = tn.tn_contract_norm(lat, tn.TN_FP64)
        assert abs(math.log2(abs(m)) + e - ref.log2_norm) < 1e-11 * abs(ref.log2_norm)
        for k in (0, 7, 19):
            v = tn.tn_expectation(lat, tn.TN_FP64, tn.TN_OP_X, k)
            assert abs(v - ref.sx[k]) < 1e-10
        for bi, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W)):
            if bi % 6:
                continue
            v = tn.tn_expectation(lat, tn.TN_FP64, tn.TN_OP_ZZ, ri * W + ci, rj * W + cj)
            assert abs(v - ref.szsz[bi]) < 1e-10
    finally:
        tn.tn_destroy_lattice(lat)


# ------------------------------------------------------------- batches

def test_batch_member_equals_alone_bitwise(ctx):
    """Each lattice gives the same bits alone and inside a mixed batch."""
    shapes = [(4, 4, 2), (3, 5, 2), (4, 4, 3), (5, 5, 2), (4, 4, 2)]
    Ls, Ws, Ds = zip(*shapes)
    hs = np.array([2.0, 3.04, 4.0, 0.7, 1.5])
    b = tn.tn_batch_create(ctx, Ls, Ws, Ds, tn.TN_FP32)
    try:
        tn.tn_batch_fill_random(b, 777)
        tn.tn_batch_run(b, 1.0, hs)
        res = tn.tn_batch_results_host(b)
    finally:
        tn.tn_batch_destroy(b)
    off = 0
    for k, (L, W, D) in enumerate(shapes):
        nb = L * (W - 1) + W * (L - 1)
        seg = res[off:off + 6 + 2 * L * W + nb]
        off += seg.size
        A = inputs.random_lattice(L, W, D, inputs.lattice_seed(777, k))
        b1 = tn.tn_batch_create(ctx, [L], [W], [D], tn.TN_FP32)
        try:
            tn.tn_batch_set_tensors(b1, A)
            tn.tn_batch_run(b1, 1.0, hs[k:k + 1])
            alone = tn.tn_batch_results_host(b1)
        finally:
            tn.tn_batch_destroy(b1)
        assert np.array_equal(seg, alone), k
        ref = oracle.observables(L, W, D, A)
        check_energy(seg[0], ref.energy(1.0, hs[k]), ref.sx, ref.szsz, 1.0, hs[k], tn.TN_FP32)


def test_graph_replay_is_deterministic(ctx):
    b = tn.tn_batch_create(ctx, [6, 6], [6, 5], [2, 2], tn.TN_FP32)
    try:
        tn.tn_batch_fill_random(b, 3)
        out = []
        for _ in range(3):
            tn.tn_batch_run(b, 1.0, np.array([3.04, 3.04]))
            out.append(tn.tn_batch_results_host(b).copy())
        assert np.array_equal(out[0], out[1]) and np.array_equal(out[1], out[2])
    finally:
        tn.tn_batch_destroy(b)


# ---------------------------------------------------- plain absorption

@pytest.mark.parametrize("K,N,P,S", [(16, 16, 7, 1000), (4, 16, 1, 4096), (16, 4, 33, 1),
                                     (81, 81, 3, 300), (9, 81, 5, 81), (1, 16, 1000, 1)])
@pytest.mark.parametrize("dtype", [0, 1])
def test_tn_absorb_matches_reference(K, N, P, S, dtype):
    import torch
    tdt = torch.float64 if dtype == 0 else torch.float32
    g = torch.Generator().manual_seed(K * N + P + S)
    x = torch.rand(P, K, S, generator=g, dtype=torch.float64) * 2 - 1
    E = torch.rand(K, N, generator=g, dtype=torch.float64) * 2 - 1
    ref = torch.einsum("pks,kn->pns", x, E)
    xd, Ed = x.to(tdt).cuda(), E.to(tdt).cuda()
    out = torch.empty(P, N, S, dtype=tdt, device="cuda")
    tn.tn_absorb(dtype, xd, Ed, out, P, K, N, S, torch.cuda.current_stream())
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == 0 else 2e-6 * K
    assert torch.allclose(out.double().cpu(), ref, atol=tol, rtol=0)


@pytest.mark.parametrize("K,N,P,S", [(16, 16, 7, 1000), (4, 16, 1, 4096), (16, 4, 33, 1),
                                     (81, 81, 3, 300), (9, 81, 5, 81), (1, 1, 5000, 3)])
@pytest.mark.parametrize("dtype", [0, 1])
def test_tn_absorb_dot_matches_reference(K, N, P, S, dtype):
    import torch
    tdt = torch.float64 if dtype == 0 else torch.float32
    g = torch.Generator().manual_seed(3 * K + N + P + S)
    x = torch.rand(P, K, S, generator=g, dtype=torch.float64) * 2 - 1
    E = torch.rand(K, N, generator=g, dtype=torch.float64) * 2 - 1
    adj = torch.rand(P, N, S, generator=g, dtype=torch.float64) * 2 - 1
    ref = float(torch.einsum("pks,kn,pns->", x, E, adj))
    scale = float(torch.einsum("pks,kn,pns->", x.abs(), E.abs(), adj.abs()))
    xd, Ed, ad = x.to(tdt).cuda(), E.to(tdt).cuda(), adj.to(tdt).cuda()
    res = torch.zeros(2, dtype=torch.float64, device="cuda")
    st = torch.cuda.current_stream()
    tn.tn_absorb_dot(dtype, xd, Ed, ad, P, K, N, S, res[0:1], st)
    tn.tn_absorb_dot(dtype, xd, Ed, ad, P, K, N, S, res[1:2], st)
    torch.cuda.synchronize()
    tol = 1e-13 if dtype == 0 else 1e-6
    got = res.cpu().numpy()
    assert abs(got[0] - ref) <= tol * scale
    assert got[0] == got[1]          # deterministic finish of the tile partials


# ------------------------------------------------ tensor-core ring products

@pytest.mark.parametrize("prec", [tn.TN_BF16X3, tn.TN_BF16X6])
def test_c2_8x8_d2_tensor_core_precisions(ctx, prec):
    """256-wide ring products on tcgen05 (split BF16, FP32 accumulation).  By
    default products this small run on FP32 SIMT (the same bits as FP32);
    program choice 31 puts them on the tensor cores."""
    L, W, D = 8, 8, 2
    A = inputs.random_lattice(L, W, D, 88)
    ref = oracle.observables(L, W, D, A)
    r32, _, _ = _energy(ctx, L, W, D, A, tn.TN_FP32, tn.TN_SCHED_AUTO)
    r16, _, _ = _energy(ctx, L, W, D, A, prec, tn.TN_SCHED_AUTO)
    assert r32.energy == r16.energy
    tn.tn_autotune_set(L, W, D, prec, tn.TN_WORK_ENERGY, 31)
    try:
        lat = tn.tn_create_lattice(ctx, L, W, D)
        try:
            tn.tn_set_site_tensors(lat, A)
            for h in (2.0, 3.04, 4.0):
                r, sx, zz = tn.tn_energy(lat, 1.0, h, prec, tn.TN_SCHED_AUTO, L, W)
                _check(r, sx, zz, ref, prec, 1.0, h)
            # the tensor-core result is not the FP32 SIMT result bit for bit
            rt, _, _ = tn.tn_energy(lat, 1.0, 3.04, prec, tn.TN_SCHED_AUTO, L, W)
            assert r32.energy != rt.energy
        finally:
            tn.tn_destroy_lattice(lat)
    finally:
        tn.tn_autotune_clear()


def test_tensor_core_d3_5x5(ctx):
    """D = 3: 729 x 729 ring products (odd extents, padded tiles) on tcgen05."""
    L, W, D = 5, 5, 3
    A = inputs.random_lattice(L, W, D, 5353)
    ref = oracle.observables(L, W, D, A)
    for prec in (tn.TN_BF16X3, tn.TN_BF16X6, tn.TN_FP32):
        r, sx, zz = _energy(ctx, L, W, D, A, prec, tn.TN_SCHED_AUTO)
        _check(r, sx, zz, ref, prec)


def test_tensor_core_all_ones_exact(ctx):
    """All-ones D = 2: every split plane beyond the first is zero, products exact."""
    L, W = 8, 8
    A = inputs.ones_lattice(L, W, 2)
    for prec in (tn.TN_BF16X3, tn.TN_BF16X6):
        r, sx, zz = _energy(ctx, L, W, 2, A, prec, tn.TN_SCHED_AUTO)
        N, nb = L * W, L * (W - 1) + W * (L - 1)
        assert r.norm.mant == 0.5 and r.norm.exp2 == N + 2 * nb + 1
        assert np.all(sx == 1.0) and np.all(zz == 0.0)
