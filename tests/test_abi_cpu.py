"""Host-only checks of the C-ABI library (no kernel is launched here).

* libtn loads and exports every function include/tn.h declares;
* the planner inside libtn reproduces the oracle's independent planner
  bit-exactly (partition, orientation, per-step P, K, N, S, bottleneck, MACs);
* tn_fill_random reproduces the published SplitMix64 definition in inputs.py;
* argument validation and planning-only contexts behave as documented.
"""
import os
import re

import numpy as np
import pytest

import oracle.planner as planner
from paper_1908_08553_gb300 import inputs, tn

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include", "tn.h")


def _declared():
    txt = open(HDR).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    names = set(re.findall(r"\b(tn_[a-z0-9_]+)\s*\(", txt))
    return {n for n in names if not n.endswith("_t")}


def test_header_symbols_exported():
    lib = tn.lib()
    names = _declared()
    assert len(names) >= 30
    missing = [n for n in sorted(names) if not hasattr(lib, n)]
    assert not missing, missing
    # the binding covers the same surface
    assert names == set(tn.SIGNATURES), sorted(names ^ set(tn.SIGNATURES))


@pytest.fixture(scope="module")
def cpu_ctx():
    ctx = tn.tn_ctx_create(-1)
    yield ctx
    tn.tn_ctx_destroy(ctx)


SHAPES = [(1, 1, 2), (1, 5, 2), (5, 1, 3), (2, 2, 1), (3, 3, 2), (4, 4, 2), (4, 10, 2), (10, 4, 3),
          (5, 7, 3), (7, 5, 2), (8, 8, 2), (8, 8, 3), (9, 10, 3), (10, 10, 3), (12, 12, 2), (6, 6, 4),
          (12, 11, 2), (16, 16, 2)]


@pytest.mark.parametrize("L,W,D", SHAPES)
def test_planner_bit_exact_vs_oracle(cpu_ctx, L, W, D):
    lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
    try:
        for sched in (tn.TN_SCHED_AUTO, tn.TN_SCHED_ROW, tn.TN_SCHED_COL, tn.TN_SCHED_QUADRANT):
            hdr, steps = tn.plan_steps(tn.tn_plan(lat, sched))
            p = planner.plan(L, W, D, sched)
            assert (hdr["o"], hdr["i"], hdr["j"]) == (p["o"], p["i"], p["j"])
            assert hdr["peak"] == p["peak"] and hdr["mac"] == p["mac"]
            ref = np.array([[s["corner"], s["k"], s["c"], s["r"], s["col"], s["P"], s["K"], s["N"], s["S"]]
                            for s in p["steps"]], dtype=np.int64).reshape(-1, 9)
            assert np.array_equal(steps, ref)
            # every site is absorbed exactly once
            sites = sorted((int(r), int(c)) for r, c in steps[:, 3:5])
            assert sites == [(r, c) for r in range(L) for c in range(W)]
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,D", SHAPES + [(8, 9, 3), (8, 10, 3), (9, 8, 3), (7, 12, 3)])
def test_energy_planner_bit_exact_vs_oracle(cpu_ctx, L, W, D):
    lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
    try:
        hdr, steps = tn.plan_steps(tn.tn_plan_work(lat, tn.TN_SCHED_AUTO, tn.TN_WORK_ENERGY))
        p = planner.plan(L, W, D, planner.AUTO, energy=True)
        assert (hdr["o"], hdr["i"], hdr["j"], hdr["peak"], hdr["mac"]) == (p["o"], p["i"], p["j"], p["peak"], p["mac"])
        ref = np.array([[s["corner"], s["k"], s["c"], s["r"], s["col"], s["P"], s["K"], s["N"], s["S"]]
                        for s in p["steps"]], dtype=np.int64).reshape(-1, 9)
        assert np.array_equal(steps, ref)
        # the same bottleneck as the norm's plan
        assert hdr["peak"] == planner.plan(L, W, D)["peak"]
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (8, 8, 2), (3, 5, 3)])
@pytest.mark.parametrize("seed", [0, 1, 12345, 2 ** 63 + 7])
def test_fill_random_matches_generator(cpu_ctx, L, W, D, seed):
    lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
    try:
        tn.tn_fill_random(lat, seed)
        got = tn.tn_get_site_tensors(lat, tn.tn_lattice_elems(L, W, D))
        assert np.array_equal(got, inputs.random_lattice(L, W, D, seed))
        assert got.min() >= -1.0 and got.max() < 1.0
    finally:
        tn.tn_destroy_lattice(lat)


def test_lattice_elems_matches_layout():
    for L, W, D in SHAPES:
        assert tn.tn_lattice_elems(L, W, D) == inputs.n_elems(L, W, D)
    assert tn.tn_lattice_elems(4, 4, 2) == 288
    assert tn.tn_lattice_elems(12, 12, 2) == 3872
    assert tn.tn_lattice_elems(8, 8, 3) == 7200
    assert tn.tn_lattice_elems(0, 4, 2) == 0


def test_invalid_arguments(cpu_ctx):
    with pytest.raises(tn.TNError) as e:
        tn.tn_create_lattice(cpu_ctx, 0, 4, 2)
    assert e.value.status == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError):
        tn.tn_create_lattice(cpu_ctx, 4, 4, 5)
    lat = tn.tn_create_lattice(cpu_ctx, 3, 3, 2)
    try:
        with pytest.raises(tn.TNError) as e:
            tn.tn_set_site_tensors(lat, np.zeros(7))
        assert e.value.status == tn.TN_ERR_INVALID
        # planning works without a device, contraction does not
        assert tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY) > 0
        with pytest.raises(tn.TNError) as e:
            tn.tn_contract_norm(lat, tn.TN_FP64)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
        # observables: arguments are checked before any device work
        with pytest.raises(tn.TNError) as e:
            tn.tn_expectation(lat, tn.TN_FP64, tn.TN_OP_Z, 9)
        assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_expectation(lat, tn.TN_FP64, tn.TN_OP_Z, 4)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
        for a, b in ((tn.TN_OP_ZZ, tn.TN_OP_X), (tn.TN_OP_X, tn.TN_OP_NORM), (7, tn.TN_OP_Z)):
            with pytest.raises(tn.TNError) as e:
                tn.tn_bond_correlators(lat, tn.TN_FP64, a, b, 3, 3)
            assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_bond_correlators(lat, tn.TN_FP64, tn.TN_OP_X, tn.TN_OP_Z, 3, 3)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
        # arbitrary pairs: sites and operators are checked before any device work
        for a, b, i, j in ((tn.TN_OP_Z, tn.TN_OP_Z, 2, 2), (tn.TN_OP_Z, tn.TN_OP_Z, -1, 3),
                           (tn.TN_OP_Z, tn.TN_OP_Z, 0, 9), (tn.TN_OP_ZZ, tn.TN_OP_Z, 0, 1),
                           (tn.TN_OP_Y, 5, 0, 1)):
            with pytest.raises(tn.TNError) as e:
                tn.tn_pair_correlators(lat, tn.TN_FP64, a, b, [i], [j])
            assert e.value.status == tn.TN_ERR_INVALID
        for a, b in ((tn.TN_OP_Y, tn.TN_OP_Y), (tn.TN_OP_X, tn.TN_OP_Y)):
            with pytest.raises(tn.TNError) as e:
                tn.tn_pair_correlators(lat, tn.TN_FP64, a, b, [0, 8], [8, 4])
            assert e.value.status == tn.TN_ERR_NO_DEVICE
            with pytest.raises(tn.TNError) as e:
                tn.tn_bond_correlators(lat, tn.TN_FP64, a, b, 3, 3)
            assert e.value.status == tn.TN_ERR_NO_DEVICE
    finally:
        tn.tn_destroy_lattice(lat)
    with pytest.raises(tn.TNError) as e:
        tn.tn_wait_selfcheck(cpu_ctx, 0.0)
    assert e.value.status == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError) as e:
        tn.tn_wait_selfcheck(cpu_ctx, 20.0)
    assert e.value.status == tn.TN_ERR_NO_DEVICE
    with pytest.raises(tn.TNError) as e:
        tn.tn_absorb(1, 0, 0, 0, 1, 16, 16, 1)
    assert e.value.status == tn.TN_ERR_INVALID
    assert tn.lib().tn_status_string(tn.TN_ERR_OVER_BUDGET).decode().startswith("footprint")


def test_footprint_monotone_in_precision(cpu_ctx):
    lat = tn.tn_create_lattice(cpu_ctx, 8, 8, 2)
    try:
        f64 = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP64, tn.TN_WORK_ENERGY)
        f32 = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY)
        nrm = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_NORM)
        row = tn.tn_footprint(lat, tn.TN_SCHED_ROW, tn.TN_FP32, tn.TN_WORK_NORM)
        assert f64 > f32 > nrm > 0
        assert row > nrm          # the row scheme's bottleneck is d times the quadrant's
        # the footprint holds at least the bottleneck tensor in and out (Sec. 4)
        p = planner.plan(8, 8, 2)
        assert nrm >= 2 * p["peak"] * 4
    finally:
        tn.tn_destroy_lattice(lat)


def test_submit_needs_a_device(cpu_ctx):
    with pytest.raises(tn.TNError) as e:
        tn.tn_submit(cpu_ctx, 4, 4, 2, tn.TN_FP32, 1.0, 3.04, seed=1)
    assert e.value.status == tn.TN_ERR_NO_DEVICE


@pytest.mark.parametrize("entry", ["tn_absorb", "tn_absorb_dot", "tn_absorb_dot_noalloc"])
@pytest.mark.parametrize("P,S", [(2 ** 62, 2 ** 62), (2 ** 40, 2 ** 40), (2 ** 33, 2 ** 31), (1, 2 ** 63 - 1)])
def test_kernel_entries_reject_overflowing_sizes(entry, P, S):
    """Sizes whose product P * S (or P * 16 * S) would overflow int64 are rejected
    before any product is formed or any device call is made (the dummy pointers
    are never dereferenced)."""
    fake = 0x1000
    lib = tn.lib()
    if entry == "tn_absorb":
        st = lib.tn_absorb(1, tn.c_void_p(fake), tn.c_void_p(fake), tn.c_void_p(fake), P, 16, 16, S, None)
    else:
        st = getattr(lib, entry)(1, tn.c_void_p(fake), tn.c_void_p(fake), tn.c_void_p(fake), P, 16, 16, S,
                                 tn.c_void_p(fake), None)
    assert st == tn.TN_ERR_INVALID


def test_noalloc_rejects_beyond_its_fixed_scratch():
    fake = 0x1000
    lib = tn.lib()
    # 16,777,217 outer positions: one more than the 65,536 tiles of 256 positions
    st = lib.tn_absorb_dot_noalloc(1, tn.c_void_p(fake), tn.c_void_p(fake), tn.c_void_p(fake), 16777217, 16, 16, 1,
                                   tn.c_void_p(fake), None)
    assert st == tn.TN_ERR_INVALID
    assert "16777216" in lib.tn_last_error().decode()


def test_inject_wait_timeout_arguments(cpu_ctx):
    tn.tn_ctx_inject_wait_timeout(cpu_ctx, 0)
    with pytest.raises(tn.TNError) as e:
        tn.tn_ctx_inject_wait_timeout(cpu_ctx, -1)
    assert e.value.status == tn.TN_ERR_INVALID


def test_ite_arguments_and_initial_state(cpu_ctx):
    """tn_ite_init_product writes the uniform superposition of Sec. 5 (host
    only); tn_ite_run checks its parameters before any device work."""
    import oracle.ite as ite
    L, W, D = 3, 4, 2
    lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
    try:
        tn.tn_ite_init_product(lat)
        got = tn.tn_get_site_tensors(lat, tn.tn_lattice_elems(L, W, D))
        assert np.array_equal(got, ite.pad(ite.product_plus(L, W), L, W, D))
        with pytest.raises(tn.TNError) as e:
            tn.tn_ite_run(lat, L, W, 1.0, 1.0, 0.01, 2, D, 0.01)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
    finally:
        tn.tn_destroy_lattice(lat)


def test_bmps_arguments(cpu_ctx):
    lat = tn.tn_create_lattice(cpu_ctx, 4, 4, 2)
    try:
        with pytest.raises(tn.TNError) as e:
            tn.tn_bmps_norm(lat, 129)            # max(chi, 4) * 4 > 512
        assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_bmps_norm(lat, 8)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
        for prec in (tn.TN_FP32, tn.TN_FP64):
            with pytest.raises(tn.TNError) as e:
                tn.tn_bmps_norm(lat, 8, prec)
            assert e.value.status == tn.TN_ERR_NO_DEVICE
        for prec in (tn.TN_BF16X3, tn.TN_BF16X6, 7):
            with pytest.raises(tn.TNError) as e:
                tn.tn_bmps_norm(lat, 8, prec)
            assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_bmps_expectation(lat, 8, tn.TN_OP_ZZ, 0)
        assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_bmps_expectation(lat, 8, tn.TN_OP_Z, 3, tn.TN_OP_Z, 3)
        assert e.value.status == tn.TN_ERR_INVALID
    finally:
        tn.tn_destroy_lattice(lat)


def test_autotune_table_on_the_host(cpu_ctx, tmp_path):
    """The tuning table: set / lookup / save / load / clear, and a shape's knobs
    reach its program (no fused pairs when bit 0 is off)."""
    tn.tn_autotune_clear()
    try:
        assert tn.tn_autotune_lookup(8, 8, 2, tn.TN_FP32) == {"knobs": 15, "best_ms": 0.0, "default_ms": 0.0,
                                                             "tuned": False}
        lat = tn.tn_create_lattice(cpu_ctx, 8, 8, 2)
        try:
            assert tn.tn_program_info(lat, tn.TN_FP32)["fused_pairs"] > 0
            tn.tn_autotune_set(8, 8, 2, tn.TN_FP32, tn.TN_WORK_ENERGY, 14)
            assert tn.tn_program_info(lat, tn.TN_FP32)["fused_pairs"] == 0
        finally:
            tn.tn_destroy_lattice(lat)
        path = str(tmp_path / "tune.txt")
        tn.tn_autotune_save(path)
        tn.tn_autotune_clear()
        assert not tn.tn_autotune_lookup(8, 8, 2, tn.TN_FP32)["tuned"]
        tn.tn_autotune_load(path)
        assert tn.tn_autotune_lookup(8, 8, 2, tn.TN_FP32) ["knobs"] == 14
        with pytest.raises(tn.TNError):
            tn.tn_autotune_set(8, 8, 2, tn.TN_FP32, tn.TN_WORK_ENERGY, 64)
        with pytest.raises(tn.TNError) as e:
            tn.tn_autotune(cpu_ctx, [4], [4], [2], tn.TN_FP32)
        assert e.value.status == tn.TN_ERR_NO_DEVICE
        # D = 3 without the factored form builds the 81 x 81 site matrices again
        lat = tn.tn_create_lattice(cpu_ctx, 4, 4, 3)
        try:
            f = tn.tn_program_info(lat, tn.TN_FP64)["arena_bytes"]
            tn.tn_autotune_set(4, 4, 3, tn.TN_FP64, tn.TN_WORK_ENERGY, 15 & ~4)
            assert tn.tn_program_info(lat, tn.TN_FP64)["arena_bytes"] > f
        finally:
            tn.tn_destroy_lattice(lat)
    finally:
        tn.tn_autotune_clear()


def test_complex_lattice_on_the_host(cpu_ctx):
    L, W, D = 3, 4, 2
    lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
    try:
        n = tn.tn_lattice_elems(L, W, D)
        A = inputs.random_complex_lattice(L, W, D, 3)
        with pytest.raises(tn.TNError) as e:
            tn.tn_set_site_tensors_complex(lat, A[:-1])
        assert e.value.status == tn.TN_ERR_INVALID
        fp_real = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY)
        info_real = tn.tn_program_info(lat, tn.TN_FP32)
        tn.tn_set_site_tensors_complex(lat, A)
        assert tn.tn_lattice_is_complex(lat)
        # the complex energy program is sound (host check) and holds the <Y_k> terms too
        info = tn.tn_program_info(lat, tn.TN_FP32)
        assert info["ops"] > info_real["ops"]
        assert tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY) > fp_real
        with pytest.raises(tn.TNError) as e:       # real read-back refused
            tn.tn_get_site_tensors(lat, n)
        assert e.value.status == tn.TN_ERR_INVALID
        with pytest.raises(tn.TNError) as e:
            tn.tn_bmps_norm(lat, 4)
        assert e.value.status == tn.TN_ERR_INVALID
        for op in (tn.TN_OP_X, tn.TN_OP_Y, tn.TN_OP_Z):
            with pytest.raises(tn.TNError) as e:
                tn.tn_site_expectations(lat, tn.TN_FP64, op, L, W)
            assert e.value.status == tn.TN_ERR_NO_DEVICE
        with pytest.raises(tn.TNError) as e:
            tn.tn_site_expectations(lat, tn.TN_FP64, tn.TN_OP_ZZ, L, W)
        assert e.value.status == tn.TN_ERR_INVALID
        tn.tn_fill_random(lat, 5)                  # back to real
        assert not tn.tn_lattice_is_complex(lat)
        assert tn.tn_get_site_tensors(lat, n).size == n
    finally:
        tn.tn_destroy_lattice(lat)


def test_batch_group_arguments(cpu_ctx):
    with pytest.raises(tn.TNError) as e:
        tn.tn_batch_group_create(cpu_ctx, [4], [4], [2], tn.TN_FP32, 1 << 30)
    assert e.value.status == tn.TN_ERR_NO_DEVICE
    with pytest.raises(tn.TNError) as e:
        tn.tn_batch_group_create(cpu_ctx, [4], [4], [2], tn.TN_FP32, 0)
    assert e.value.status == tn.TN_ERR_INVALID
    with pytest.raises(tn.TNError) as e:
        tn.tn_batch_group_create(cpu_ctx, [], [], [], tn.TN_FP32, 1 << 30)
    assert e.value.status == tn.TN_ERR_INVALID


def test_recompute_form_footprints(cpu_ctx):
    """Program choice bit 32 (the recompute form of the energy program): its
    programs pass the builder's consistency check (ordering, lifetimes, no two
    live tensors sharing bytes), need less memory than the cached form, and
    bring the D = 3 lattices of up to 10 x 10 under one GB300's memory."""
    tn.tn_autotune_clear()
    try:
        E = tn.TN_WORK_ENERGY
        cases = [(6, 6, 2, tn.TN_FP32), (8, 8, 2, tn.TN_FP64), (6, 6, 3, tn.TN_BF16X6), (7, 7, 3, tn.TN_FP32),
                 (5, 7, 3, tn.TN_FP32), (12, 12, 2, tn.TN_BF16X3)]
        for (L, W, D, prec) in cases:
            lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
            try:
                cached = tn.tn_program_info(lat, prec, tn.TN_SCHED_AUTO, E)
                tn.tn_autotune_set(L, W, D, prec, E, 15 | 32)
                rec = tn.tn_program_info(lat, prec, tn.TN_SCHED_AUTO, E)     # verified by the builder
                tn.tn_autotune_set(L, W, D, prec, E, 15)
                assert rec["footprint_bytes"] < cached["footprint_bytes"], (L, W, D, prec)
                assert rec["product_macs"] == cached["product_macs"]
                assert rec["ops"] > cached["ops"]                   # the recomputed chain steps
            finally:
                tn.tn_destroy_lattice(lat)
        # cached form vs recompute form, FP32 (GB): the ring products stay, the caches go
        for (L, W, D, lim) in [(9, 9, 3, 80e9), (9, 10, 3, 130e9), (10, 10, 3, 160e9), (9, 11, 3, 64e9),
                               (8, 12, 3, 8e9)]:
            lat = tn.tn_create_lattice(cpu_ctx, L, W, D)
            try:
                cached = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, E)
                tn.tn_autotune_set(L, W, D, tn.TN_FP32, E, 15 | 32)
                rec = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, E)
                assert cached > 200e9 and rec < lim, (L, W, D, cached, rec)
            finally:
                tn.tn_destroy_lattice(lat)
    finally:
        tn.tn_autotune_clear()
