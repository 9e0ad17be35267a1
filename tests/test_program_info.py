"""Host-only checks of the contraction programs the library builds (no
device): every pairwise contraction runs after the contractions that produce
its inputs and within their lifetimes, no two tensors alive at the same time
share arena memory, and the program's algorithmic work matches the fused and
unfused forms it is built from."""
import pytest

from paper_1908_08553_gb300 import tn


@pytest.fixture(scope="module")
def cpu_ctx():
    c = tn.tn_ctx_create(-1, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _info(ctx, L, W, D, prec, work, sched=tn.TN_SCHED_AUTO):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        return tn.tn_program_info(lat, prec, sched, work)
    finally:
        tn.tn_destroy_lattice(lat)


SHAPES = [(1, 1, 2), (1, 5, 2), (2, 2, 1), (3, 3, 2), (4, 4, 2), (3, 5, 3), (5, 4, 2), (6, 6, 2), (8, 8, 2),
          (4, 4, 3), (7, 5, 2), (10, 10, 2)]


@pytest.mark.parametrize("L,W,D", SHAPES)
@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X3, tn.TN_BF16X6])
@pytest.mark.parametrize("work", [tn.TN_WORK_NORM, tn.TN_WORK_ENERGY])
def test_programs_are_consistent(cpu_ctx, L, W, D, prec, work):
    info = _info(cpu_ctx, L, W, D, prec, work)     # raises TN_ERR_NUMERIC if inconsistent
    assert info["ops"] > 0 and info["waves"] > 0
    assert 0 < info["arena_bytes"] < info["footprint_bytes"]


@pytest.mark.parametrize("sched", [tn.TN_SCHED_ROW, tn.TN_SCHED_COL, tn.TN_SCHED_QUADRANT])
def test_forced_schedules_are_consistent(cpu_ctx, sched):
    for L, W, D in [(4, 6, 2), (5, 5, 2), (3, 4, 3)]:
        _info(cpu_ctx, L, W, D, tn.TN_FP32, tn.TN_WORK_ENERGY, sched)


def test_fused_pairs_only_where_the_fp32_kernel_runs(cpu_ctx):
    # FP64 programs take one step at a time; FP32 D = 2 energies fuse chain steps
    assert _info(cpu_ctx, 8, 8, 2, tn.TN_FP64, tn.TN_WORK_ENERGY)["fused_pairs"] == 0
    f32 = _info(cpu_ctx, 8, 8, 2, tn.TN_FP32, tn.TN_WORK_ENERGY)
    f64 = _info(cpu_ctx, 8, 8, 2, tn.TN_FP64, tn.TN_WORK_ENERGY)
    assert f32["fused_pairs"] > 0
    # the same contractions, except that FP64 divides every ratio by the ring's norm and so
    # skips the four products that give the cut-crossing bonds their path norms (256^3 each)
    assert f32["product_macs"] - f64["product_macs"] == 4 * 256 ** 3
    # absorption bytes (per entry) lower in FP32 by the fused intermediates
    assert f32["absorb_bytes"] / 4 < f64["absorb_bytes"] / 8
    # the 8x8 D=2 energy moves 80.8 MB per lattice in FP32 (125 MB before fusion)
    assert 80e6 < f32["absorb_bytes"] < 82e6
    # a norm has no observable chains, hence nothing to fuse
    assert _info(cpu_ctx, 8, 8, 2, tn.TN_FP32, tn.TN_WORK_NORM)["fused_pairs"] == 0


def test_invalid_work_is_rejected(cpu_ctx):
    lat = tn.tn_create_lattice(cpu_ctx, 3, 3, 2)
    try:
        with pytest.raises(tn.TNError) as e:
            tn.tn_program_info(lat, tn.TN_FP32, tn.TN_SCHED_AUTO, 5)
        assert e.value.status == tn.TN_ERR_INVALID
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,D", SHAPES + [(6, 6, 3), (7, 7, 3), (8, 8, 3), (2, 9, 3), (9, 1, 2), (5, 4, 4)])
@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X6])
def test_recompute_programs_are_consistent(cpu_ctx, L, W, D, prec):
    """Program choice bit 32 (the recompute form): the same checks, every
    product of the cached form kept, the recomputed chain steps on top, and
    never more memory than the cached form once the cached chain states pass
    a few megabytes."""
    tn.tn_autotune_clear()
    try:
        cached = _info(cpu_ctx, L, W, D, prec, tn.TN_WORK_ENERGY)
        tn.tn_autotune_set(L, W, D, prec, tn.TN_WORK_ENERGY, 15 | 32)
        rec = _info(cpu_ctx, L, W, D, prec, tn.TN_WORK_ENERGY)
    finally:
        tn.tn_autotune_clear()
    assert rec["product_macs"] == cached["product_macs"]
    assert rec["ops"] >= cached["ops"] and rec["absorb_bytes"] >= cached["absorb_bytes"]
    if cached["arena_bytes"] > 4e6:
        assert rec["footprint_bytes"] < cached["footprint_bytes"]
