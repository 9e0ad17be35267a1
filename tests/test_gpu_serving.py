"""Serving (tn_submit / tn_poll / tn_wait): continuous batching under an HBM budget.

* every served result equals the same lattice evaluated alone (tn_energy),
  bit for bit, whatever else shared its batch;
* a budget that holds only a few jobs at a time still completes every job,
  and all budget memory returns when the queue drains;
* a job larger than the whole budget is refused at submit time;
* tn_wait honours its deadline; tn_poll reports NOT_READY then the result.
"""
import numpy as np
import pytest

import oracle
from energy_tol import check_energy
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

MIX = [(4, 4, 2, tn.TN_FP32), (3, 5, 2, tn.TN_FP32), (5, 5, 2, tn.TN_FP32), (4, 4, 3, tn.TN_FP32),
       (6, 4, 2, tn.TN_FP64), (4, 6, 2, tn.TN_FP64), (5, 3, 3, tn.TN_FP32), (6, 6, 2, tn.TN_FP32)]


def _alone(ctx, L, W, D, A, prec, h):
    lat = tn.tn_create_lattice(ctx, L, W, D)
    try:
        tn.tn_set_site_tensors(lat, A)
        return tn.tn_energy(lat, 1.0, h, prec, tn.TN_SCHED_AUTO, L, W)
    finally:
        tn.tn_destroy_lattice(lat)


def test_served_results_equal_alone_bitwise():
    import torch
    torch.cuda.init()
    ctx = tn.tn_ctx_create(0, 0)
    try:
        jobs = []
        for k in range(24):
            L, W, D, prec = MIX[k % len(MIX)]
            A = inputs.random_lattice(L, W, D, 500 + k)
            h = 0.5 + 0.2 * k
            t = tn.tn_submit(ctx, L, W, D, prec, 1.0, h, tensors=A)
            jobs.append((t, L, W, D, prec, A, h))
        for t, L, W, D, prec, A, h in jobs:
            r, sx, zz = tn.tn_wait(ctx, t, 60.0, L, W)
            ra, sxa, zza = _alone(ctx, L, W, D, A, prec, h)
            assert r.energy == ra.energy
            assert np.array_equal(sx, sxa) and np.array_equal(zz, zza)
            assert (r.norm.mant, r.norm.exp2) == (ra.norm.mant, ra.norm.exp2)
        # and against the oracle for two of them
        for t, L, W, D, prec, A, h in jobs[:2]:
            ref = oracle.observables(L, W, D, A)
            ra, _, _ = _alone(ctx, L, W, D, A, prec, h)
            check_energy(ra.energy, ref.energy(1.0, h), ref.sx, ref.szsz, 1.0, h, prec)
    finally:
        tn.tn_ctx_destroy(ctx)


def test_budget_admission_and_release():
    import torch
    torch.cuda.init()
    probe_ctx = tn.tn_ctx_create(-1)
    lat = tn.tn_create_lattice(probe_ctx, 6, 6, 2)
    fp = tn.tn_footprint(lat, tn.TN_SCHED_AUTO, tn.TN_FP32, tn.TN_WORK_ENERGY)
    tn.tn_destroy_lattice(lat)
    tn.tn_ctx_destroy(probe_ctx)
    budget = int(2.5 * fp)          # at most two 6x6 jobs on the device at once
    ctx = tn.tn_ctx_create(0, budget)
    try:
        tickets = []
        for k in range(10):
            A = inputs.random_lattice(6, 6, 2, 900 + k)
            tickets.append((tn.tn_submit(ctx, 6, 6, 2, tn.TN_FP32, 1.0, 3.04, tensors=A), A))
        for t, A in tickets:
            r, sx, zz = tn.tn_wait(ctx, t, 60.0, 6, 6)
            ref = oracle.observables(6, 6, 2, A)
            check_energy(r.energy, ref.energy(1.0, 3.04), ref.sx, ref.szsz, 1.0, 3.04, tn.TN_FP32)
        used, b = tn.tn_ctx_memory(ctx)
        assert b == budget and used == 0
        # a job that can never fit is refused up front
        with pytest.raises(tn.TNError) as e:
            tn.tn_submit(ctx, 10, 10, 2, tn.TN_FP32, 1.0, 3.04, seed=1)
        assert e.value.status == tn.TN_ERR_OVER_BUDGET
    finally:
        tn.tn_ctx_destroy(ctx)


def test_wait_deadline_and_poll():
    import torch
    torch.cuda.init()
    ctx = tn.tn_ctx_create(0, 0)
    try:
        ts = [tn.tn_submit(ctx, 8, 8, 2, tn.TN_FP64, 1.0, 3.04, seed=k) for k in range(40)]
        # the last of 40 queued FP64 jobs cannot be finished at once
        with pytest.raises(tn.TNError) as e:
            tn.tn_wait(ctx, ts[-1], 0.0, 8, 8)
        assert e.value.status == tn.TN_ERR_TIMEOUT
        got = None
        for _ in range(200000):
            got = tn.tn_poll(ctx, ts[0], 8, 8)
            if got is not None:
                break
        assert got is not None
        lat = tn.tn_create_lattice(ctx, 8, 8, 2)
        tn.tn_fill_random(lat, 0)
        ra, _, _ = tn.tn_energy(lat, 1.0, 3.04, tn.TN_FP64, tn.TN_SCHED_AUTO, 8, 8)
        tn.tn_destroy_lattice(lat)
        assert got[0].energy == ra.energy
        for t in ts[1:]:
            tn.tn_wait(ctx, t, 120.0, 8, 8)
        with pytest.raises(tn.TNError) as e:
            tn.tn_poll(ctx, ts[0], 8, 8)      # a ticket is released once read
        assert e.value.status == tn.TN_ERR_INVALID
    finally:
        tn.tn_ctx_destroy(ctx)


def test_served_wait_timeout_reaches_the_caller():
    """A served batch whose status word says a bounded device wait ran out
    reports TN_ERR_TIMEOUT to every job in it (host-side injection: the word is
    set after the batch's kernels, as an expired wait would set it); the next
    job, and a blocking call after one injected failure, run normally."""
    import torch
    torch.cuda.init()
    ctx = tn.tn_ctx_create(0, 0)
    try:
        L, W, D = 5, 5, 3          # 729-wide ring products on the tensor cores in BF16x3
        A = inputs.random_lattice(L, W, D, 77)
        tn.tn_ctx_inject_wait_timeout(ctx, 1)
        t = tn.tn_submit(ctx, L, W, D, tn.TN_BF16X3, 1.0, 3.04, tensors=A)
        with pytest.raises(tn.TNError) as e:
            tn.tn_wait(ctx, t, 60.0, L, W)
        assert e.value.status == tn.TN_ERR_TIMEOUT
        t = tn.tn_submit(ctx, L, W, D, tn.TN_BF16X3, 1.0, 3.04, tensors=A)
        r, sx, zz = tn.tn_wait(ctx, t, 60.0, L, W)
        ra, sxa, zza = _alone(ctx, L, W, D, A, tn.TN_BF16X3, 3.04)
        assert r.energy == ra.energy and np.array_equal(sx, sxa)
        # the blocking path reads the same word
        lat = tn.tn_create_lattice(ctx, L, W, D)
        try:
            tn.tn_set_site_tensors(lat, A)
            tn.tn_ctx_inject_wait_timeout(ctx, 1)
            with pytest.raises(tn.TNError) as e:
                tn.tn_energy(lat, 1.0, 3.04, tn.TN_BF16X3, tn.TN_SCHED_AUTO, L, W)
            assert e.value.status == tn.TN_ERR_TIMEOUT
            r2, _, _ = tn.tn_energy(lat, 1.0, 3.04, tn.TN_BF16X3, tn.TN_SCHED_AUTO, L, W)
            assert r2.energy == ra.energy
        finally:
            tn.tn_destroy_lattice(lat)
    finally:
        tn.tn_ctx_destroy(ctx)


def test_light_jobs_overtake_a_heavy_one():
    # an 8x9 D=3 FP32 energy (seconds of work, a low-priority stream of its
    # own) must not hold back 4x4 D=2 jobs submitted after it: they finish
    # while it is still running, and every result equals its alone value
    import time

    import torch
    torch.cuda.init()
    ctx = tn.tn_ctx_create(0, 0)
    try:
        Lh, Wh, Dh = 8, 9, 3
        Ah = inputs.random_lattice(Lh, Wh, Dh, 899)
        th = tn.tn_submit(ctx, Lh, Wh, Dh, tn.TN_FP32, 1.0, 3.04, tensors=Ah)
        time.sleep(0.2)
        light = []
        for k in range(6):
            A = inputs.random_lattice(4, 4, 2, 440 + k)
            light.append((tn.tn_submit(ctx, 4, 4, 2, tn.TN_FP32, 1.0, 3.04, tensors=A), A))
        got = [tn.tn_wait(ctx, t, 30.0, 4, 4) for t, _ in light]
        assert tn.tn_poll(ctx, th, Lh, Wh) is None        # the heavy job is still running
        r, _, _ = tn.tn_wait(ctx, th, 300.0, Lh, Wh)
        ra, _, _ = _alone(ctx, Lh, Wh, Dh, Ah, tn.TN_FP32, 3.04)
        assert r.energy == ra.energy
        for (r, sx, zz), (_, A) in zip(got, light):
            ra, sxa, zza = _alone(ctx, 4, 4, 2, A, tn.TN_FP32, 3.04)
            assert r.energy == ra.energy and np.array_equal(sx, sxa) and np.array_equal(zz, zza)
    finally:
        tn.tn_ctx_destroy(ctx)
