"""Failure detection without a GPU fault: a device wait on a flag that nothing
sets runs out after its short limit, the kernel records the expiry and exits,
the host reads the status, and the context stays usable for a contraction."""
import numpy as np
import pytest

import oracle
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu


def test_bounded_wait_expires_and_context_survives():
    import torch
    torch.cuda.init()
    ctx = tn.tn_ctx_create(0, 0)
    try:
        assert tn.tn_wait_selfcheck(ctx, 20.0)
        L, W, D = 3, 3, 2
        A = inputs.random_lattice(L, W, D, 5)
        lat = tn.tn_create_lattice(ctx, L, W, D)
        try:
            tn.tn_set_site_tensors(lat, A)
            r, sx, zz = tn.tn_energy(lat, 1.0, 3.04, tn.TN_FP64, tn.TN_SCHED_AUTO, L, W)
        finally:
            tn.tn_destroy_lattice(lat)
        ref = oracle.observables(L, W, D, A)
        assert abs(r.energy - ref.energy(1.0, 3.04)) <= 1e-10 * abs(ref.energy(1.0, 3.04))
        np.testing.assert_allclose(sx, ref.sx, atol=1e-10)
    finally:
        tn.tn_ctx_destroy(ctx)
