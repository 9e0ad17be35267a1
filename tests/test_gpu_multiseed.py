"""8x8 D=2 parity over 16 seeded lattices: every precision against the oracle.

The lattices are lattice_seed(4242, k), k < 16, with h cycling through
{2.0, 3.04, 4.0}; among them are energies whose terms nearly cancel (k = 2:
E = 0.080 at h = 2 against a scale S = 48), where the reduced precisions are
held to |dE| <= 1e-6 S and FP64 to |dE| <= 1e-10 |E| (energy_tol).  All 16
run as one batch per precision (one CUDA graph), so this also exercises the
grouped launches at a size between the single-lattice tests and the bench.
"""
import numpy as np
import pytest

import oracle
from energy_tol import check_energy, energy_errors
from paper_1908_08553_gb300 import inputs, tn

pytestmark = pytest.mark.gpu

L, W, D, NLAT = 8, 8, 2, 16
HS = np.array([(2.0, 3.04, 4.0)[k % 3] for k in range(NLAT)])
TOL_OBS = {tn.TN_FP64: 1e-10, tn.TN_FP32: 1e-6, tn.TN_BF16X6: 1e-6, tn.TN_BF16X3: 1e-5}


@pytest.fixture(scope="module")
def lattices():
    out = []
    for k in range(NLAT):
        A = inputs.random_lattice(L, W, D, inputs.lattice_seed(4242, k))
        out.append((A, oracle.observables(L, W, D, A)))
    return out


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


@pytest.mark.parametrize("prec", [tn.TN_FP64, tn.TN_FP32, tn.TN_BF16X6, tn.TN_BF16X3])
def test_8x8_d2_sixteen_seeds(ctx, lattices, prec):
    b = tn.tn_batch_create(ctx, [L] * NLAT, [W] * NLAT, [D] * NLAT, prec)
    try:
        tn.tn_batch_set_tensors(b, np.concatenate([A for A, _ in lattices]))
        tn.tn_batch_run(b, 1.0, HS)
        res = tn.tn_batch_results_host(b)
    finally:
        tn.tn_batch_destroy(b)
    nb = L * (W - 1) + W * (L - 1)
    stride = 6 + 2 * L * W + nb
    worst = []
    for k, (A, ref) in enumerate(lattices):
        seg = res[k * stride:(k + 1) * stride]
        e_ref = ref.energy(1.0, HS[k])
        worst.append(check_energy(seg[0], e_ref, ref.sx, ref.szsz, 1.0, HS[k], prec))
        sx, zz = seg[6:6 + L * W], seg[6 + L * W:6 + L * W + nb]
        tol = TOL_OBS[prec]
        assert np.max(np.abs(sx - ref.sx)) <= tol, (k, np.max(np.abs(sx - ref.sx)))
        assert np.max(np.abs(zz - ref.szsz)) <= tol, (k, np.max(np.abs(zz - ref.szsz)))
        # the header's sums are the sums of the returned terms
        assert abs(seg[4] - sx.sum()) <= 1e-12 * max(1.0, np.abs(sx).sum())
    rel = max(w[0] for w in worst)
    rel_s = max(w[1] for w in worst)
    print(f"prec {prec}: max |dE|/|E| = {rel:.3g}, max |dE|/S = {rel_s:.3g}")
