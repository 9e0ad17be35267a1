"""Imaginary time evolution on the GPU (tn_ite_run, Sec. 5) against the oracle.

* The GPU evolution and the oracle's (oracle/ite.py: numpy SVD, the same gate
  order) give the same energies at every evaluation and the same final
  observables; the SVD gauge may differ, so states are compared through
  what they compute, not tensor by tensor.
* Without truncation the evolved state is the Trotterised 2^N state vector.
* Fig. 4's setting (2x2 and 3x3, chi = 2, tau = 3 in 200 steps): the energy is
  above the exact ground energy and within 1e-2 per site of it.
* A D = 4 lattice exercises 128 x 128 SVDs.
"""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.ite as ite
from paper_1908_08553_gb300 import tn
from test_oracle_ite import trotter_state_vector

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    import torch
    torch.cuda.init()
    c = tn.tn_ctx_create(0, 0)
    yield c
    tn.tn_ctx_destroy(c)


def _gpu_ite(ctx, L, W, J, gamma, dtau, steps, chi, eps, every, prec=tn.TN_FP64):
    lat = tn.tn_create_lattice(ctx, L, W, chi)
    try:
        tn.tn_ite_init_product(lat)
        en, dims, disc = tn.tn_ite_run(lat, L, W, J, gamma, dtau, steps, chi, eps, every, prec)
        flat = tn.tn_get_site_tensors(lat, tn.tn_lattice_elems(L, W, chi))
        return en, dims, disc, flat
    finally:
        tn.tn_destroy_lattice(lat)


@pytest.mark.parametrize("L,W,chi,gamma,steps", [(3, 3, 2, 1.0, 20), (2, 4, 3, 2.0, 12), (4, 3, 2, 0.5, 16)])
def test_gpu_ite_matches_oracle(ctx, L, W, chi, gamma, steps):
    J, dtau, eps = 1.0, 0.03, 0.01
    en, dims, disc, flat = _gpu_ite(ctx, L, W, J, gamma, dtau, steps, chi, eps, 2)
    ref = ite.evolve(L, W, J, gamma, dtau, steps, chi, eps, energy_every=2)
    e_ref = np.array([e for _, e in ref["energies"]])
    assert en.shape == e_ref.shape
    np.testing.assert_allclose(en, e_ref, rtol=1e-9, atol=0)
    assert list(dims) == list(ref["bond_dims"])
    assert abs(disc - ref["max_discarded"]) <= 1e-9
    ob, ob_ref = oracle.observables(L, W, chi, flat), oracle.observables(L, W, chi, ref["flat"])
    np.testing.assert_allclose(ob.sx, ob_ref.sx, atol=1e-9)
    np.testing.assert_allclose(ob.szsz, ob_ref.szsz, atol=1e-9)
    # the evolved state is normalised
    assert abs(ob.log2_norm) < 1e-9


@pytest.mark.parametrize("L,W,chi,steps", [(1, 4, 4, 4), (4, 1, 4, 4), (2, 2, 4, 1), (1, 3, 2, 6)])
def test_gpu_ite_untruncated_is_the_trotter_state(ctx, L, W, chi, steps):
    J, gamma, dtau = 0.8, 1.3, 0.1
    en, dims, disc, flat = _gpu_ite(ctx, L, W, J, gamma, dtau, steps, chi, 1e-13, 0)
    assert disc < 1e-12
    psi = brute.state_vector(L, W, chi, flat)
    psi /= np.linalg.norm(psi)
    ref = trotter_state_vector(L, W, J, gamma, dtau, steps)
    assert abs(abs(psi @ ref) - 1.0) < 1e-11


@pytest.mark.parametrize("L,W", [(2, 2), (3, 3)])
@pytest.mark.parametrize("gamma", [0.5, 3.0])
def test_gpu_ite_fig4_regime(ctx, L, W, gamma):
    en, dims, disc, flat = _gpu_ite(ctx, L, W, 1.0, gamma, 3.0 / 200, 200, 2, 0.0, 50)
    e0 = brute.ground_energy(L, W, 1.0, gamma)
    assert np.all(en >= e0 - 1e-9)
    assert (en[-1] - e0) / (L * W) < 1e-2
    ref = ite.evolve(L, W, 1.0, gamma, 3.0 / 200, 200, 2, 0.0, energy_every=50)
    np.testing.assert_allclose(en, [e for _, e in ref["energies"]], rtol=1e-9)


def test_gpu_ite_d4_large_svds(ctx):
    """D = 4 interior bonds: Theta of 128 x 128, the largest the kernel takes;
    with eps = 1e-4 every bond fills to chi = 4 and truncation drops a value."""
    L, W, chi = 4, 4, 4
    en, dims, disc, flat = _gpu_ite(ctx, L, W, 1.0, 1.5, 0.05, 6, chi, 1e-4, 2)
    ref = ite.evolve(L, W, 1.0, 1.5, 0.05, 6, chi, 1e-4, energy_every=2)
    np.testing.assert_allclose(en, [e for _, e in ref["energies"]], rtol=1e-9)
    assert list(dims) == list(ref["bond_dims"]) and min(dims) == 4
    assert abs(disc - ref["max_discarded"]) <= 1e-9 and disc > 1e-4


def test_gpu_ite_energies_in_fp32(ctx):
    """Energy evaluations in FP32 (the evolution itself stays FP64)."""
    L, W, chi = 3, 3, 2
    en64, _, _, _ = _gpu_ite(ctx, L, W, 1.0, 1.0, 0.03, 10, chi, 0.01, 2, tn.TN_FP64)
    en32, _, _, _ = _gpu_ite(ctx, L, W, 1.0, 1.0, 0.03, 10, chi, 0.01, 2, tn.TN_FP32)
    np.testing.assert_allclose(en32, en64, rtol=1e-5)
