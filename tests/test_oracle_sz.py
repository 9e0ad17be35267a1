"""Pins of the oracle's single-site <Z_k> and the connected correlator
c_ij = <Z_i Z_j> - <Z_i><Z_j> (Sec. 3, Eqs. mz and cij, Pauli Z with
p = 1 <-> sigma = +1), against the 2^N state vector, the D = 1 product closed
form (where c_ij vanishes identically), the Z2-symmetric Ising PEPS (where
<Z_k> = 0) and the all-ones workload."""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs


@pytest.mark.parametrize("L,W,D", [(1, 3, 2), (2, 2, 2), (3, 3, 2), (2, 3, 3), (4, 4, 2), (3, 4, 1)])
def test_sz_matches_state_vector(L, W, D):
    A = inputs.random_lattice(L, W, D, 5000 + 31 * L + 7 * W + D)
    ob = oracle.observables(L, W, D, A, with_z=True)
    np.testing.assert_allclose(ob.sz, brute.sz(L, W, D, A), rtol=0, atol=1e-12)
    # connected correlator straight from the state vector
    n, _, zz = brute.observables(L, W, D, A)
    z = brute.sz(L, W, D, A)
    c = [zz[b] - z[ri * W + ci] * z[rj * W + cj] for b, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W))]
    np.testing.assert_allclose(ob.connected(L, W), c, rtol=0, atol=1e-12)


@pytest.mark.parametrize("L,W", [(3, 5), (6, 6)])
def test_sz_product_closed_form(L, W):
    rng = np.random.default_rng(7 * L + W)
    a0, a1 = rng.uniform(-1, 1, L * W), rng.uniform(-1, 1, L * W)
    ob = oracle.observables(L, W, 1, inputs.product_lattice(L, W, a0, a1), with_z=True)
    np.testing.assert_allclose(ob.sz, (a1 ** 2 - a0 ** 2) / (a0 ** 2 + a1 ** 2), atol=1e-13)
    np.testing.assert_allclose(ob.connected(L, W), 0.0, atol=1e-13)


@pytest.mark.parametrize("L,W,K", [(3, 3, 0.3), (3, 4, 0.7)])
def test_sz_vanishes_for_ising_peps(L, W, K):
    """psi(s) = psi(-s): <Z_k> = 0 and c_ij = <s_i s_j> of the classical model."""
    ob = oracle.observables(L, W, 2, inputs.ising_peps_lattice(L, W, K), with_z=True)
    _, corr, _ = oracle.ising_enumerate(L, W, K)
    np.testing.assert_allclose(ob.sz, 0.0, atol=1e-13)
    np.testing.assert_allclose(ob.connected(L, W), corr, atol=1e-12)


def test_sz_all_ones_is_zero():
    ob = oracle.observables(4, 5, 2, inputs.ones_lattice(4, 5, 2), with_z=True)
    assert np.all(ob.sz == 0.0)


def test_expect_one_z_matches_cached():
    L, W, D = 4, 5, 2
    A = inputs.random_lattice(L, W, D, 41)
    ob = oracle.observables(L, W, D, A, with_z=True)
    for k in (0, 6, 13, 19):
        v, _, _ = oracle.expect_one(L, W, D, A, "z", k)
        assert abs(v - ob.sz[k]) < 1e-12
