"""Pins of the oracle's imaginary time evolution (oracle/ite.py), CPU only.

* Without truncation (chains and short runs whose SVDs drop nothing), the PEPS
  after m Trotter steps is exactly the state vector evolved by the same gates
  applied to the 2^N amplitudes directly: exp(Gamma t X) as c psi + s psi(bit
  flipped), exp(J t Z_i Z_j) as a sign-dependent factor per basis state (Sec. 5,
  second-order Trotter split).
* The ITE energy is an expectation value of H, so it can never lie below the
  exact ground energy (variational bound), and with chi_max = 2, tau = 3 in 200
  steps on 2x2 and 3x3 it comes close to it (Fig. 4).
* J = 0: the initial state is an eigenstate of every one-body gate, so it stays
  the uniform superposition: <X_k> = 1, E = -Gamma N.
* The SVD split keeps what the cutoff says: a bond never exceeds chi_max, and a
  large eps leaves bond dimension 1.
"""
import math

import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.ite as ite


def trotter_state_vector(L, W, J, gamma, dtau, steps):
    N = L * W
    idx = np.arange(1 << N)
    psi = np.full(1 << N, 2.0 ** (-N / 2))
    c, s = math.cosh(gamma * dtau / 2), math.sinh(gamma * dtau / 2)
    sig = [np.where((idx >> k) & 1, 1.0, -1.0) for k in range(N)]
    from paper_1908_08553_gb300.inputs import bonds
    phase = np.zeros(1 << N)
    for (ri, ci), (rj, cj) in bonds(L, W):
        phase += sig[ri * W + ci] * sig[rj * W + cj]
    zz = np.exp(J * dtau * phase)

    def one_body(v):
        for k in range(N):
            v = c * v + s * v[idx ^ (1 << k)]
        return v

    for _ in range(steps):
        psi = one_body(psi)
        psi = psi * zz
        psi = one_body(psi)
        psi /= np.linalg.norm(psi)
    return psi


@pytest.mark.parametrize("L,W,chi,steps", [(1, 3, 2, 5), (3, 1, 2, 5), (1, 4, 4, 4), (4, 1, 4, 4), (2, 2, 4, 1)])
def test_untruncated_evolution_is_the_trotter_state(L, W, chi, steps):
    J, gamma, dtau = 0.8, 1.3, 0.1
    r = ite.evolve(L, W, J, gamma, dtau, steps, chi, 0.0, energy_every=0)
    assert r["max_discarded"] < 1e-12            # nothing was truncated
    psi = brute.state_vector(L, W, chi, r["flat"])
    psi /= np.linalg.norm(psi)
    ref = trotter_state_vector(L, W, J, gamma, dtau, steps)
    assert abs(abs(psi @ ref) - 1.0) < 1e-12
    # and the energy of the exact contraction is that of the state vector
    ob = oracle.observables(L, W, chi, r["flat"])
    H = brute.hamiltonian(L, W, J, gamma)
    assert abs(ob.energy(J, gamma) - float(ref @ (H @ ref))) < 1e-10 * (L * W)


@pytest.mark.parametrize("L,W", [(2, 2), (3, 3)])
@pytest.mark.parametrize("gamma", [0.5, 1.0, 3.0])
def test_ite_energy_is_variational_and_close_to_ed(L, W, gamma):
    r = ite.evolve(L, W, 1.0, gamma, 3.0 / 200, 200, 2, 0.0, energy_every=50)
    e0 = brute.ground_energy(L, W, 1.0, gamma)
    N = L * W
    for _, e in r["energies"]:
        assert e >= e0 - 1e-9
    assert (r["energies"][-1][1] - e0) / N < 1e-2
    assert max(r["bond_dims"]) <= 2


def test_no_coupling_keeps_the_uniform_superposition():
    L, W, gamma = 3, 3, 0.7
    r = ite.evolve(L, W, 0.0, gamma, 0.05, 6, 2, 0.01, energy_every=2)
    ob = oracle.observables(L, W, 2, r["flat"])
    np.testing.assert_allclose(ob.sx, 1.0, atol=1e-12)
    for _, e in r["energies"]:
        assert abs(e + gamma * L * W) < 1e-11
    assert max(r["bond_dims"]) == 1


def test_cutoff_limits_the_bond_dimension():
    r = ite.evolve(3, 3, 1.0, 1.0, 0.05, 4, 3, 0.0, energy_every=0)
    assert max(r["bond_dims"]) <= 3 and max(r["bond_dims"]) >= 2
    r = ite.evolve(3, 3, 1.0, 1.0, 0.05, 4, 3, 0.9, energy_every=0)
    assert max(r["bond_dims"]) == 1
