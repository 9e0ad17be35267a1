"""Pins of the oracle's nearest-neighbour two-site correlators <A_i B_j>,
A, B in {X, Z} (the insertion of Sec. 5 with one operator on each site of a
bond): the 2^N state vector, the D = 1 product closed form (<A_i B_j> =
<A_i><B_j>), the all-ones lattice (the uniform superposition: <X_i X_j> = 1,
every correlator with a Z is 0) and the ZZ case of the energy path."""
import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs

PAIRS = [("x", "x"), ("x", "z"), ("z", "x"), ("z", "z")]


@pytest.mark.parametrize("L,W,D", [(1, 4, 2), (2, 3, 2), (3, 3, 2), (2, 3, 3), (3, 4, 1)])
@pytest.mark.parametrize("a,b", PAIRS)
def test_bonds_match_state_vector(L, W, D, a, b):
    A = inputs.random_lattice(L, W, D, 700 + 11 * L + W + D)
    np.testing.assert_allclose(oracle.bond_correlators(L, W, D, A, a, b),
                               brute.bond_correlators(L, W, D, A, a, b), rtol=0, atol=1e-12)


@pytest.mark.parametrize("a,b", PAIRS)
def test_bonds_product_closed_form(a, b):
    L, W = 4, 5
    rng = np.random.default_rng(45)
    a0, a1 = rng.uniform(-1, 1, L * W), rng.uniform(-1, 1, L * W)
    q = a0 ** 2 + a1 ** 2
    one = {"x": 2 * a0 * a1 / q, "z": (a1 ** 2 - a0 ** 2) / q}
    ref = [one[a][ri * W + ci] * one[b][rj * W + cj] for (ri, ci), (rj, cj) in inputs.bonds(L, W)]
    got = oracle.bond_correlators(L, W, 1, inputs.product_lattice(L, W, a0, a1), a, b)
    np.testing.assert_allclose(got, ref, atol=1e-13)


def test_bonds_all_ones():
    L, W = 4, 4
    A = inputs.ones_lattice(L, W, 2)
    assert np.all(oracle.bond_correlators(L, W, 2, A, "x", "x") == 1.0)
    for a, b in PAIRS[1:]:
        assert np.all(oracle.bond_correlators(L, W, 2, A, a, b) == 0.0)


def test_zz_matches_energy_path():
    L, W, D = 4, 5, 2
    A = inputs.random_lattice(L, W, D, 17)
    np.testing.assert_allclose(oracle.bond_correlators(L, W, D, A, "z", "z"),
                               oracle.observables(L, W, D, A).szsz, rtol=0, atol=1e-14)
