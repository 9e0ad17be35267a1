"""Pins of the oracle's arbitrary-pair correlators (oracle.pair), CPU only.

Any two sites, any of X, Y, Z on each, against the complex 2^N state vector
with the Pauli matrices applied directly (oracle.brute.pair_correlator) -- Y
there is the complex matrix itself, not the real R the contraction uses; and
against the nearest-neighbour correlators already pinned, where they overlap.
"""
import itertools

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs


@pytest.mark.parametrize("L,W,D", [(3, 3, 2), (2, 4, 2), (3, 2, 3)])
def test_pairs_against_the_state_vector(L, W, D):
    A = inputs.random_lattice(L, W, D, 500 + L * W + D)
    N = L * W
    rng = np.random.default_rng(L * 10 + W)
    pairs = [(0, N - 1), (1, N - 2), (0, 1)] + [tuple(rng.choice(N, 2, replace=False)) for _ in range(3)]
    for (i, j), (a, b) in itertools.product(pairs, itertools.product("xyz", repeat=2)):
        ref = brute.pair_correlator(L, W, D, A, a, int(i), b, int(j))
        got = oracle.pair(L, W, D, A, a, int(i), b, int(j))
        assert isinstance(ref, float), (a, b, ref)      # real for a real state
        assert abs(got - ref) < 1e-12, (a, b, i, j, got, ref)


def test_mixed_y_vanishes_and_yy_is_real():
    L, W, D = 3, 3, 2
    A = inputs.random_lattice(L, W, D, 12)
    assert brute.pair_correlator(L, W, D, A, "x", 0, "y", 8) == pytest.approx(0.0, abs=1e-14)
    assert brute.pair_correlator(L, W, D, A, "y", 2, "z", 4) == pytest.approx(0.0, abs=1e-14)
    v = brute.pair_correlator(L, W, D, A, "y", 0, "y", 8)
    assert isinstance(v, float) and abs(v) > 1e-6


def test_nearest_neighbour_pairs_match_the_bond_correlators():
    L, W, D = 4, 3, 2
    A = inputs.random_lattice(L, W, D, 33)
    for a, b in (("x", "z"), ("z", "z")):
        bonds = oracle.bond_correlators(L, W, D, A, a, b)
        for k, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W)):
            assert abs(oracle.pair(L, W, D, A, a, ri * W + ci, b, rj * W + cj) - bonds[k]) < 1e-12
