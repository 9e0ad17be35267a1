"""Pins for the FP64 CPU oracle: it is checked against things other than itself.

Each test ties the oracle to a fact fixed by the paper or by mathematics:
brute-force state vectors (Eqs. Psi, norm, mx, cij, Etot), the explicit TFIM
Hamiltonian and its exact ground energy, closed forms (D = 1 product states,
the all-ones workload of Sec. 6, 1D and 2x2 Ising), enumeration of the
classical Ising model written as a tensor network, and invariances of an exact
contraction (order, gauge, scale).  A dropped term, a sign error, a wrong leg
index or a transposed operand in the oracle breaks at least one of them.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle
import oracle.brute as brute
import oracle.planner as planner
from paper_1908_08553_gb300 import inputs

GOLD = os.path.join(os.path.dirname(__file__), "golden")


def _value(m, e):
    return m * 2.0 ** e


# ------------------------------------------------------ brute force (Sec. 3)

@pytest.mark.parametrize("L,W,D", [(1, 1, 2), (1, 4, 2), (2, 2, 1), (2, 2, 2), (2, 3, 3),
                                   (3, 3, 2), (3, 2, 3), (4, 4, 2), (4, 3, 3), (4, 4, 1)])
def test_oracle_matches_state_vector(L, W, D):
    A = inputs.random_lattice(L, W, D, 1000 + 17 * L + W + 101 * D)
    ob = oracle.observables(L, W, D, A)
    n, sx, zz = brute.observables(L, W, D, A)
    assert abs(_value(ob.norm_m, ob.norm_e) - n) <= 1e-12 * abs(n)
    np.testing.assert_allclose(ob.sx, sx, rtol=0, atol=1e-12)
    np.testing.assert_allclose(ob.szsz, zz, rtol=0, atol=1e-12)


def test_oracle_4x4_d3_state_vector():
    L = W = 4
    D = 3
    A = inputs.random_lattice(L, W, D, 77)
    ob = oracle.observables(L, W, D, A)
    n, sx, zz = brute.observables(L, W, D, A)
    assert abs(_value(ob.norm_m, ob.norm_e) - n) <= 1e-12 * abs(n)
    np.testing.assert_allclose(ob.sx, sx, atol=1e-12)
    np.testing.assert_allclose(ob.szsz, zz, atol=1e-12)


@pytest.mark.parametrize("h", [2.0, 3.04, 4.0])
def test_energy_equals_hamiltonian_expectation(h):
    """E from the oracle equals <psi|H|psi>/<psi|psi> with H built explicitly."""
    L, W, D = 4, 4, 2
    A = inputs.random_lattice(L, W, D, 2024)
    ob = oracle.observables(L, W, D, A)
    e_tn = ob.energy(1.0, h)
    e_h = brute.energy(L, W, D, A, 1.0, h)
    assert abs(e_tn - e_h) <= 1e-12 * abs(e_h)


def test_energy_above_exact_ground_state():
    """Variational bound: any state's energy is >= E_0 of the 4x4 TFIM."""
    L, W, D, h = 4, 4, 2, 3.04
    e0 = brute.ground_energy(L, W, 1.0, h)
    for seed in (1, 2, 3):
        A = inputs.random_lattice(L, W, D, seed)
        assert oracle.observables(L, W, D, A).energy(1.0, h) >= e0 - 1e-9
    # the uniform superposition of Sec. 5 (all sigma equal weight, chi = 1) has
    # <X> = 1 and <ZZ> = 0, hence E = -h N, also above E_0
    a = np.full(L * W, 1.0 / math.sqrt(2.0))
    ob = oracle.observables(L, W, 1, inputs.product_lattice(L, W, a, a))
    assert abs(ob.energy(1.0, h) + h * L * W) < 1e-12
    assert -h * L * W >= e0


# ---------------------------------------------------- closed forms (D = 1)

@pytest.mark.parametrize("L,W", [(3, 5), (6, 6), (12, 12)])
def test_product_state_closed_form(L, W):
    rng = np.random.default_rng(L * 100 + W)
    a0 = rng.uniform(-1, 1, L * W)
    a1 = rng.uniform(-1, 1, L * W)
    A = inputs.product_lattice(L, W, a0, a1)
    ob = oracle.observables(L, W, 1, A)
    q = a0 ** 2 + a1 ** 2
    log2n = np.sum(np.log2(q))
    assert abs(ob.log2_norm - log2n) < 1e-12 * max(1.0, abs(log2n))
    np.testing.assert_allclose(ob.sx, 2 * a0 * a1 / q, atol=1e-13)
    z = (a1 ** 2 - a0 ** 2) / q       # p = 1 is sigma = +1
    zz = [z[ri * W + ci] * z[rj * W + cj] for (ri, ci), (rj, cj) in inputs.bonds(L, W)]
    np.testing.assert_allclose(ob.szsz, zz, atol=1e-13)


@pytest.mark.parametrize("L,W,D", [(3, 4, 2), (2, 3, 3)])
def test_product_state_with_bonds_closed_form(L, W, D):
    # the same product state written with bond dimension D (one vector per
    # bond on both ends): each bond adds |v|^4 to the norm, nothing else
    rng = np.random.default_rng(L * 10 + W + D)
    a0 = rng.uniform(-1, 1, L * W)
    a1 = rng.uniform(-1, 1, L * W)
    A, hv, vv = inputs.product_lattice_bonds(L, W, D, a0, a1, 77, with_bonds=True)
    ob = oracle.observables(L, W, D, A)
    q = a0 ** 2 + a1 ** 2
    log2n = np.sum(np.log2(q)) + 2 * (np.sum(np.log2(np.sum(hv ** 2, -1))) + np.sum(np.log2(np.sum(vv ** 2, -1))))
    assert abs(ob.log2_norm - log2n) < 1e-12 * max(1.0, abs(log2n))
    np.testing.assert_allclose(ob.sx, 2 * a0 * a1 / q, atol=1e-13)
    z = (a1 ** 2 - a0 ** 2) / q
    zz = [z[ri * W + ci] * z[rj * W + cj] for (ri, ci), (rj, cj) in inputs.bonds(L, W)]
    np.testing.assert_allclose(ob.szsz, zz, atol=1e-13)


# --------------------------------------- all-ones workload of Sec. 6 (exact)

@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (5, 5, 2), (6, 6, 2), (8, 8, 2), (3, 7, 2)])
def test_all_ones_exact_power_of_two(L, W, D):
    """norm = 2^N D^(2 nb), <X> = 1, <ZZ> = 0, E = -h N: exact for D = 2."""
    A = inputs.ones_lattice(L, W, D)
    ob = oracle.observables(L, W, D, A)
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    exact_log2 = N + 2 * nb * math.log2(D)
    assert ob.norm_m == 0.5 and ob.norm_e == int(exact_log2) + 1
    assert np.all(ob.sx == 1.0)
    assert np.all(ob.szsz == 0.0)
    assert ob.energy(1.0, 3.04) == -3.04 * N


@pytest.mark.parametrize("L,W,D", [(4, 4, 3), (3, 5, 3), (2, 2, 4)])
def test_all_ones_odd_bond(L, W, D):
    A = inputs.ones_lattice(L, W, D)
    ob = oracle.observables(L, W, D, A)
    N, nb = L * W, L * (W - 1) + W * (L - 1)
    assert abs(ob.log2_norm - (N + 2 * nb * math.log2(D))) < 1e-12 * (N + 2 * nb * 2)
    np.testing.assert_allclose(ob.sx, 1.0, atol=1e-13)
    np.testing.assert_allclose(ob.szsz, 0.0, atol=1e-13)


# ------------------------------------------ classical Ising as a TN (bond 2)

def _ising_grid(L, W, K):
    """Single-layer tensors T[u][l][dn][rt] = sum_s prod_legs Q[s, leg], W = Q Q^T,
    w(s, s') = exp(K s s'); edge legs are left out (dimension 1)."""
    a, b = math.exp(K), math.exp(-K)
    Q = np.array([[math.sqrt((a + b) / 2), math.sqrt((a - b) / 2)],
                  [math.sqrt((a + b) / 2), -math.sqrt((a - b) / 2)]])
    dims, ts = [], []
    for r in range(L):
        for c in range(W):
            d = inputs.site_dims(L, W, 2, r, c)
            T = np.zeros(d)
            for s in range(2):
                vs = [Q[s, :k] if k > 1 else np.ones(1) for k in d]
                T += np.einsum("a,b,c,d->abcd", *vs)
            dims.append(d)
            ts.append(T)
    return np.array(dims), ts


def test_ising_enumeration_closed_forms():
    """The enumeration itself against textbook closed forms."""
    for K in (0.0, 0.4, 1.1):
        lz, _, _ = oracle.ising_enumerate(1, 6, K)
        assert abs(lz - (math.log(2) + 5 * math.log(2 * math.cosh(K)))) < 1e-12
        lz, _, _ = oracle.ising_enumerate(2, 2, K)
        ring = (2 * math.cosh(K)) ** 4 + (2 * math.sinh(K)) ** 4
        assert abs(lz - math.log(ring)) < 1e-12
    lz, corr, xf = oracle.ising_enumerate(3, 4, 0.0)
    assert abs(lz - 12 * math.log(2)) < 1e-12
    assert np.allclose(corr, 0.0) and np.allclose(xf, 1.0)
    # 1D chain: <s_i s_{i+1}> = tanh K
    _, corr, _ = oracle.ising_enumerate(1, 5, 0.7)
    np.testing.assert_allclose(corr, math.tanh(0.7), atol=1e-12)


@pytest.mark.parametrize("L,W", [(1, 6), (2, 2), (3, 3), (4, 4), (3, 5), (5, 5)])
@pytest.mark.parametrize("K", [0.0, 0.3, 0.9])
def test_single_layer_grid_is_ising_partition_function(L, W, K):
    dims, ts = _ising_grid(L, W, K)
    m, e = oracle.grid_contract(L, W, dims, ts)
    logz_tn = math.log(m) + e * math.log(2)
    logz, _, _ = oracle.ising_enumerate(L, W, K)
    assert abs(logz_tn - logz) < 1e-11 * max(1.0, abs(logz))


@pytest.mark.parametrize("L,W", [(2, 3), (3, 3), (4, 4), (4, 5)])
@pytest.mark.parametrize("K", [0.2, 0.6])
def test_ising_peps_double_layer(L, W, K):
    """psi(s) = prod exp(K s s'/2): norm = Z(K), <zz> classical, <x> = <exp(-K s_k h_k)>."""
    A = inputs.ising_peps_lattice(L, W, K)
    ob = oracle.observables(L, W, 2, A)
    logz, corr, xf = oracle.ising_enumerate(L, W, K)
    assert abs(ob.log2_norm * math.log(2) - logz) < 1e-11 * max(1.0, logz)
    np.testing.assert_allclose(ob.szsz, corr, atol=1e-12)
    np.testing.assert_allclose(ob.sx, xf, atol=1e-12)


def test_ising_peps_padded_to_d3():
    """The same state with every bond padded by a zero channel (D = 3)."""
    L, W, K = 3, 4, 0.5
    A2 = inputs.split_sites(inputs.ising_peps_lattice(L, W, K), L, W, 2)
    sites = []
    for r in range(L):
        for c in range(W):
            d3 = inputs.site_dims(L, W, 3, r, c)
            B = np.zeros((2,) + d3)
            a = A2[r * W + c]
            B[:, :a.shape[1], :a.shape[2], :a.shape[3], :a.shape[4]] = a
            sites.append(B)
    A3 = inputs.join_sites(sites)
    ob3 = oracle.observables(L, W, 3, A3)
    ob2 = oracle.observables(L, W, 2, inputs.join_sites(A2))
    assert abs(ob3.log2_norm - ob2.log2_norm) < 1e-12 * abs(ob2.log2_norm)
    np.testing.assert_allclose(ob3.sx, ob2.sx, atol=1e-13)
    np.testing.assert_allclose(ob3.szsz, ob2.szsz, atol=1e-13)


# ------------------------------------------------------------- invariances

def _transpose_lattice(A, L, W, D):
    """Site (r, c) -> (c, r) with legs u<->l, dn<->rt: the same network."""
    sites = inputs.split_sites(A, L, W, D)
    out = []
    for r in range(W):          # new lattice is W x L
        for c in range(L):
            out.append(np.transpose(sites[c * W + r], (0, 2, 1, 4, 3)))
    return inputs.join_sites(out)


def _flip_lattice(A, L, W, D):
    """Upside down: site (r, c) -> (L-1-r, c), legs u <-> dn."""
    sites = inputs.split_sites(A, L, W, D)
    out = []
    for r in range(L):
        for c in range(W):
            out.append(np.transpose(sites[(L - 1 - r) * W + c], (0, 3, 2, 1, 4)))
    return inputs.join_sites(out)


@pytest.mark.parametrize("L,W,D", [(3, 5, 2), (4, 4, 2), (3, 3, 3)])
def test_order_invariance(L, W, D):
    A = inputs.random_lattice(L, W, D, 555 + L + W)
    m, e = oracle.norm_all_cuts(L, W, D, A)
    ref = math.log2(abs(m[0])) + e[0]
    for r in range(L + 1):
        assert m[r] > 0
        assert abs(math.log2(abs(m[r])) + e[r] - ref) < 1e-12 * max(1, abs(ref))
    ob = oracle.observables(L, W, D, A)
    obt = oracle.observables(W, L, D, _transpose_lattice(A, L, W, D))
    assert abs(obt.log2_norm - ob.log2_norm) < 1e-12 * max(1, abs(ref))
    sx_t = obt.sx.reshape(W, L).T.ravel()
    np.testing.assert_allclose(sx_t, ob.sx, atol=1e-12)
    # transposed bonds: same set of values
    np.testing.assert_allclose(np.sort(obt.szsz), np.sort(ob.szsz), atol=1e-12)
    obf = oracle.observables(L, W, D, _flip_lattice(A, L, W, D))
    np.testing.assert_allclose(obf.sx.reshape(L, W)[::-1].ravel(), ob.sx, atol=1e-12)
    nm, ne = oracle.norm(L, W, D, A)
    assert abs(math.log2(nm) + ne - ref) < 1e-12 * max(1, abs(ref))


def test_gauge_invariance():
    """Insert G G^-1 on bonds: the network, hence every observable, is unchanged."""
    L, W, D = 3, 4, 2
    A = inputs.random_lattice(L, W, D, 9)
    sites = [s.copy() for s in inputs.split_sites(A, L, W, D)]
    rng = np.random.default_rng(3)
    for r in range(L):
        for c in range(W - 1):      # horizontal bond (r,c)-(r,c+1): rt of left, l of right
            G = rng.normal(size=(D, D)) + 3 * np.eye(D)
            Gi = np.linalg.inv(G)
            sites[r * W + c] = np.einsum("pulde,ef->puldf", sites[r * W + c], G)
            sites[r * W + c + 1] = np.einsum("fe,puedr->pufdr", Gi, sites[r * W + c + 1])
    for r in range(L - 1):
        for c in range(W):          # vertical bond: dn of upper, u of lower
            G = rng.normal(size=(D, D)) + 3 * np.eye(D)
            Gi = np.linalg.inv(G)
            sites[r * W + c] = np.einsum("pulde,df->pulfe", sites[r * W + c], G)
            sites[(r + 1) * W + c] = np.einsum("fu,puldr->pfldr", Gi, sites[(r + 1) * W + c])
    B = inputs.join_sites(sites)
    a, b = oracle.observables(L, W, D, A), oracle.observables(L, W, D, B)
    assert abs(a.log2_norm - b.log2_norm) < 1e-10
    np.testing.assert_allclose(b.sx, a.sx, atol=1e-10)
    np.testing.assert_allclose(b.szsz, a.szsz, atol=1e-10)


def test_scale_invariance():
    L, W, D, lam = 3, 3, 2, 3.75
    A = inputs.random_lattice(L, W, D, 11)
    sites = [s.copy() for s in inputs.split_sites(A, L, W, D)]
    sites[4] *= lam
    B = inputs.join_sites(sites)
    a, b = oracle.observables(L, W, D, A), oracle.observables(L, W, D, B)
    assert abs(b.log2_norm - a.log2_norm - 2 * math.log2(lam)) < 1e-12
    np.testing.assert_allclose(b.sx, a.sx, atol=1e-13)
    np.testing.assert_allclose(b.szsz, a.szsz, atol=1e-13)


def test_expect_one_matches_cached():
    L, W, D = 4, 5, 2
    A = inputs.random_lattice(L, W, D, 31)
    ob = oracle.observables(L, W, D, A)
    for k in (0, 7, 19):
        v, _, _ = oracle.expect_one(L, W, D, A, "x", k)
        assert abs(v - ob.sx[k]) < 1e-12
    for bi, ((ri, ci), (rj, cj)) in enumerate(inputs.bonds(L, W)):
        if bi % 5:
            continue
        v, _, _ = oracle.expect_one(L, W, D, A, "zz", ri * W + ci, rj * W + cj)
        assert abs(v - ob.szsz[bi]) < 1e-12


# ------------------------------------------------------ counts and planner

def test_paper_counts():
    with open(os.path.join(GOLD, "paper_counts.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        L = case["L"]
        assert len(inputs.bonds(L, L)) == case["bonds"] == 2 * L * (L - 1)
        assert L * L == case["sites"]


def _recount(L, W, D, o, i, j):
    """Brute-force leg bookkeeping: keep the boundary as a list of named legs and
    apply the pairwise-contraction size rule of Sec. 4 -- shared legs vanish,
    the rest survive -- with no formula for P, K, N, S."""
    d = D * D
    Lp, Wp = (L, W) if o == 0 else (W, L)

    def leg_dim(name):
        kind, a, b = name
        if kind == "h":  # horizontal bond between (a, b) and (a, b+1)
            return d if 0 <= b < Wp - 1 else 1
        return d if 0 <= a < Lp - 1 else 1   # vertical bond between (a, b), (a+1, b)

    out = []
    for q in range(4):
        rows = range(0, i) if q in (0, 1) else range(Lp - 1, i - 1, -1)
        cols = range(0, j) if q in (0, 2) else range(Wp - 1, j - 1, -1)
        rows, cols = list(rows), list(cols)
        if not rows or not cols:
            continue
        bnd = []    # ordered boundary legs
        for k, r in enumerate(rows):
            for c_i, c in enumerate(cols):
                up = ("v", r - 1, c) if q in (0, 1) else ("v", r, c)
                dn = ("v", r, c) if q in (0, 1) else ("v", r - 1, c)
                lf = ("h", r, c - 1) if q in (0, 2) else ("h", r, c)
                rt = ("h", r, c) if q in (0, 2) else ("h", r, c - 1)
                site = [up, lf, dn, rt]
                if c_i == 0:
                    bnd.insert(0, lf)      # dimension-1 entering leg (lattice edge)
                if k == 0:
                    bnd.insert(c_i + 1, up)
                n_in = math.prod(leg_dim(x) for x in bnd)
                shared = [x for x in bnd if x in site]
                pos = bnd.index(shared[0])
                bnd = [x for x in bnd if x not in site]
                bnd[pos:pos] = [dn, rt]
                n_site = math.prod(leg_dim(x) for x in site)
                n_shared = math.prod(leg_dim(x) for x in shared)
                n_out = math.prod(leg_dim(x) for x in bnd)
                assert n_out == n_in * n_site // (n_shared * n_shared)
                out.append((n_in, n_out))
            # the row's last rt leg stays in place; the next row's entering h is new
    return out


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (5, 3, 2), (6, 6, 3), (3, 7, 2), (7, 5, 2)])
def test_planner_sizes_match_leg_recount(L, W, D):
    for (o, i, j) in [(0, L, W), (1, W, L), (0, (L + 1) // 2, (W + 1) // 2), (0, 0, 0), (1, 2, 1),
                      (0, 1, W - 1)]:
        ev = planner.evaluate(L, W, D, o, i, j)
        rec = _recount(L, W, D, o, i, j)
        assert [(s["n_in"], s["n_out"]) for s in ev["steps"]] == rec


def test_planner_scheme_sizes_from_paper():
    with open(os.path.join(GOLD, "scheme_sizes.json")) as f:
        g = json.load(f)
    for case in g["cases"]:
        L, D = case["L"], case["D"]
        row = planner.evaluate(L, L, D, 0, L, L)
        # the boundary after the first L/2 rows: output of the last site of that row
        per_row = [s for s in row["steps"] if s["k"] == L // 2 - 1]
        assert per_row[-1]["n_out"] == case["row_boundary"]
        q = planner.evaluate(L, L, D, 0, L // 2, L // 2)
        tl = [s for s in q["steps"] if s["corner"] == 0][-1]["n_out"]
        assert tl == case["ring_leg_group"] ** 2      # two leg groups per ring tensor
        assert q["peak"] == case["ring_leg_group"] ** 2
        assert row["peak"] == case["row_boundary"] * D * D   # one extra leg mid-row


def test_planner_auto_prefers_quadrant_on_squares():
    for L, D in [(4, 2), (8, 2), (12, 2), (8, 3), (6, 3)]:
        p = planner.plan(L, L, D)
        assert (p["o"], p["i"], p["j"]) == (0, L // 2, L // 2)
        assert p["peak"] == (D * D) ** L
    p = planner.plan(4, 10, 2)
    assert p["peak"] == 4 ** 5       # thin lattices: sweep along the long side


@pytest.mark.parametrize("L,W,D", [(4, 4, 2), (5, 3, 2), (3, 6, 3), (12, 12, 2), (8, 8, 3)])
def test_sweep_macs_equal_row_scheme_macs(L, W, D):
    """The multiply-adds the bench's CPU sample scales by: a full row sweep
    counted site by site (oracle.sweep_macs) equals the summed multiply-adds
    of the oracle planner's row-scheme chain (Fig. 2a, cut (L, W)), counted
    from its own leg bookkeeping; a partial sweep lies strictly between."""
    import oracle.planner as planner
    full = oracle.sweep_macs(L, W, D, L)
    assert full == sum(st["mac"] for st in planner.evaluate(L, W, D, 0, L, W)["steps"])
    part = oracle.sweep_macs(L, W, D, 1, 2)
    assert oracle.sweep_macs(L, W, D, 1) < part < full


def test_sweep_rows_sample_matches_norm():
    """A full sweep by sweep_rows is the norm; a partial one runs and returns."""
    L, W, D = 4, 5, 2
    A = inputs.random_lattice(L, W, D, 31)
    assert oracle.sweep_rows(L, W, D, A, L) == oracle.norm(L, W, D, A)
    oracle.sweep_rows(L, W, D, A, 2, 3)
    with pytest.raises(ValueError):
        oracle.sweep_rows(L, W, D, A, L, 1)
