"""Planted mistakes in the oracle must be caught by its pins.

Each case copies ``oracle/tn_oracle.c``, applies one plausible mistake (a
dropped term, a swapped index, a transposed operand, a wrong sign), compiles
the copy on the CPU and checks that comparing it with the brute-force state
vector or a closed form now fails.  Nothing here touches the GPU.
"""
import ctypes
import os
import subprocess

import numpy as np
import pytest

import oracle
import oracle.brute as brute
from paper_1908_08553_gb300 import inputs

SRC = os.path.join(os.path.dirname(oracle.__file__), "tn_oracle.c")

MUTATIONS = {
    # operator X loses one off-diagonal entry
    "dropped_x_term": ("static const double OP_X[4] = {0, 1, 1, 0};",
                       "static const double OP_X[4] = {0, 1, 0, 0};"),
    # the second copy reads the first copy's physical index (q term dropped).
    # (Swapping the two copies' digits on every l leg is NOT a mistake: it
    # equals relabelling the copies on odd columns, a symmetry of the double
    # layer when the inserted operator is symmetric, so it is not listed.)
    "second_copy_physical_index": ("A[(((size_t)(q * Du + ub) * Dl + lb) * Dd + db) * Dr + rb]",
                                   "A[(((size_t)(p * Du + ub) * Dl + lb) * Dd + db) * Dr + rb]"),
    # site tensor read with h and u exchanged
    "transposed_site_index": ("T[((size_t)(u * Dh + h) * Ddn + n) * Drt + q]",
                              "T[((size_t)(h * Du + u) * Ddn + n) * Drt + q]"),
    # ratio exponent with the wrong sign
    "ratio_exponent_sign": ("ldexp(mo / mn, (int)(eo - en))", "ldexp(mo / mn, (int)(en - eo))"),
    # vertical bond: second Z one column off
    "vertical_bond_column": ("over[c] = ez[(r + 1) * W + c];",
                             "over[c] = ez[(r + 1) * W + (c + 1) % W];"),
    # rescale forgets to record the exponent
    "rescale_exponent_lost": ("b->e += ex;", "(void)ex;"),
}


def _build_mutant(name, tmp_path):
    old, new = MUTATIONS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.or_peps_observables.argtypes = [i32, i32, i32, P, P, P, P, P]
    return lib


def _observables(lib, L, W, D, A):
    nb = L * (W - 1) + W * (L - 1)
    m, e = np.zeros(1), np.zeros(1, np.int64)
    sx, zz = np.zeros(L * W), np.zeros(nb)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    lib.or_peps_observables(L, W, D, p(A), p(m), p(e), p(sx), p(zz))
    return m[0], int(e[0]), sx, zz


def _pins_pass(lib):
    """The state-vector pin and the all-ones pin of the real suite, condensed."""
    L, W, D = 3, 3, 2
    A = inputs.random_lattice(L, W, D, 4242)
    m, e, sx, zz = _observables(lib, L, W, D, A)
    n, bsx, bzz = brute.observables(L, W, D, A)
    ok = abs(m * 2.0 ** e - n) <= 1e-12 * abs(n)
    ok &= np.allclose(sx, bsx, atol=1e-12) and np.allclose(zz, bzz, atol=1e-12)
    A1 = inputs.ones_lattice(4, 4, 2)
    m, e, sx, zz = _observables(lib, 4, 4, 2, A1)
    ok &= (m == 0.5 and e == 16 + 48 + 1 and np.all(sx == 1.0) and np.all(zz == 0.0))
    return bool(ok)


def test_unmutated_oracle_passes(tmp_path):
    lib = oracle.lib()
    assert _pins_pass(lib)


@pytest.mark.parametrize("name", sorted(MUTATIONS))
def test_mutant_is_caught(name, tmp_path):
    lib = _build_mutant(name, tmp_path)
    assert not _pins_pass(lib), f"planted mistake {name} was not caught"


# ---- single-site <Z_k> and two-site correlators (their own pins) ----------

MUTATIONS_Z = {
    # <Z_k> computed with the X site matrix
    "sz_uses_x": ("double *ez = double_layer(A + off[r * W + c], d, OP_Z);",
                  "double *ez = double_layer(A + off[r * W + c], d, OP_X);"),
    # <Z_k> closed with the bottom boundary of the wrong row
    "sz_bottom_row": ("bnd_dot(&b, &bots[r + 1], &m, &e);\n            sz[r * W + c]",
                      "bnd_dot(&b, &bots[r], &m, &e);\n            sz[r * W + c]"),
    # the first operator of a bond ignored (always Z)
    "bond_ignores_op_a": ("const double *oa = op_a == 1 ? OP_X : OP_Z,",
                          "const double *oa = OP_Z,"),
    # vertical bonds: the two operators exchanged between the rows
    "bond_vertical_swapped": ("            over[c] = ea;\n            absorb_row(&g, r, over, &b);\n            over[c] = eb;",
                              "            over[c] = eb;\n            absorb_row(&g, r, over, &b);\n            over[c] = ea;"),
}


def _build_mutant_z(name, tmp_path):
    old, new = MUTATIONS_Z[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not found exactly once"
    path = tmp_path / f"{name}.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / f"{name}.so"
    subprocess.check_call(["gcc", "-O1", "-fopenmp", "-shared", "-fPIC", "-std=c11",
                           "-o", str(so), str(path), "-lm"])
    lib = ctypes.CDLL(str(so))
    P, i32 = ctypes.c_void_p, ctypes.c_int
    lib.or_peps_sz.argtypes = [i32, i32, i32, P, P]
    lib.or_peps_bond_ops.argtypes = [i32, i32, i32, P, i32, i32, P]
    return lib


def _z_pins_pass(lib):
    """The state-vector pins of <Z_k> and of the X-X and X-Z bond correlators."""
    L, W, D = 3, 3, 2
    A = inputs.random_lattice(L, W, D, 4343)
    p = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    sz = np.zeros(L * W)
    lib.or_peps_sz(L, W, D, p(A), p(sz))
    ok = np.allclose(sz, brute.sz(L, W, D, A), atol=1e-12)
    nb = L * (W - 1) + W * (L - 1)
    for a, b, ca, cb in (("x", "x", 1, 1), ("x", "z", 1, 2)):
        out = np.zeros(nb)
        lib.or_peps_bond_ops(L, W, D, p(A), ca, cb, p(out))
        ok &= np.allclose(out, brute.bond_correlators(L, W, D, A, a, b), atol=1e-12)
    return bool(ok)


def test_unmutated_oracle_passes_z_pins():
    assert _z_pins_pass(oracle.lib())


@pytest.mark.parametrize("name", sorted(MUTATIONS_Z))
def test_z_mutant_is_caught(name, tmp_path):
    lib = _build_mutant_z(name, tmp_path)
    assert not _z_pins_pass(lib), f"planted mistake {name} was not caught"
