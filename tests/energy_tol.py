"""Energy tolerances shared by the GPU parity tests.

The bound on E (Eqs. Hamiltonian and Etot) depends on the precision:
  * FP64: relative to E itself, |dE| <= 1e-10 |E|.
  * FP32, BF16x3, BF16x6: relative to the energy's scale
        S = |J| sum_<ij> |<Z_i Z_j>| + |h| sum_k |<X_k>|   (>= |E|),
    |dE| <= 1e-6 S.  E is a sum of terms of both signs: for random states the
    terms can cancel to |E| << S (8x8 D=2, seed lattice_seed(4242, 2), h = 2:
    E = 0.080 with S = 48), and a result stored with a 24-bit significand
    cannot resolve E better than about 2^-24 S.  Where the terms do not cancel
    (S <= 10 |E|) the bound is also checked relative to E itself.
Per-term bounds (<X_k>, <Z_k>, <Z_i Z_j>: O(1) quantities that can be ~0) stay
|d| <= tol * max(1, |value|).
"""
from __future__ import annotations

import numpy as np

FP64, FP32, BF16X3, BF16X6 = 0, 1, 2, 3
REL_E = {FP64: 1e-10, FP32: 1e-6, BF16X3: 1e-6, BF16X6: 1e-6}


def energy_scale(sx, zz, J: float, h: float) -> float:
    return abs(J) * float(np.abs(zz).sum()) + abs(h) * float(np.abs(sx).sum())


def energy_errors(e: float, e_ref: float, sx_ref, zz_ref, J: float, h: float):
    """(|dE| / |E|, |dE| / S, S / |E|)."""
    d = abs(e - e_ref)
    S = energy_scale(sx_ref, zz_ref, J, h)
    return d / abs(e_ref) if e_ref else float("inf"), d / S if S else d, S / abs(e_ref) if e_ref else float("inf")


def check_energy(e: float, e_ref: float, sx_ref, zz_ref, J: float, h: float, prec: int, factor: float = 1.0):
    """Assert the energy bound of `prec` (factor loosens it only where a test says why)."""
    tol = REL_E[prec] * factor
    rel, rel_scale, kappa = energy_errors(e, e_ref, sx_ref, zz_ref, J, h)
    if prec == FP64:
        assert rel <= tol, f"FP64 |dE|/|E| = {rel:.3g} > {tol:g} (E = {e!r}, ref {e_ref!r})"
    else:
        assert rel_scale <= tol, f"|dE|/S = {rel_scale:.3g} > {tol:g} (E = {e!r}, ref {e_ref!r}, S/|E| = {kappa:.3g})"
        if kappa <= 10.0:
            assert rel <= tol, f"|dE|/|E| = {rel:.3g} > {tol:g} with S/|E| = {kappa:.3g}"
    return rel, rel_scale, kappa
