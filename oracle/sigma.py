"""Conductivity profiles at the quadrature points (Sec. IV, Eq. 23).

Test infrastructure: only the tests, the smoke check and the benchmark
baselines use this module.

The absorber conductivity is sigma0 * u((x - x0)/L) with the monomial
u(s) = s^d on 0 <= s <= 1 and 0 for s < 0 (Eq. 23).  A profile here is a sum
of such segments, each with an axis and a direction (+1: grows with x,
-1: grows towards smaller x, for an absorber at the left end); beyond s = 1
the segment stays at sigma0 (u = 1).
"""

from __future__ import annotations

import numpy as np


def monomial(points, segments):
    """sigma [S] at points (..., 3) for segments [(x0, L, sigma0, d, axis, dir), ...]."""
    pts = np.asarray(points, dtype=np.float64)
    sig = np.zeros(pts.shape[:-1])
    for x0, L, s0, d, axis, sgn in segments:
        s = sgn * (pts[..., int(axis)] - x0) / L
        u = np.minimum(s, 1.0)
        val = np.where(s < 0.0, 0.0, s0 * np.power(np.maximum(u, 0.0), d))
        sig = sig + val
    return sig


def bspline_knots(ncoef: int, degree: int = 3):
    """Clamped uniform knot vector on [0, 1] for ncoef coefficients."""
    if ncoef < degree + 1:
        raise ValueError("need at least degree + 1 coefficients")
    inner = np.linspace(0.0, 1.0, ncoef - degree + 1)
    return np.concatenate([np.zeros(degree), inner, np.ones(degree)])


def bspline_basis(s, knots, k, degree):
    """N_{k,degree}(s) by the Cox-de Boor recursion (0/0 taken as 0); the
    last non-empty knot interval is closed on the right so that s = 1
    belongs to it."""
    s = np.asarray(s, dtype=np.float64)
    if degree == 0:
        lo, hi = knots[k], knots[k + 1]
        last = hi == knots[-1] and lo < hi
        inside = (s >= lo) & ((s < hi) | (last & (s == hi)))
        return inside.astype(np.float64)
    out = np.zeros_like(s)
    d1 = knots[k + degree] - knots[k]
    if d1 > 0:
        out = out + (s - knots[k]) / d1 * bspline_basis(s, knots, k, degree - 1)
    d2 = knots[k + degree + 1] - knots[k + 1]
    if d2 > 0:
        out = out + (knots[k + degree + 1] - s) / d2 * bspline_basis(s, knots, k + 1, degree - 1)
    return out


def bspline(points, x0, L, coef, axis=0):
    """sigma [S] at points (..., 3): sum_k coef[k] N_{k,3}(s), s = (x_axis - x0) / L,
    cubic B-splines on clamped uniform knots over s in [0, 1]; zero outside."""
    pts = np.asarray(points, dtype=np.float64)
    coef = np.asarray(coef, dtype=np.float64)
    knots = bspline_knots(len(coef), 3)
    s = (pts[..., int(axis)] - x0) / L
    sig = np.zeros(pts.shape[:-1])
    for k, c in enumerate(coef):
        sig = sig + c * bspline_basis(s, knots, k, 3)
    return np.where((s < 0.0) | (s > 1.0), 0.0, sig)
