"""Conductivity profiles at the quadrature points (Sec. IV, Eq. 23).

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
