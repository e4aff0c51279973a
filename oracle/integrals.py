"""Potential integrals of a flat source triangle at an observation point.

The paper evaluates the MPIE operators (Eqs. 15-16, with G = exp(-jkR)/(4 pi R))
by panel quadrature; it is silent on the singular and near-singular panel
integrals.  This module uses singularity extraction:

    G = 1/(4 pi R) + g_s(R)/(4 pi),     g_s(R) = (exp(-jkR) - 1)/R,

with the static 1/R part integrated in closed form over the source triangle
(the line-integral formulas for flat triangles of Wilton et al. 1984 and
Graglia 1993, restated here from the divergence theorem) and the bounded
remainder g_s by the triangle's own quadrature rule.

For an observation point r and a source triangle S with centroid c the module
returns the three "potential moments" used everywhere downstream:

    P0 = int_S G dS'              (scalar)
    P1 = int_S G (r' - c) dS'     (vector)
    Q  = int_S grad_r G dS'       (vector)

When r lies on S itself the normal distance is set to zero (principal value of
the normal derivative) and the source point that coincides with r contributes
the R -> 0 limits of g_s (value -jk, gradient 0).
"""

from __future__ import annotations

import numpy as np


def _dot(a, b):
    return np.sum(a * b, axis=-1)


def static_triangle(r, v0, v1, v2, self_mask):
    """Closed-form integrals of 1/R over the flat triangle (v0, v1, v2).

    Returns (I, Irho, gradI) with
      I     = int 1/R dS',
      Irho  = int (rho' - rho)/R dS'   (rho = projection of r onto the plane),
      gradI = int grad_r (1/R) dS'.
    All arguments broadcast; ``self_mask`` forces the normal distance to 0.
    """
    n = np.cross(v1 - v0, v2 - v0)
    n = n / np.linalg.norm(n, axis=-1, keepdims=True)
    d = _dot(r - v0, n)
    d = np.where(self_mask, 0.0, d)
    rho = r - d[..., None] * n
    ad = np.abs(d)
    I = np.zeros(np.broadcast(d, d).shape)
    Irho = np.zeros(I.shape + (3,))
    grad = np.zeros(I.shape + (3,))
    omega = np.zeros(I.shape)
    for a, b in ((v0, v1), (v1, v2), (v2, v0)):
        lv = b - a
        lh = lv / np.linalg.norm(lv, axis=-1, keepdims=True)
        uh = np.cross(lh, n)  # outward in-plane normal of this edge
        sm = _dot(a - rho, lh)
        sp = _dot(b - rho, lh)
        t = _dot(a - rho, uh)
        r0sq = t * t + d * d
        Rm = np.sqrt(r0sq + sm * sm)
        Rp = np.sqrt(r0sq + sp * sp)
        with np.errstate(divide="ignore", invalid="ignore"):
            f_pos = np.log((Rp + sp) / (Rm + sm))
            f_neg = np.log((Rm - sm) / (Rp - sp))
        f = np.where(sp + sm > 0, f_pos, f_neg)
        beta = np.arctan2(t * sp, r0sq + ad * Rp) - np.arctan2(t * sm, r0sq + ad * Rm)
        I = I + t * f - ad * beta
        Irho = Irho + 0.5 * uh * (r0sq * f + sp * Rp - sm * Rm)[..., None]
        grad = grad - uh * f[..., None]
        omega = omega + beta
    grad = grad - n * (np.sign(d) * omega)[..., None]
    return I, Irho, grad, rho


def gs_value(R, k):
    """(exp(-jkR) - 1)/R, written to avoid cancellation at small kR."""
    kr = k * R
    return (-2.0 * np.sin(kr / 2) ** 2 - 1j * np.sin(kr)) / R


def gs_deriv(R, k):
    """d/dR of (exp(-jkR) - 1)/R = (1 - exp(-jkR)(1 + jkR))/R^2."""
    kr = k * R
    s, c = np.sin(kr), np.cos(kr)
    return (2.0 * np.sin(kr / 2) ** 2 - kr * s + 1j * (s - kr * c)) / (R * R)


def point_triangle(r, tri_v, cen, spts, sw, k, self_mask, self_idx):
    """Potential moments (P0, P1, Q) of source triangles at observation points.

    r        (..., 3)      observation points
    tri_v    (..., 3, 3)   source triangle vertices
    cen      (..., 3)      source centroids (P1 is taken about these)
    spts     (..., q, 3)   source quadrature points
    sw       (..., q)      source quadrature weights (including the area)
    k        wavenumber (real)
    self_mask (...)        True where r lies on the source triangle
    self_idx  (...)        index of the source point equal to r (or -1)
    """
    v0, v1, v2 = tri_v[..., 0, :], tri_v[..., 1, :], tri_v[..., 2, :]
    I, Irho, gI, rho = static_triangle(r, v0, v1, v2, self_mask)
    diff = r[..., None, :] - spts  # (..., q, 3)
    R = np.linalg.norm(diff, axis=-1)
    q = spts.shape[-2]
    coincide = (np.asarray(self_idx)[..., None] == np.arange(q)) & np.asarray(self_mask)[..., None]
    Rs = np.where(coincide, 1.0, R)
    gv = np.where(coincide, -1j * k, gs_value(Rs, k))
    gd = np.where(coincide, 0.0, gs_deriv(Rs, k) / Rs)
    P0s = np.sum(sw * gv, axis=-1)
    P1s = np.sum((sw * gv)[..., None] * (spts - cen[..., None, :]), axis=-2)
    Qs = np.sum((sw * gd)[..., None] * diff, axis=-2)
    inv4pi = 1.0 / (4.0 * np.pi)
    P0 = (I + P0s) * inv4pi
    P1 = (Irho + (rho - cen) * I[..., None] + P1s) * inv4pi
    Q = (gI + Qs) * inv4pi
    return P0, P1, Q
