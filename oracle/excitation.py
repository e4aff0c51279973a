"""Incident fields and the tested right-hand side b (Appendix A of the paper).

Time convention exp(+jwt) (Sec. II).  Units: eta0 = 1, so H here is eta0*H.

* Plane wave:  E = e exp(-jk d.r),  H = (d x e)/z exp(-jk d.r).
* Electric current element of unit moment p at r_s in a medium (k, z):
      E = -z L_pt(p),  L_pt(p) = jk [G p + k^-2 grad(grad G . p)],
      H = grad G x p,
  with G = exp(-jkR)/(4 pi R).  With G' = -(jk + 1/R) G and
  G'' = ((jk + 1/R)^2 + 1/R^2) G:
      grad(grad G . p) = G'' (Rh.p) Rh + (G'/R) (p - (Rh.p) Rh).
* Complex-source-point beam (Sec. II, ref. erez94): the same element placed at
  r_s = r0 - j b d (complex position), R = sqrt((r - r_s).(r - r_s)) on the
  branch Re R >= 0; it radiates a Gaussian beam along +d with waist
  sqrt(2b/k) at r0.

Right-hand side rows (row types as in ``mesh.row_index``; Eq. 13 tested as
in ``operator``).  Interior incidence (the paper's case, Eqs. 8-9):
[<X,E_inc>, <X,H_inc>, <X,H_inc>, <sigma X, E_inc>].  Exterior incidence
(mirror of Eqs. 6-7, used for the sphere):
[-<X,E_inc>, -<X,H_inc>, -<X,H_inc> + <sigma (n x X), E_inc>, 0].
"""

from __future__ import annotations

import numpy as np

from .mesh import Geometry, row_index
from .operator import sigma_normalised


def plane_wave(r, k, z, d, e):
    d = np.asarray(d, dtype=np.float64)
    e = np.asarray(e, dtype=np.complex128)
    ph = np.exp(-1j * k * (r @ d))
    E = ph[..., None] * e
    H = ph[..., None] * (np.cross(d, e) / z)
    return E, H


def dipole(r, k, z, rs, p):
    """Fields of a unit electric current element; ``rs`` may be complex."""
    rs = np.asarray(rs, dtype=np.complex128)
    p = np.asarray(p, dtype=np.complex128)
    D = r.astype(np.complex128) - rs
    R = np.sqrt(np.sum(D * D, axis=-1))
    Rh = D / R[..., None]
    G = np.exp(-1j * k * R) / (4 * np.pi * R)
    G1 = -(1j * k + 1.0 / R) * G
    G2 = ((1j * k + 1.0 / R) ** 2 + 1.0 / R**2) * G
    rp = Rh @ p
    hess_p = (G2 * rp)[..., None] * Rh + (G1 / R)[..., None] * (p - rp[..., None] * Rh)
    Lpt = 1j * k * (G[..., None] * p + hess_p / k**2)
    E = -z * Lpt
    H = np.cross(G1[..., None] * Rh, p)
    return E, H


def beam(r, k, z, r0, d, b, p):
    r0 = np.asarray(r0, dtype=np.float64)
    d = np.asarray(d, dtype=np.float64)
    return dipole(r, k, z, r0 - 1j * b * d, p)


def incident(kind, r, k, z, **kw):
    if kind == "planewave":
        return plane_wave(r, k, z, kw["d"], kw["e"])
    if kind == "dipole":
        return dipole(r, k, z, kw["rs"], kw["p"])
    if kind == "beam":
        return beam(r, k, z, kw["r0"], kw["d"], kw["b"], kw["p"])
    raise ValueError(kind)


def rhs(g: Geometry, media, sigma_pts_S, side: str, kind: str, **kw):
    """Tested incident field b for one excitation (vector of length N)."""
    (ke, ki), (ze, zi) = media.k, media.z
    k, z = (ki, zi) if side == "i" else (ke, ze)
    r = g.qpts  # (nt, q, 3)
    E, H = incident(kind, r.reshape(-1, 3), k, z, **kw)
    E = E.reshape(g.nt, g.q, 3)
    H = H.reshape(g.nt, g.q, 3)
    sig = sigma_normalised(sigma_pts_S)
    n = g.normal
    cX = g.tri_sign * g.edge_len[g.tri_edge] / (2.0 * g.area[:, None])
    X = cX[:, :, None, None] * (r[:, None, :, :] - g.V[g.T][:, :, None, :])  # (nt, k, q, 3)
    w = g.qw
    tE = np.einsum("tkqx,tq,tqx->tk", X, w, E)
    tH = np.einsum("tkqx,tq,tqx->tk", X, w, H)
    nX = np.cross(n[:, None, None, :], X)
    tnsE = np.einsum("tkqx,tq,tqx->tk", nX, w * sig, E)
    tsE = np.einsum("tkqx,tq,tqx->tk", X, w * sig, E)
    if side == "i":
        val = np.stack([tE, tH, tH, tsE], axis=-1)
    else:
        val = np.stack([-tE, -tH, -tH + tnsE, np.zeros_like(tE)], axis=-1)
    b = np.zeros(g.N, dtype=np.complex128)
    rows = row_index(g)[g.tri_edge]  # (nt, 3, 4)
    m = rows >= 0
    np.add.at(b, rows[m], val[m])
    return b
