"""Post-processing: SWR to r, fields off the surface, axis fit, far field.

* Standing-wave ratio to reflection (Sec. I, Table 1): r = (SWR-1)/(SWR+1),
  with SWR = max|E| / min|E| along the guide axis in the standing-wave region.
* Field at off-surface points from the interior currents (Sec. II, Eq. 8):
  inside the guide the total field is E_inc + E_i(J_i, M_i), evaluated by the
  triangle quadrature rule with the point-source Green's function.
* Axis fit (reading of the paper's SWR measure): least squares for
  E(x_k) = a exp(-j beta x_k) + c exp(+j beta x_k); r = c/a, with beta fixed
  or scanned to minimise the residual.
* Decay-rate fit (Sec. III): the field inside a guide with uniform surface
  conductivity decays along the axis; least squares for
  E(t) = a exp(-g tau) + c exp(g tau), g = alpha + j beta, tau = t - tm (tm the
  midpoint of the samples), both waves decaying along their direction of
  travel, over a grid of (alpha, beta) candidates.
* Decay rate by Poynting's theorem (Sec. III-B): for a guide along x, the
  loss per unit length (the sheet's Joule loss around the perimeter plus the
  power leaving the cross-section's outer boundary) over twice the power
  flowing through the cross-section.
* Far field of the exterior currents, exp(+jwt):
  E ~ F exp(-jkr)/r,  F = -jk/(4 pi) [z (J^ - r (r.J^)) - r x M^],
  J^ = int J exp(jk r.r') dS'.
"""

from __future__ import annotations

import numpy as np

from . import ETA0
from .mesh import Geometry
from .operator import current_sets


def swr_to_r(swr):
    swr = np.asarray(swr, dtype=np.float64)
    return (swr - 1.0) / (swr + 1.0)


def _point_currents(g: Geometry, summ):
    a, beta = summ
    rel = g.qpts - g.centroid[:, None, :]
    J = rel[..., None] * a[:, None, None, :] - beta[:, None, :, :]  # (nt, q, 3, B)
    rho = 2.0 * np.broadcast_to(a[:, None, :], (g.nt, g.q, a.shape[-1]))
    return J, rho


def radiated(g: Geometry, x, pts, k, z, side: str):
    """E of the ``side`` ('i' or 'e') current set radiating in (k, z) at pts (P,3)."""
    x = np.asarray(x, dtype=np.complex128)
    X2 = x[:, None] if x.ndim == 1 else x
    Jes, Jis, Ms = current_sets(g, X2)
    if side == "i":
        Js, Mss = Jis, (-Ms[0], -Ms[1])
    else:
        Js, Mss = Jes, Ms
    J, rhoJ = _point_currents(g, Js)
    M, _ = _point_currents(g, Mss)
    src = g.qpts.reshape(-1, 3)
    w = g.qw.reshape(-1)
    J = J.reshape(-1, 3, J.shape[-1]) * w[:, None, None]
    M = M.reshape(-1, 3, M.shape[-1]) * w[:, None, None]
    rhoJ = rhoJ.reshape(-1, rhoJ.shape[-1]) * w[:, None]
    out = []
    for p in pts:
        D = p - src
        R = np.linalg.norm(D, axis=1)
        G = np.exp(-1j * k * R) / (4 * np.pi * R)
        gG = (-(1j * k + 1.0 / R) * G / R)[:, None] * D  # grad_r G
        A = np.einsum("s,sib->ib", G, J)
        gphi = np.einsum("si,sb->ib", gG, rhoJ)
        curlF = np.einsum("ijk,sj,skb->ib", _EPS, gG, M)
        out.append(-z * (1j * k * A + (1j / k) * gphi) - curlF)
    E = np.array(out)
    return E[..., 0] if x.ndim == 1 else E


def radiated_fields(g: Geometry, x, pts, k, z, side: str):
    """(E, H) of the ``side`` current set radiating in (k, z) at pts (P,3), x one column.

    E = -Z L(J) + K(M) and H = -K(J) - L(M)/Z (Eqs. 15-16), with L(X) = jk A_X + (j/k) grad phi_X
    and K(X) = -curl A_X, A_X = int G X, phi_X = int G div X (fields in the eta0 = 1 scaling)."""
    x = np.asarray(x, dtype=np.complex128)
    Jes, Jis, Ms = current_sets(g, x[:, None])
    if side == "i":
        Js, Mss = Jis, (-Ms[0], -Ms[1])
    else:
        Js, Mss = Jes, Ms
    J, rhoJ = _point_currents(g, Js)
    M, rhoM = _point_currents(g, Mss)
    src = g.qpts.reshape(-1, 3)
    w = g.qw.reshape(-1)
    J = J[..., 0].reshape(-1, 3) * w[:, None]
    M = M[..., 0].reshape(-1, 3) * w[:, None]
    rhoJ = rhoJ[..., 0].reshape(-1) * w
    rhoM = rhoM[..., 0].reshape(-1) * w
    E, H = [], []
    for p in np.atleast_2d(pts):
        D = p - src
        R = np.linalg.norm(D, axis=1)
        G = np.exp(-1j * k * R) / (4 * np.pi * R)
        gG = (-(1j * k + 1.0 / R) * G / R)[:, None] * D  # grad_r G
        AJ, AM = G @ J, G @ M
        gphiJ, gphiM = gG.T @ rhoJ, gG.T @ rhoM
        curlAJ = np.einsum("ijk,sj,sk->i", _EPS, gG, J)
        curlAM = np.einsum("ijk,sj,sk->i", _EPS, gG, M)
        E.append(-z * (1j * k * AJ + (1j / k) * gphiJ) - curlAM)
        H.append(curlAJ - (1j * k * AM + (1j / k) * gphiM) / z)
    return np.array(E), np.array(H)


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0


def fit_reflection(xs, E, beta=None, betas=None):
    """Least-squares split of samples E(x) into forward and backward waves.

    Returns (r = c/a, beta, residual).  If ``beta`` is None, it is scanned
    over ``betas`` (1-D array) for the smallest residual.
    """
    xs = np.asarray(xs, dtype=np.float64)
    E = np.asarray(E, dtype=np.complex128)

    def solve(bt):
        Mx = np.stack([np.exp(-1j * bt * xs), np.exp(1j * bt * xs)], axis=1)
        coef, *_ = np.linalg.lstsq(Mx, E, rcond=None)
        res = np.linalg.norm(Mx @ coef - E) / np.linalg.norm(E)
        return coef, res

    if beta is None:
        best = None
        for bt in betas:
            coef, res = solve(bt)
            if best is None or res < best[2]:
                best = (coef, bt, res)
        coef, beta, res = best
    else:
        coef, res = solve(beta)
    return coef[1] / coef[0], beta, res


def fit_decay(ts, E, alphas, betas):
    """Least-squares fit of E(t) = a exp(-g tau) + c exp(g tau), g = alpha + j beta,
    tau = t - (t_first + t_last)/2, scanning every (alpha, beta) of the two 1-D grids.

    Returns (alpha, beta, relative residual, a, c) of the candidate with the smallest
    residual (the first in alpha-major order on a tie)."""
    ts = np.asarray(ts, dtype=np.float64)
    E = np.asarray(E, dtype=np.complex128)
    tau = ts - 0.5 * (ts[0] + ts[-1])
    best = None
    for al in np.atleast_1d(alphas):
        for bt in np.atleast_1d(betas):
            g = al + 1j * bt
            Mx = np.stack([np.exp(-g * tau), np.exp(g * tau)], axis=1)
            coef, *_ = np.linalg.lstsq(Mx, E, rcond=None)
            res = np.linalg.norm(Mx @ coef - E)
            if best is None or res < best[2]:
                best = (float(al), float(bt), res, coef[0], coef[1])
    al, bt, res, a, c = best
    return al, bt, res / np.linalg.norm(E), a, c


def _gl_rect(y0, y1, z0, z1, n):
    u, w = np.polynomial.legendre.leggauss(n)
    ys = 0.5 * (y1 - y0) * u + 0.5 * (y1 + y0)
    zs = 0.5 * (z1 - z0) * u + 0.5 * (z1 + z0)
    Y, Z = np.meshgrid(ys, zs, indexing="ij")
    W = np.outer(w, w) * 0.25 * (y1 - y0) * (z1 - z0)
    return np.stack([Y.ravel(), Z.ravel()], 1), W.ravel()


def poynting_decay_rate(g: Geometry, x, media, sigma_S, xc, core, box, slab, inc=None, n=10):
    """Decay rate of Sec. III-B at the cross-section x = xc of a guide along x.

    alpha = [int_L' sigma |E_tan|^2 dl + Re oint_L (E x H*) . n dl] / [2 Re int_A (E x H*) . x dS]
    with A the rectangle |y| <= box[0], |z| <= box[1] (the core |y| < core[0], |z| < core[1] holds
    the interior field, the rest the exterior field), L its outer boundary and L' the guide's
    perimeter.  The perimeter integral is the surface integral over the band |x - xc| < slab
    divided by its width 2 slab, with |E_tan| = |n x M| = |M|.  ``sigma_S`` is the uniform surface
    conductivity [S]; ``inc(pts)`` returns (E, H) of the interior incident field (or None).
    Returns (alpha, loss per length, side flux per length, cross-section flux)."""
    ke, ki = media.k
    ze, zi = media.z
    hy, hz = core
    Y, Z = box

    def fields(yz, side):
        pts = np.column_stack([np.full(len(yz), xc), yz])
        if side == "i":
            E, H = radiated_fields(g, x, pts, ki, zi, "i")
            if inc is not None:
                Ei, Hi = inc(pts)
                E, H = E + Ei, H + Hi
        else:
            E, H = radiated_fields(g, x, pts, ke, ze, "e")
        return E, H

    def sx(E, H):
        return np.real(E[:, 1] * np.conj(H[:, 2]) - E[:, 2] * np.conj(H[:, 1]))

    yz, w = _gl_rect(-hy, hy, -hz, hz, n)
    flux = np.sum(w * sx(*fields(yz, "i")))
    ys, zs = (-Y, -hy, hy, Y), (-Z, -hz, hz, Z)
    for a in range(3):
        for b in range(3):
            if a == 1 and b == 1:
                continue
            yz, w = _gl_rect(ys[a], ys[a + 1], zs[b], zs[b + 1], n)
            flux += np.sum(w * sx(*fields(yz, "e")))
    u, wu = np.polynomial.legendre.leggauss(2 * n)
    side = 0.0
    for axis, sgn in ((0, 1.0), (0, -1.0), (1, 1.0), (1, -1.0)):
        half = Z if axis == 0 else Y
        line = u * half
        yz = np.column_stack([np.full_like(line, sgn * Y), line]) if axis == 0 else \
            np.column_stack([line, np.full_like(line, sgn * Z)])
        E, H = fields(yz, "e")
        S = np.real(np.cross(E, np.conj(H)))
        side += np.sum(wu * half * sgn * S[:, 1 + axis])
    _, _, Ms = current_sets(g, np.asarray(x, dtype=np.complex128)[:, None])
    M, _ = _point_currents(g, Ms)
    band = np.abs(g.qpts[..., 0] - xc) < slab
    m2 = np.sum(np.abs(M[..., 0]) ** 2, -1)
    loss = (sigma_S * ETA0) * np.sum((g.qw * m2)[band]) / (2.0 * slab)
    return (loss + side) / (2.0 * flux), loss, side, flux


def far_field(g: Geometry, x, k, z, rhat):
    """Far-field pattern F(rhat) of the exterior current set (rhat: (P,3))."""
    x = np.asarray(x, dtype=np.complex128)
    Jes, _, Ms = current_sets(g, x[:, None])
    J, _ = _point_currents(g, Jes)
    M, _ = _point_currents(g, Ms)
    src = g.qpts.reshape(-1, 3)
    w = g.qw.reshape(-1)
    J = J[..., 0].reshape(-1, 3) * w[:, None]
    M = M[..., 0].reshape(-1, 3) * w[:, None]
    ph = np.exp(1j * k * (rhat @ src.T))  # (P, S)
    Jh = ph @ J
    Mh = ph @ M
    rJ = np.sum(rhat * Jh, axis=1)
    return (-1j * k / (4 * np.pi)) * (z * (Jh - rhat * rJ[:, None]) - np.cross(rhat, Mh))
