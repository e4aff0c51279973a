"""O2: plain definition of the grid-accelerated (precorrected-FFT) operator.

The paper accelerates the matvec with FFTs (Appendix B) and cites the
precorrected-FFT method (Phillips & White 1997, ref. Phillips97a) among the
fast solvers it builds on.  The operator defined here is

    A_fft x = T( I H P s(x)  +  sum_{near (t,S)} [exact(t,S) - (I H P)|_(t,S)] s(x) )

where
* s(x): point sources at the triangle quadrature points b (weight w_b):
  J(r_b) w_b and div J w_b for the exterior J, interior J and exterior M sets
  (12 scalar fields; the interior M is -M);
* P: projection onto the uniform grid by tensor-product Lagrange stencils of
  p points per axis, P[g, b] = W_g(r_b);
* H: grid convolution with G_l(g - g') = exp(-jk_l d)/(4 pi d), d = |g-g'| h,
  and G_l(0) = 0, done exactly (aperiodic, zero padding to 2n per axis);
* I: interpolation by the same stencils, values and first derivatives
  (grad W_g), at the target quadrature points;
* exact(t,S): the panel-integrated moments of ``integrals.point_triangle``;
* (I H P)|_(t,S): the grid's own version of the same near interaction,
      P0g = sum_b w_b Gh(a,b), P1g = sum_b w_b Gh(a,b)(r_b - c_S),
      Qg = sum_b w_b grad_a Gh(a,b), Cg = sum_b w_b grad_a Gh(a,b) x (r_b - c_S),
  with Gh(a,b) = sum_{g,g'} W_g(r_a) G(g - g') W_g'(r_b);
* near pairs: triangle pairs with |c_t - c_S|^2 < r_near^2 (the pair (t,t)
  included);
* T: the testing of ``operator.test_rows``.

With every pair near the grid cancels exactly and A_fft = A (O1).  Stencil
base per axis: floor(u - (p-2)/2) with u = (x - origin)/h; stencil nodes
base .. base+p-1.
"""

from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from .mesh import Geometry
from .operator import (
    Media,
    current_sets,
    local_current,
    medium_fields,
    scatter_rows,
    sigma_normalised,
    test_rows,
)
from .integrals import point_triangle


def lagrange(t, p):
    """Lagrange basis on nodes 0..p-1 at t (any shape) and its derivative."""
    t = np.asarray(t, dtype=np.float64)
    L = np.ones(t.shape + (p,))
    dL = np.zeros(t.shape + (p,))
    for i in range(p):
        for m in range(p):
            if m == i:
                continue
            L[..., i] *= (t - m) / (i - m)
        # derivative: sum over the dropped factor
        for j in range(p):
            if j == i:
                continue
            term = np.full(t.shape, 1.0 / (i - j))
            for m in range(p):
                if m == i or m == j:
                    continue
                term = term * (t - m) / (i - m)
            dL[..., i] += term
    return L, dL


def stencils(grid, pts):
    """Base indices (P,3), weights (P,3,p) and derivative weights (P,3,p) [1/um]."""
    pts = np.asarray(pts, dtype=np.float64).reshape(-1, 3)
    u = (pts - np.asarray(grid.origin)) / grid.h
    base = np.floor(u - 0.5 * (grid.p - 2)).astype(np.int64)
    n = np.asarray(grid.n)
    if np.any(base < 0) or np.any(base + grid.p - 1 >= n):
        raise ValueError("stencil outside the grid")
    L, dL = lagrange(u - base, grid.p)
    return base, L, dL / grid.h


def _offsets(p):
    o = np.arange(p)
    return np.stack(np.meshgrid(o, o, o, indexing="ij"), axis=-1).reshape(-1, 3)  # (p^3, 3)


def stencil_weights(grid, pts):
    """Full tensor-product weights: index (P,p^3), value W (P,p^3), gradient (P,3,p^3)."""
    base, L, dL = stencils(grid, pts)
    off = _offsets(grid.p)
    idx3 = base[:, None, :] + off[None]  # (P, p^3, 3)
    n = grid.n
    gidx = (idx3[..., 0] * n[1] + idx3[..., 1]) * n[2] + idx3[..., 2]
    Lx, Ly, Lz = L[:, 0][:, off[:, 0]], L[:, 1][:, off[:, 1]], L[:, 2][:, off[:, 2]]
    dx, dy, dz = dL[:, 0][:, off[:, 0]], dL[:, 1][:, off[:, 1]], dL[:, 2][:, off[:, 2]]
    W = Lx * Ly * Lz
    gW = np.stack([dx * Ly * Lz, Lx * dy * Lz, Lx * Ly * dz], axis=1)
    return gidx, W, gW, base


def projection_matrix(grid, pts):
    gidx, W, _, _ = stencil_weights(grid, pts)
    P = len(gidx)
    ng = int(np.prod(grid.n))
    rows = gidx.reshape(-1)
    cols = np.repeat(np.arange(P), gidx.shape[1])
    return sp.csr_matrix((W.reshape(-1), (rows, cols)), shape=(ng, P))


def green_grid(k, h, dvec):
    """G(d) = exp(-jk|d|h)/(4 pi |d| h) on integer offsets d (...,3); 0 at d = 0."""
    dist = np.linalg.norm(np.asarray(dvec, dtype=np.float64), axis=-1) * h
    out = np.zeros(dist.shape, dtype=np.complex128)
    nz = dist > 0
    out[nz] = np.exp(-1j * k * dist[nz]) / (4 * np.pi * dist[nz])
    return out


def padded_green(grid, k):
    """G on the 2n-periodic padded grid (circular offsets; offset n set to 0)."""
    dims = []
    for a in range(3):
        m = 2 * grid.n[a]
        i = np.arange(m)
        d = np.where(i < grid.n[a], i, i - m).astype(np.float64)
        d[grid.n[a]] = np.nan
        dims.append(d)
    D = np.stack(np.meshgrid(*dims, indexing="ij"), axis=-1)
    G = green_grid(k, grid.h, np.nan_to_num(D, nan=0.0))
    bad = np.isnan(D).any(axis=-1)
    G[bad] = 0.0
    return G


def convolve(grid, Gpad, src):
    """Aperiodic grid convolution out = G * src on the physical grid (src (n0,n1,n2,B))."""
    n = grid.n
    Pd = tuple(2 * v for v in n)
    Gh = np.fft.fftn(Gpad)
    out = np.empty(src.shape, dtype=np.complex128)
    for b in range(src.shape[-1]):
        s = np.zeros(Pd, dtype=np.complex128)
        s[: n[0], : n[1], : n[2]] = src[..., b]
        out[..., b] = np.fft.ifftn(Gh * np.fft.fftn(s))[: n[0], : n[1], : n[2]]
    return out


def direct_convolve(grid, k, src):
    """Brute-force grid convolution (tiny grids only; pins ``convolve``)."""
    n = grid.n
    idx = np.stack(np.meshgrid(*[np.arange(v) for v in n], indexing="ij"), axis=-1).reshape(-1, 3)
    G = green_grid(k, grid.h, idx[:, None, :] - idx[None, :, :])
    flat = src.reshape(-1, src.shape[-1])
    return (G @ flat).reshape(src.shape)


def near_pairs(g: Geometry, r_near: float, targets=None):
    """List of (t, S) with |c_t - c_S|^2 < r_near^2, sorted by t then S."""
    tt = np.arange(g.nt) if targets is None else np.asarray(targets)
    c = g.centroid
    d2 = np.sum((c[tt][:, None, :] - c[None, :, :]) ** 2, axis=-1)
    ti, si = np.nonzero(d2 < r_near * r_near)
    return tt[ti], si


def grid_moments(grid, g: Geometry, Gpad, pt, ps):
    """(I H P)|_(t,S) moments for near pairs (pt[i], ps[i]) at all target points.

    ``Gpad`` is the padded grid Green's function of ``padded_green`` (the
    values G(g - g') are read from it by circular offset).

    Returns P0g (np, q), P1g (np, q, 3), Qg (np, q, 3), Cg (np, q, 3).
    """
    q = g.q
    p3 = grid.p ** 3
    _, Wt, gWt, bt = stencil_weights(grid, g.qpts[pt].reshape(-1, 3))
    _, Ws, _, bs = stencil_weights(grid, g.qpts[ps].reshape(-1, 3))
    npair = len(pt)
    Wt = Wt.reshape(npair, q, p3)
    gWt = gWt.reshape(npair, q, 3, p3)
    bt = bt.reshape(npair, q, 3)
    Ws = Ws.reshape(npair, q, p3)
    bs = bs.reshape(npair, q, 3)
    off = _offsets(grid.p)
    # grid offset between target stencil node i and source stencil node j
    dvec = (
        bt[:, :, None, None, None, :] + off[None, None, None, :, None, :]
        - bs[:, None, :, None, None, :] - off[None, None, None, None, :, :]
    )  # (np, qa, qb, p3, p3, 3)
    n2 = np.asarray(grid.padded)
    dm = np.mod(dvec, n2)
    Gv = Gpad[dm[..., 0], dm[..., 1], dm[..., 2]]
    Gab = np.einsum("paj,pbk,pabjk->pab", Wt, Ws, Gv, optimize=True)
    gGab = np.einsum("paxj,pbk,pabjk->paxb", gWt, Ws, Gv, optimize=True)
    wb = g.qw[ps]  # (np, q)
    rel = g.qpts[ps] - g.centroid[ps][:, None, :]  # (np, qb, 3)
    P0g = np.einsum("pab,pb->pa", Gab, wb)
    P1g = np.einsum("pab,pb,pbx->pax", Gab, wb, rel)
    Qg = np.einsum("paxb,pb->pax", gGab, wb)
    Cg = np.einsum("ijk,pajb,pb,pbk->pai", _EPS, gGab, wb, rel)
    return P0g, P1g, Qg, Cg


_EPS = np.zeros((3, 3, 3))
_EPS[0, 1, 2] = _EPS[1, 2, 0] = _EPS[2, 0, 1] = 1.0
_EPS[0, 2, 1] = _EPS[2, 1, 0] = _EPS[1, 0, 2] = -1.0


def exact_moments_pairs(g: Geometry, k, pt, ps):
    """Exact (P0, P1, Q, C) of source ps[i] at the points of target pt[i]."""
    q = g.q
    r = g.qpts[pt]  # (np, q, 3)
    same = (pt == ps)[:, None] & np.ones((1, q), bool)
    sidx = np.where(same, np.arange(q)[None, :], -1)
    tv = g.V[g.T[ps]][:, None]
    cen = g.centroid[ps][:, None]
    P0, P1, Q = point_triangle(r, tv, cen, g.qpts[ps][:, None], g.qw[ps][:, None], k, same, sidx)
    C = np.cross(Q, r - cen)
    return P0, P1, Q, C


def near_corrections(grid, g: Geometry, media: Media, Gpads, pt, ps, chunk: int = 64):
    """Per near pair and target point: exact - grid moments, for (k_e, k_i)."""
    out = []
    for k, Gpad in zip(media.k, Gpads):
        parts = []
        for i in range(0, len(pt), chunk):
            a, b = pt[i : i + chunk], ps[i : i + chunk]
            E0, E1, EQ, EC = exact_moments_pairs(g, k, a, b)
            G0, G1, GQ, GC = grid_moments(grid, g, Gpad, a, b)
            parts.append((E0 - G0, E1 - G1, EQ - GQ, EC - GC))
        out.append(tuple(np.concatenate([p[j] for p in parts]) for j in range(4)))
    return out


def _near_fields(g: Geometry, corr, pt, ps, summ, targets):
    """Sum over near pairs of correction moments applied to source summaries.

    Returns A, phi, gphi, curl at the points of ``targets`` (in that order).
    """
    d0, d1, dq, dc = corr
    a, beta = summ
    B = a.shape[-1]
    pos = {int(t): i for i, t in enumerate(targets)}
    ti = np.array([pos[int(t)] for t in pt], dtype=np.int64)
    q = g.q
    aS, bS = a[ps], beta[ps]  # (np, B), (np, 3, B)
    A = d1[..., None] * aS[:, None, None, :] - d0[:, :, None, None] * bS[:, None, :, :]
    phi = 2.0 * d0[..., None] * aS[:, None, :]
    gphi = 2.0 * dq[..., None] * aS[:, None, None, :]
    curl = dc[..., None] * aS[:, None, None, :] - np.cross(dq[:, :, :, None], bS[:, None, :, :], axisa=2, axisb=2, axisc=2)
    nt = len(targets)
    outs = []
    for arr in (A, phi, gphi, curl):
        acc = np.zeros((nt,) + arr.shape[1:], dtype=np.complex128)
        np.add.at(acc, ti, arr)
        outs.append(acc)
    return outs


class PFFT:
    """O2 operator on one mesh and grid."""

    def __init__(self, g: Geometry, media: Media, grid, r_near: float):
        self.g, self.media, self.grid, self.r_near = g, media, grid, r_near
        pts = g.qpts.reshape(-1, 3)
        self.P = projection_matrix(grid, pts)
        gidx, W, gW, _ = stencil_weights(grid, pts)
        ng = int(np.prod(grid.n))
        npnt = len(pts)
        cols = gidx.reshape(-1)
        rows = np.repeat(np.arange(npnt), gidx.shape[1])
        self.I = sp.csr_matrix((W.reshape(-1), (rows, cols)), shape=(npnt, ng))
        self.D = [sp.csr_matrix((gW[:, a].reshape(-1), (rows, cols)), shape=(npnt, ng)) for a in range(3)]
        self.Gpad = [padded_green(grid, k) for k in media.k]

    # -- grid part ------------------------------------------------------
    def grid_fields(self, sets, targets=None):
        """Interpolated grid potentials of both media at the target points."""
        g, grid = self.g, self.grid
        Jes, Jis, Ms = sets
        w = g.qw.reshape(-1)
        B = Jes[0].shape[-1]

        def pointsrc(summ, sgn=1.0):
            a, beta = summ
            rel = g.qpts - g.centroid[:, None, :]
            J = rel[..., None] * a[:, None, None, :] - beta[:, None, :, :]
            rho = 2.0 * np.broadcast_to(a[:, None, :], (g.nt, g.q, B))
            J = sgn * J.reshape(-1, 3, B) * w[:, None, None]
            rho = sgn * rho.reshape(-1, B) * w[:, None]
            return [J[:, 0], J[:, 1], J[:, 2], rho]

        n = grid.n
        if targets is None:
            rsel = slice(None)
        else:
            rsel = (np.asarray(targets)[:, None] * g.q + np.arange(g.q)[None, :]).reshape(-1)
        res = []
        for med, (k, Gp) in enumerate(zip(self.media.k, self.Gpad)):
            Jsrc = pointsrc(Jes if med == 0 else Jis)
            Msrc = pointsrc(Ms, 1.0 if med == 0 else -1.0)
            fields = []
            for comps in (Jsrc, Msrc):
                grids = [(self.P @ c).reshape(n + (B,)) for c in comps]
                conv = [convolve(grid, Gp, s).reshape(-1, B) for s in grids]
                vec = np.stack([self.I[rsel] @ conv[i] for i in range(3)], axis=1)  # (p,3,B)
                sca = self.I[rsel] @ conv[3]
                # gradient of each component: grad[c][axis]
                grad = [[self.D[ax][rsel] @ conv[c] for ax in range(3)] for c in range(4)]
                gsca = np.stack(grad[3], axis=1)
                curl = np.stack(
                    [grad[2][1] - grad[1][2], grad[0][2] - grad[2][0], grad[1][0] - grad[0][1]], axis=1
                )
                fields.append((vec, sca, gsca, curl))
            res.append(fields)
        return res

    # -- near corrections ----------------------------------------------
    def near(self, targets=None):
        """Near pairs and their corrections (exact - grid moments) for the targets; those of the
        whole mesh (targets None) are computed once and kept, since they do not depend on x or sigma."""
        if targets is None and getattr(self, "_near_all", None) is not None:
            return self._near_all
        tg = np.arange(self.g.nt) if targets is None else np.asarray(targets)
        pt, ps = near_pairs(self.g, self.r_near, tg)
        corr = near_corrections(self.grid, self.g, self.media, self.Gpad, pt, ps)
        if targets is None:
            self._near_all = (pt, ps, corr)
        return pt, ps, corr

    # -- full apply -----------------------------------------------------
    def apply(self, x, sigma_pts_S, targets=None):
        """y = A_fft x (rows of all triangles, or the rows touched by ``targets``)."""
        g, media = self.g, self.media
        x = np.asarray(x, dtype=np.complex128)
        squeeze = x.ndim == 1
        X2 = x[:, None] if squeeze else x
        sets = current_sets(g, X2)
        tg = np.arange(g.nt) if targets is None else np.asarray(targets)
        gf = self.grid_fields(sets, None if targets is None else tg)
        pt, ps, corr = self.near(tg if targets is not None else None)
        (ke, ki), (ze, zi) = media.k, media.z
        B = X2.shape[1]
        q = g.q
        meds = []
        for med, (k, z) in enumerate(((ke, ze), (ki, zi))):
            Jsumm = sets[0] if med == 0 else sets[1]
            Msumm = sets[2] if med == 0 else (-sets[2][0], -sets[2][1])
            Jg, Mg = gf[med]
            Jn = _near_fields(g, corr[med], pt, ps, Jsumm, tg)
            Mn = _near_fields(g, corr[med], pt, ps, Msumm, tg)
            Jtot = [Jg[i].reshape((len(tg), q) + Jg[i].shape[1:]) + Jn[i] for i in range(4)]
            Mtot = [Mg[i].reshape((len(tg), q) + Mg[i].shape[1:]) + Mn[i] for i in range(4)]
            meds.append(medium_fields(Jtot, Mtot, k, z))
        sig = sigma_normalised(sigma_pts_S)
        Jsum = local_current(g, tg, sets[0]) + local_current(g, tg, sets[1])
        Ml = local_current(g, tg, sets[2])
        val = test_rows(g, tg, meds[0], meds[1], Jsum, Ml, sig[tg])
        y = np.zeros((g.N, B), dtype=np.complex128)
        scatter_rows(g, tg, val, y)
        return y[:, 0] if squeeze else y


# ---------------------------------------------------------------- transpose
def dense(op: "PFFT", sigma_pts_S, chunk: int = 128):
    """The O2 matrix, column by column (apply to blocks of unit vectors)."""
    N = op.g.N
    A = np.zeros((N, N), dtype=np.complex128)
    for c0 in range(0, N, chunk):
        c1 = min(N, c0 + chunk)
        E = np.zeros((N, c1 - c0), dtype=np.complex128)
        E[np.arange(c0, c1), np.arange(c1 - c0)] = 1.0
        A[:, c0:c1] = op.apply(E, sigma_pts_S)
    return A


def apply_transpose(op: "PFFT", y, sigma_pts_S, A=None):
    """A^T y for the O2 operator: the plain definition, the transposed matrix
    (no conjugation).  Pass a precomputed ``dense(op, sigma)`` as A to reuse it."""
    if A is None:
        A = dense(op, sigma_pts_S)
    return A.T @ np.asarray(y, dtype=np.complex128)
