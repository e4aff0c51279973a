"""O1: the Galerkin PMCHW operator with surface-conductive absorber rows.

Definitions followed (paper Sec. II and Appendix A):

* Fields of medium l (Eqs. 15-16), in units with eta0 = 1:
      E_l = -z_l L_l(J) + K_l(M),      H_l = -K_l(J) - L_l(M)/z_l,
      L_l(X) = jk_l int [X + k_l^-2 grad div' X] G_l dS',
      K_l(X) = -int grad G_l x X dS',
  with z_l = sqrt(mu_l/eps_l), k_l = 2 pi sqrt(eps_l mu_l)/lambda0.
  In potentials: with A = int G J, phi = int G div'J, F = int G M,
  psi = int G div'M,
      E_l = -z_l (jk A + (j/k) grad phi) - curl F,
      H_l = curl A - (1/z_l) (jk F + (j/k) grad psi).
* Current sets (Eqs. 10-12): exterior (J_e, M), interior (J_i, -M).
* Rows, tested with the RWG X_n (Eqs. testedLOp/testedKOp, testedSig*):
      Eq. 1 / Eq. 3:  <X_n, E_e - E_i>                      (weak form)
      Eq. 2:          <X_n, H_e - H_i>                      (weak form)
      Eq. 13:         <X_n, H_e^+ - H_i^-> - <sigma (n x X_n), E_e^+>
      Eq. 14:         <X_n, J_e + J_i> - <sigma X_n, E_i^->
  Readings of the paper (it is silent on these; see the design notes):
  - The operators of Eqs. 15-16 are principal values; the side limits add
    H_tan^+- = H_tan,pv +- (J x n)/2 and E_tan^+- = E_tan,pv +- (n x M)/2
    (exterior set on the + side, interior set on the - side).
  - Eq. 13 (n x dH = sigma E_tan) is tested the way the paper tests Eq. 2,
    whose n x H continuity becomes <X_n, H> with the Galerkin operators:
    rotating both sides gives dH_tan = -sigma n x E, so
    <X_n, dH> = <sigma (n x X_n), E>.  The H part is then exactly the
    Eq. 2 row (Appendix A's tested operators); with sigma = 0 the absorber
    rows reduce exactly to PMCHW.  Side-limit terms: +<X_n, (J_e+J_i) x n>/2
    and -<sigma X_n, M>/2 in Eq. 13, -<sigma X_n, n x M>/2 in Eq. 14.
  - The sigma-weighted E is evaluated in strong form (gradient of the scalar
    potential at the points).  The weak forms use
    <X_n, grad phi> = -<div X_n, phi> (RWG is div-conforming).

Everything is evaluated at the triangle quadrature points: per target point
the potentials of every source triangle S follow from three moments
(``integrals.point_triangle``) and the per-triangle current summary
J(r') = a (r' - c_S) - beta:

      A = a P1 - beta P0,  phi = 2 a P0,  grad phi = 2 a Q,
      curl A = a C - Q x beta,  with C = Q x (r - c_S)
  (grad G is parallel to r - r', so int grad G x (r' - c) = Q x (r - c)).
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np
import scipy.sparse as sp

from . import ETA0
from .integrals import point_triangle
from .mesh import Geometry, edge_coefficients, row_index


@dataclasses.dataclass
class Media:
    """Interior (i) and exterior (e) media, relative and real; wavelength in um."""

    eps_i: float
    mu_i: float
    eps_e: float
    mu_e: float
    lam0: float

    @property
    def k(self):  # (k_e, k_i) in 1/um
        w = 2 * math.pi / self.lam0
        return (w * math.sqrt(self.eps_e * self.mu_e), w * math.sqrt(self.eps_i * self.mu_i))

    @property
    def z(self):  # (z_e, z_i), relative impedances
        return (math.sqrt(self.mu_e / self.eps_e), math.sqrt(self.mu_i / self.eps_i))


# ---------------------------------------------------------------- summaries
def summaries(g: Geometry, coef: np.ndarray):
    """Per-triangle summary (a, beta) of the RWG expansion with edge coefficients ``coef``.

    On triangle t, J(r) = sum_k coef_k s_k l_k/(2A_t) (r - v_k) = a (r - c_t) - beta.
    coef: (ne, B) -> a: (nt, B), beta: (nt, 3, B).
    """
    jk = coef[g.tri_edge] * (g.tri_sign * g.edge_len[g.tri_edge] / (2.0 * g.area[:, None]))[..., None]
    a = jk.sum(axis=1)
    rel = g.V[g.T] - g.centroid[:, None, :]  # (nt, 3 local, 3 xyz)
    beta = np.einsum("tkx,tkb->txb", rel, jk)
    return a, beta


def current_sets(g: Geometry, x: np.ndarray):
    """Summaries of the exterior J, interior J and exterior M sets (x: (N, B))."""
    Je, Ji, Me = edge_coefficients(g, x)
    return summaries(g, Je), summaries(g, Ji), summaries(g, Me)


def local_current(g: Geometry, tris, summ):
    """J at the quadrature points of triangles ``tris`` from their own summary."""
    a, beta = summ
    rel = g.qpts[tris] - g.centroid[tris][:, None, :]  # (nt_c, q, 3)
    return rel[..., None] * a[tris][:, None, None, :] - beta[tris][:, None, :, :]


# ---------------------------------------------------------------- fields
def _cross(u, v, axis_u=-1, axis_v=-1):
    return np.cross(u, v, axisa=axis_u, axisb=axis_v)


def fields_from_moments(P0, P1, Q, C, summ):
    """Potentials at points from moments (P0 (p,S), P1/Q/C (p,S,3)) and summaries.

    Returns A (p,3,B), phi (p,B), grad phi (p,3,B), curl A (p,3,B).
    """
    a, beta = summ
    A = np.einsum("psi,sb->pib", P1, a) - np.einsum("ps,sib->pib", P0, beta)
    phi = 2.0 * np.einsum("ps,sb->pb", P0, a)
    gphi = 2.0 * np.einsum("psi,sb->pib", Q, a)
    curl = np.einsum("psi,sb->pib", C, a)
    # - sum_s Q_s x beta_s
    eps = np.zeros((3, 3, 3))
    eps[0, 1, 2] = eps[1, 2, 0] = eps[2, 0, 1] = 1.0
    eps[0, 2, 1] = eps[2, 1, 0] = eps[1, 0, 2] = -1.0
    curl = curl - np.einsum("ijk,psj,skb->pib", eps, Q, beta)
    return A, phi, gphi, curl


def medium_fields(Jf, Mf, k, z):
    """Combine potentials of one medium into the quantities the rows need.

    Jf = (A, phi, grad phi, curl A) of the J set, Mf = the same of the M set.
    Returns dict with weak-form pieces and the strong-form E, H (principal value).
    """
    A, phi, gphi, curlA = Jf
    F, psi, gpsi, curlF = Mf
    jk = 1j * k
    return {
        "WE": -z * jk * A - curlF,  # tested with X
        "wE": z * (1j / k) * phi,  # tested with div X
        "WH": curlA - (jk / z) * F,
        "wH": (1j / (k * z)) * psi,
        "E": -z * (jk * A + (1j / k) * gphi) - curlF,
        "H": curlA - (1.0 / z) * (jk * F + (1j / k) * gpsi),
    }


# ---------------------------------------------------------------- testing
def test_rows(g: Geometry, tris, fe, fi, Jsum_loc, Mloc, sig):
    """Tested values of triangles ``tris`` for their 3 local RWG functions.

    fe, fi: ``medium_fields`` dicts for the exterior / interior medium, arrays
    shaped (nt_c, q, 3, B) (vectors) or (nt_c, q, B) (scalars).
    Jsum_loc: J_e + J_i at the points, Mloc: M (exterior) at the points
    (nt_c, q, 3, B).  sig: normalised conductivity at the points (nt_c, q).
    Returns val (nt_c, 3 local, 4 row types, B).
    """
    T = g.T[tris]
    w = g.qw[tris]  # (nt_c, q)
    r = g.qpts[tris]
    n = g.normal[tris]
    cX = g.tri_sign[tris] * g.edge_len[g.tri_edge[tris]] / (2.0 * g.area[tris][:, None])  # (nt_c, 3)
    divX = 2.0 * cX
    vk = g.V[T]  # (nt_c, 3 local, 3)
    X = cX[:, :, None, None] * (r[:, None, :, :] - vk[:, :, None, :])  # (nt_c, k, q, 3)

    def tX(V):  # <X_k, V>
        return np.einsum("tkqx,tq,tqxb->tkb", X, w, V)

    def tX_sig(V):
        return np.einsum("tkqx,tq,tqxb->tkb", X, w * sig, V)

    def tnX_sig(V):  # <sigma n x X_k, V>
        nX = np.cross(n[:, None, None, :], X)
        return np.einsum("tkqx,tq,tqxb->tkb", nX, w * sig, V)

    def tdiv(s):
        return np.einsum("tk,tq,tqb->tkb", divX, w, s)

    def ncross(V):  # n x V at each point, n per triangle
        return np.cross(n[:, None, :, None], V, axisa=-2, axisb=-2, axisc=-2)

    B = fe["WE"].shape[-1]
    val = np.zeros((len(tris), 3, 4, B), dtype=np.complex128)
    val[:, :, 0] = tX(fe["WE"] - fi["WE"]) + tdiv(fe["wE"] - fi["wE"])
    val[:, :, 1] = tX(fe["WH"] - fi["WH"]) + tdiv(fe["wH"] - fi["wH"])
    nM = ncross(Mloc)
    val[:, :, 2] = (
        val[:, :, 1] - 0.5 * tX(ncross(Jsum_loc)) - tnX_sig(fe["E"]) - 0.5 * tX_sig(Mloc)
    )
    val[:, :, 3] = tX(Jsum_loc) - tX_sig(fi["E"]) - 0.5 * tX_sig(nM)
    return val


def scatter_rows(g: Geometry, tris, val, y):
    """y[row(edge(t,k), type)] += val[t, k, type] for existing rows."""
    rows = row_index(g)
    e = g.tri_edge[tris]  # (nt_c, 3)
    rr = rows[e]  # (nt_c, 3, 4)
    m = rr >= 0
    np.add.at(y, rr[m], val[m])


def sigma_normalised(sigma_S):
    return np.asarray(sigma_S, dtype=np.float64) * ETA0


# ---------------------------------------------------------------- O1 direct matvec
def _exact_moments(g: Geometry, tris, k, srcs=None):
    """Exact moments of source triangles ``srcs`` at the points of ``tris``."""
    if srcs is None:
        srcs = np.arange(g.nt)
    r = g.qpts[tris]  # (nt_c, q, 3)
    q = g.q
    rr = r[:, :, None, :]
    same = tris[:, None, None] == srcs[None, None, :]  # (nt_c, 1, S)
    same = np.broadcast_to(same, (len(tris), q, len(srcs)))
    sidx = np.broadcast_to(np.arange(q)[None, :, None], same.shape)
    tv = g.V[g.T[srcs]][None, None]  # (1,1,S,3,3)
    cen = g.centroid[srcs][None, None]
    sp_ = g.qpts[srcs][None, None]
    sw = g.qw[srcs][None, None]
    P0, P1, Q = point_triangle(rr, tv, cen, sp_, sw, k, same, np.where(same, sidx, -1))
    C = np.cross(Q, rr - cen)
    return P0, P1, Q, C


def point_fields_exact(g: Geometry, media: Media, tris, sets, srcs=None):
    """Exterior and interior ``medium_fields`` at the points of ``tris`` (O1)."""
    (ke, ki), (ze, zi) = media.k, media.z
    Jes, Jis, Ms = sets
    if srcs is not None:
        Jes = tuple(v[srcs] for v in Jes)
        Jis = tuple(v[srcs] for v in Jis)
        Ms = tuple(v[srcs] for v in Ms)
    nq = len(tris) * g.q
    out = []
    for k, z, Js, msign in ((ke, ze, Jes, 1.0), (ki, zi, Jis, -1.0)):
        P0, P1, Q, C = _exact_moments(g, tris, k, srcs)
        S = P0.shape[-1]
        P0, P1, Q, C = P0.reshape(nq, S), P1.reshape(nq, S, 3), Q.reshape(nq, S, 3), C.reshape(nq, S, 3)
        Jf = fields_from_moments(P0, P1, Q, C, Js)
        Mf = fields_from_moments(P0, P1, Q, C, (msign * Ms[0], msign * Ms[1]))
        f = medium_fields(Jf, Mf, k, z)
        out.append({key: v.reshape((len(tris), g.q) + v.shape[1:]) for key, v in f.items()})
    return out[0], out[1]


def matvec(g: Geometry, media: Media, x, sigma_pts_S, chunk: int = 8, tris=None):
    """Direct O(N^2) matvec y = A x of the dense operator (O1), matrix free.

    x: (N,) or (N, B).  sigma_pts_S: conductivity [S] at every quadrature
    point (nt, q).  ``tris`` restricts the evaluation to the rows of those
    target triangles (their contributions are still complete for each row only
    when both triangles of an edge are included).
    """
    x = np.asarray(x, dtype=np.complex128)
    squeeze = x.ndim == 1
    X2 = x[:, None] if squeeze else x
    sets = current_sets(g, X2)
    sig = sigma_normalised(sigma_pts_S)
    y = np.zeros((g.N, X2.shape[1]), dtype=np.complex128)
    all_t = np.arange(g.nt) if tris is None else np.asarray(tris)
    for i in range(0, len(all_t), chunk):
        tc = all_t[i : i + chunk]
        fe, fi = point_fields_exact(g, media, tc, sets)
        Jsum = local_current(g, tc, sets[0]) + local_current(g, tc, sets[1])
        Ml = local_current(g, tc, sets[2])
        val = test_rows(g, tc, fe, fi, Jsum, Ml, sig[tc])
        scatter_rows(g, tc, val, y)
    return y[:, 0] if squeeze else y


# ---------------------------------------------------------------- O1 dense assembly
def summary_map(g: Geometry):
    """Sparse map x -> stacked summaries [(set, tri, comp)] (12 nt rows, N cols).

    set 0 = J_e, 1 = J_i, 2 = M (exterior); comp 0 = a, 1..3 = beta_xyz.
    """
    N = g.N
    rows, cols, vals = [], [], []
    L = g.edge_class == 0
    ci = g.edge_cidx
    # coefficient of unknown -> edge coefficient, per set
    def unknown_of(set_id, e):
        if L[e]:
            base = {0: g.block("JL"), 1: g.block("JL"), 2: g.block("ML")}[set_id]
            sgn = -1.0 if set_id == 1 else 1.0
        else:
            base = {0: g.block("JeR"), 1: g.block("JiR"), 2: g.block("MR")}[set_id]
            sgn = 1.0
        return base + ci[e], sgn

    rel = g.V[g.T] - g.centroid[:, None, :]
    for t in range(g.nt):
        for kk in range(3):
            e = g.tri_edge[t, kk]
            jk = g.tri_sign[t, kk] * g.edge_len[e] / (2.0 * g.area[t])
            for s in range(3):
                col, sgn = unknown_of(s, e)
                base = (s * g.nt + t) * 4
                rows.append(base)
                cols.append(col)
                vals.append(sgn * jk)
                for c in range(3):
                    rows.append(base + 1 + c)
                    cols.append(col)
                    vals.append(sgn * jk * rel[t, kk, c])
    return sp.csr_matrix((vals, (rows, cols)), shape=(12 * g.nt, N))


def _unit_fields(P0, P1, Q, C):
    """Potentials at points of unit summaries of each source (no sum over S).

    Inputs (p, S) / (p, S, 3).  Returns A, phi, gphi, curl shaped
    (p, 3, S*4) / (p, S*4) with the column order (S, comp).
    """
    p, S = P0.shape
    A = np.zeros((p, 3, S, 4), dtype=np.complex128)
    phi = np.zeros((p, S, 4), dtype=np.complex128)
    gphi = np.zeros((p, 3, S, 4), dtype=np.complex128)
    curl = np.zeros((p, 3, S, 4), dtype=np.complex128)
    A[:, :, :, 0] = np.moveaxis(P1, 2, 1)
    phi[:, :, 0] = 2.0 * P0
    gphi[:, :, :, 0] = 2.0 * np.moveaxis(Q, 2, 1)
    curl[:, :, :, 0] = np.moveaxis(C, 2, 1)
    for c in range(3):
        e = np.zeros(3)
        e[c] = 1.0
        A[:, c, :, 1 + c] = -P0
        curl[:, :, :, 1 + c] = -np.moveaxis(np.cross(Q, e), 2, 1)
    return (A.reshape(p, 3, S * 4), phi.reshape(p, S * 4), gphi.reshape(p, 3, S * 4), curl.reshape(p, 3, S * 4))


def assemble(g: Geometry, media: Media, sigma_pts_S, chunk: int = 2, tris=None, rows_out=None) -> np.ndarray:
    """Dense N x N matrix of O1 (for small meshes).  ``tris`` restricts the assembly to the
    rows those target triangles contribute to (a row is complete when both triangles of its edge
    are included; the other rows stay zero or partial).  With ``rows_out`` (row indices) only
    those rows are kept, as a len(rows_out) x N matrix, so large meshes fit in memory."""
    return assemble_many(g, media, [sigma_pts_S], chunk, tris, rows_out)[0]


def assemble_many(g: Geometry, media: Media, sigmas, chunk: int = 2, tris=None, rows_out=None):
    """``assemble`` for several conductivity profiles of one mesh at once: the panel moments
    are computed once per target chunk and tested with each profile in turn.  Returns one
    matrix per entry of ``sigmas`` (each a per-point conductivity [S], (nt, q))."""
    (ke, ki), (ze, zi) = media.k, media.z
    S = g.nt
    smap = summary_map(g)
    sigs = [sigma_normalised(s) for s in sigmas]
    nrow = g.N if rows_out is None else len(rows_out)
    As = [np.zeros((nrow, g.N), dtype=np.complex128) for _ in sigs]
    if rows_out is None:
        keep = np.arange(g.N)
    else:
        rows_out = np.asarray(rows_out)
        keep = -np.ones(g.N, dtype=np.int64)
        keep[rows_out] = np.arange(len(rows_out))
    rows = row_index(g)
    targets = np.arange(g.nt) if tris is None else np.asarray(tris)
    for i in range(0, len(targets), chunk):
        tc = targets[i : i + chunk]
        nq = len(tc) * g.q
        meds = []
        for k in (ke, ki):
            P0, P1, Q, C = _exact_moments(g, tc, k)
            meds.append(_unit_fields(P0.reshape(nq, S), P1.reshape(nq, S, 3), Q.reshape(nq, S, 3), C.reshape(nq, S, 3)))
        B = 3 * S * 4

        def stack(v0, v1, v2):  # place per-set blocks along the column axis
            return np.concatenate([v0, v1, v2], axis=-1)

        Ue, Ui = meds
        # medium e: J fields from set 0, M fields from set 2; medium i: J from set 1, M = -(set 2)
        Jf_e = tuple(stack(u, np.zeros_like(u), np.zeros_like(u)) for u in Ue)
        Mf_e = tuple(stack(np.zeros_like(u), np.zeros_like(u), u) for u in Ue)
        Jf_i = tuple(stack(np.zeros_like(u), u, np.zeros_like(u)) for u in Ui)
        Mf_i = tuple(stack(np.zeros_like(u), np.zeros_like(u), -u) for u in Ui)
        fe = medium_fields(Jf_e, Mf_e, ke, ze)
        fi = medium_fields(Jf_i, Mf_i, ki, zi)
        fe = {kk: v.reshape((len(tc), g.q) + v.shape[1:]) for kk, v in fe.items()}
        fi = {kk: v.reshape((len(tc), g.q) + v.shape[1:]) for kk, v in fi.items()}
        # local currents of unit summaries: only columns of the target triangle itself
        Jsum = np.zeros((len(tc), g.q, 3, B), dtype=np.complex128)
        Ml = np.zeros((len(tc), g.q, 3, B), dtype=np.complex128)
        for j, t in enumerate(tc):
            rel = g.qpts[t] - g.centroid[t]  # (q, 3)
            for sid, tgt in ((0, Jsum), (1, Jsum), (2, Ml)):
                base = sid * S * 4 + t * 4
                tgt[j, :, :, base] += rel
                for c in range(3):
                    tgt[j, :, c, base + 1 + c] -= 1.0
        e = g.tri_edge[tc]
        rr = rows[e]
        m = rr >= 0
        kr = keep[rr[m]]
        sel = kr >= 0
        for A, sig in zip(As, sigs):
            val = test_rows(g, tc, fe, fi, Jsum, Ml, sig[tc])  # (nt_c, 3, 4, 12S)
            contrib = np.asarray((smap.T @ val[m].T).T)
            np.add.at(A, kr[sel], contrib[sel])
    return As


def solve_dense(A, b):
    """LU solve of the dense system (numpy / LAPACK)."""
    return np.linalg.solve(A, b)
