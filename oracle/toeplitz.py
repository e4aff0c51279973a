"""Exact block-Toeplitz product of the dense operator on a straight extruded guide.

The paper's own fast product (Appendix B): on a mesh that repeats along x with period dx, the
interaction between the basis functions of two slices depends only on the slices' offset. So the
plain-surface block A_LL, restricted to the regular slices, is block Toeplitz, and it applies by
circulant embedding and FFTs along the slice index.

TEST INFRASTRUCTURE: an independent evaluation of O1 on periodic meshes.  Every block comes from
O1 entries: operator.assemble restricted to the rows of the first and the last regular slice
gives the offsets of both signs.  Each product equals O1's direct matvec on those rows to rounding.

Slices: an edge of a mesh built from uniform x-nodes x0 + i dx belongs to slice floor((m_x - x0)/dx)
(m its midpoint).  Rings of edges at x_i and the edges between x_i and x_(i+1) both belong to slice
i.  The regular slices (by default those strictly between the end caps, 1 .. nslices - 1; or a given
range, such as the plain section between two absorbers) hold plain-surface edges joining lateral
triangles only, and their edges are translates of the first regular slice's.
Within a slice the edges are ordered by midpoint.  Each edge carries a sign, -1 where the
translate has its two triangles in the opposite roles (its basis function is then the negated
translate).
"""

from __future__ import annotations

import numpy as np

from . import operator
from .mesh import Geometry


class SliceLayout:
    """Regular slices of the plain-surface (L) edges: ``edges[s]`` the edges of regular slice
    ``first + s`` in the common local order, ``sign[e]`` the orientation of edge e relative to the
    first regular slice."""

    def __init__(self, g: Geometry, x0: float, dx: float, nslices: int, first: int = 1, count: int | None = None):
        mid = 0.5 * (g.V[g.edge_v[:, 0]] + g.V[g.edge_v[:, 1]])
        u = (mid[:, 0] - x0) / dx
        s = np.floor(u + 1e-9).astype(np.int64)
        frac = np.round(u - s, 6)
        tri_x = g.V[g.T][:, :, 0]
        cap = np.ptp(tri_x, axis=1) < 1e-12 * dx
        lateral = ~cap[g.edge_t[:, 0]] & ~cap[g.edge_t[:, 1]]
        count = nslices - first if count is None else count
        if not (1 <= first and count >= 1 and first + count <= nslices):
            raise ValueError(f"regular slices {first} .. {first + count - 1} must lie within 1 .. {nslices - 1} "
                             "(slice 0 and the end caps are not regular)")
        self.first = first
        self.count = count
        ok = (g.edge_class == 0) & lateral & (s >= self.first) & (s < self.first + self.count)
        self.edges, self.sign = [], np.zeros(g.ne)
        ref_keys = ref_plus = None
        for k in range(self.count):
            sel = np.nonzero(ok & (s == self.first + k))[0]
            keys = np.stack([frac[sel], np.round(mid[sel, 1], 9), np.round(mid[sel, 2], 9)], 1)
            order = np.lexsort(keys.T[::-1])
            sel, keys = sel[order], keys[order]
            plus = g.centroid[g.edge_t[sel, 0]] - mid[sel]
            if ref_keys is None:
                ref_keys, ref_plus = keys, plus
                self.sign[sel] = 1.0
            else:
                if keys.shape != ref_keys.shape or not np.array_equal(keys, ref_keys):
                    raise ValueError(f"slice {self.first + k} is not a translate of slice {self.first}")
                same = np.linalg.norm(plus - ref_plus, axis=1) < 1e-9 * dx
                minus = g.centroid[g.edge_t[sel, 1]] - mid[sel]
                if not np.all(same | (np.linalg.norm(minus - ref_plus, axis=1) < 1e-9 * dx)):
                    raise ValueError("edge orientation does not repeat")
                self.sign[sel] = np.where(same, 1.0, -1.0)
            self.edges.append(sel)
        self.m = 2 * len(self.edges[0])  # unknowns per slice: J then M of each edge

    def unknowns(self, g: Geometry, k: int):
        """(indices, signs) of regular slice k's unknowns in the local order."""
        e = self.edges[k]
        idx = np.concatenate([g.block("JL") + g.edge_cidx[e], g.block("ML") + g.edge_cidx[e]])
        sg = np.concatenate([self.sign[e], self.sign[e]])
        return idx, sg


def blocks(g: Geometry, media, sigma_pts_S, lay: SliceLayout):
    """T[d] for d = -(R-1) .. R-1 (R regular slices): the block of O1 coupling slice i's rows to
    slice j's unknowns with i - j = d, in the local order and orientation of the first slice."""
    R = lay.count
    T = {}
    for ref in (0, R - 1):
        tris = np.unique(g.edge_t[lay.edges[ref]].reshape(-1))
        ri, rs = lay.unknowns(g, ref)
        A = operator.assemble(g, media, sigma_pts_S, tris=tris, rows_out=ri)
        for j in range(R):
            ci, cs = lay.unknowns(g, j)
            T[ref - j] = (rs[:, None] * A[:, ci]) * cs[None, :]
    return T


def apply(T, xs):
    """y_i = sum_j T[i - j] x_j for slice vectors xs (R, m), by circulant embedding of size 2R."""
    R, m = xs.shape
    P = 2 * R
    C = np.zeros((P, m, m), dtype=np.complex128)
    for d in range(R):
        C[d] = T[d]
    for d in range(1, R):
        C[P - d] = T[-d]
    Xp = np.zeros((P, m), dtype=np.complex128)
    Xp[:R] = xs
    Y = np.fft.ifft(np.einsum("kab,kb->ka", np.fft.fft(C, axis=0), np.fft.fft(Xp, axis=0)), axis=0)
    return Y[:R]


# ---------------------------------------------------------------- circulant preconditioner
def strang(T, R):
    """Strang's circulant approximation of the block Toeplitz matrix with blocks T[d] (the
    preconditioner of Appendix B for A_LL): the block circulant whose first block column is
    c_k = T[k] for 0 <= k <= R/2 and c_k = T[k - R] for R/2 < k < R; an offset with no block in T
    gives a zero block.  Returns c (R, m, m)."""
    m = next(iter(T.values())).shape[0]
    c = np.zeros((R, m, m), dtype=np.complex128)
    for k in range(R):
        d = k if k <= R // 2 else k - R
        if d in T:
            c[k] = T[d]
    return c


def chan(T, R):
    """T. Chan's optimal circulant of the block Toeplitz matrix with blocks T[d]: the block
    circulant nearest in the Frobenius norm, c_0 = T[0] and c_k = ((R - k) T[k] + k T[k - R]) / R
    for 0 < k < R (every offset -(R-1) .. R-1 must be in T).  Returns c (R, m, m)."""
    m = T[0].shape[0]
    c = np.zeros((R, m, m), dtype=np.complex128)
    c[0] = T[0]
    for k in range(1, R):
        c[k] = ((R - k) * T[k] + k * T[k - R]) / R
    return c


def circulant_apply(c, xs):
    """y_i = sum_j c[(i - j) mod R] x_j for slice vectors xs (R, m), by the definition."""
    R = len(c)
    ys = np.zeros_like(np.asarray(xs, dtype=np.complex128))
    for i in range(R):
        for j in range(R):
            ys[i] += c[(i - j) % R] @ xs[j]
    return ys


def circulant_solve(c, vs):
    """x with circulant_apply(c, x) = vs: the block DFT over the slice index diagonalises the
    circulant (block f = sum_k c_k exp(-2 pi i f k / R)); one dense solve per frequency."""
    R = len(c)
    ch = np.fft.fft(c, axis=0)
    vh = np.fft.fft(np.asarray(vs, dtype=np.complex128), axis=0)
    xh = np.stack([np.linalg.solve(ch[f], vh[f]) for f in range(R)])
    return np.fft.ifft(xh, axis=0)
