"""Triangle geometry, quadrature, RWG edges and the unknown layout.

RWG basis (Appendix A, Eqs. RWGJ/RWGM of the paper): the basis function of
interior edge m with length l_m, shared by triangles T+ and T- with free
vertices p+ and p-, is

    X_m(r) = +l_m / (2 A+) (r - p+)   on T+,
    X_m(r) = -l_m / (2 A-) (r - p-)   on T-,          div X_m = +-l_m / A+-.

Canonical edge order (shared convention with the CUDA path, stated in the C
header): undirected edges sorted by (min vertex, max vertex); T+ is the
triangle in which the edge is traversed min -> max in its counter-clockwise
vertex cycle.  Local edge k of a triangle is the edge opposite its vertex k.

Edge classes (Sec. II): an edge is an absorber ("R") edge iff both of its
triangles carry region flag 1; otherwise it is a plain ("L") edge.  Unknowns:

    x = [J^L (E_L), M^L (E_L), J_e^R (E_R), J_i^R (E_R), M^R (E_R)]

with the per-class edge order inherited from the canonical order.  Rows of
A x = b follow the same blocks: Eq. 1 (E, L edges), Eq. 2 (H, L edges),
Eq. 3 (E, R edges), Eq. 13 (R edges), Eq. 14 (R edges).
"""

from __future__ import annotations

import dataclasses

import numpy as np

# Symmetric triangle rules (Dunavant 1985): barycentric coordinates and weights
# normalised to sum to one.  Point order is part of the interface (per-point
# conductivities are indexed by it).
_A6, _B6 = 0.445948490915965, 0.091576213509771
_W6A, _W6B = 0.223381589678011, 0.109951743655322
_A7, _B7 = 0.059715871789770, 0.470142064105115
_C7, _D7 = 0.797426985353087, 0.101286507323456
RULES = {
    1: (np.array([[1 / 3, 1 / 3, 1 / 3]]), np.array([1.0])),
    3: (
        np.array([[2 / 3, 1 / 6, 1 / 6], [1 / 6, 2 / 3, 1 / 6], [1 / 6, 1 / 6, 2 / 3]]),
        np.array([1 / 3, 1 / 3, 1 / 3]),
    ),
    6: (
        np.array(
            [
                [1 - 2 * _A6, _A6, _A6], [_A6, 1 - 2 * _A6, _A6], [_A6, _A6, 1 - 2 * _A6],
                [1 - 2 * _B6, _B6, _B6], [_B6, 1 - 2 * _B6, _B6], [_B6, _B6, 1 - 2 * _B6],
            ]
        ),
        np.array([_W6A] * 3 + [_W6B] * 3),
    ),
    7: (
        np.array(
            [
                [1 / 3, 1 / 3, 1 / 3],
                [_A7, _B7, _B7], [_B7, _A7, _B7], [_B7, _B7, _A7],
                [_C7, _D7, _D7], [_D7, _C7, _D7], [_D7, _D7, _C7],
            ]
        ),
        np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3),
    ),
}


@dataclasses.dataclass
class Geometry:
    """Per-triangle geometry, RWG edge table and unknown layout of one mesh."""

    V: np.ndarray
    T: np.ndarray
    region: np.ndarray
    area: np.ndarray  # (nt,)
    normal: np.ndarray  # (nt, 3) unit outward normal
    centroid: np.ndarray  # (nt, 3)
    # edges
    edge_v: np.ndarray  # (ne, 2) vertex ids (min, max)
    edge_t: np.ndarray  # (ne, 2) triangles (T+, T-)
    edge_len: np.ndarray  # (ne,)
    edge_class: np.ndarray  # (ne,) 0 = L, 1 = R
    edge_cidx: np.ndarray  # (ne,) index within its class
    # per triangle local edges
    tri_edge: np.ndarray  # (nt, 3) edge id of local edge k (opposite vertex k)
    tri_sign: np.ndarray  # (nt, 3) +1 if the triangle is T+ of that edge, else -1
    # quadrature
    q: int
    qpts: np.ndarray  # (nt, q, 3)
    qw: np.ndarray  # (nt, q) weights including the area

    @property
    def nt(self):
        return int(self.T.shape[0])

    @property
    def ne(self):
        return int(self.edge_v.shape[0])

    @property
    def nL(self):
        return int(np.sum(self.edge_class == 0))

    @property
    def nR(self):
        return int(np.sum(self.edge_class == 1))

    @property
    def N(self):
        return 2 * self.nL + 3 * self.nR

    # offsets of the five unknown / row blocks
    def block(self, name: str) -> int:
        nL, nR = self.nL, self.nR
        return {"JL": 0, "ML": nL, "JeR": 2 * nL, "JiR": 2 * nL + nR, "MR": 2 * nL + 2 * nR}[name]


def build(V, T, region, q: int = 6) -> Geometry:
    V = np.asarray(V, dtype=np.float64)
    T = np.asarray(T, dtype=np.int64)
    region = np.asarray(region, dtype=np.int64)
    nt = len(T)
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    cr = np.cross(b - a, c - a)
    nrm = np.linalg.norm(cr, axis=1)
    if np.any(nrm <= 0):
        raise ValueError("degenerate triangle")
    area = 0.5 * nrm
    normal = cr / nrm[:, None]
    centroid = (a + b + c) / 3.0

    # directed edges: local edge k goes from vertex k+1 to vertex k+2
    directed = {}
    for t in range(nt):
        for k in range(3):
            u, w = int(T[t, (k + 1) % 3]), int(T[t, (k + 2) % 3])
            if (u, w) in directed:
                raise ValueError("non-manifold or inconsistently oriented mesh")
            directed[(u, w)] = (t, k)
    keys = sorted({(min(u, w), max(u, w)) for (u, w) in directed})
    ne = len(keys)
    edge_v = np.array(keys, dtype=np.int64)
    edge_t = np.zeros((ne, 2), dtype=np.int64)
    tri_edge = np.zeros((nt, 3), dtype=np.int64)
    tri_sign = np.zeros((nt, 3), dtype=np.int64)
    for e, (u, w) in enumerate(keys):
        if (u, w) not in directed or (w, u) not in directed:
            raise ValueError("open mesh: every edge must be shared by two triangles")
        tp, kp = directed[(u, w)]
        tm, km = directed[(w, u)]
        edge_t[e] = (tp, tm)
        tri_edge[tp, kp], tri_sign[tp, kp] = e, 1
        tri_edge[tm, km], tri_sign[tm, km] = e, -1
    edge_len = np.linalg.norm(V[edge_v[:, 1]] - V[edge_v[:, 0]], axis=1)
    edge_class = ((region[edge_t[:, 0]] == 1) & (region[edge_t[:, 1]] == 1)).astype(np.int64)
    edge_cidx = np.zeros(ne, dtype=np.int64)
    for cls in (0, 1):
        sel = np.nonzero(edge_class == cls)[0]
        edge_cidx[sel] = np.arange(len(sel))

    bary, wts = RULES[q]
    qpts = np.einsum("qi,tij->tqj", bary, V[T])
    qw = wts[None, :] * area[:, None]
    return Geometry(
        V=V, T=T, region=region, area=area, normal=normal, centroid=centroid,
        edge_v=edge_v, edge_t=edge_t, edge_len=edge_len, edge_class=edge_class,
        edge_cidx=edge_cidx, tri_edge=tri_edge, tri_sign=tri_sign, q=q, qpts=qpts, qw=qw,
    )


def edge_coefficients(g: Geometry, x: np.ndarray):
    """Per-edge coefficients of the exterior J, interior J and exterior M sets.

    Current reduction (Eqs. 10-12): on L edges J_e = J^L, J_i = -J^L,
    M_e = M^L; on R edges J_e = J_e^R, J_i = J_i^R, M_e = M^R.  The interior
    magnetic current is always M_i = -M_e.  ``x`` may carry a trailing batch
    dimension.
    """
    x = np.asarray(x)
    L = g.edge_class == 0
    ci = g.edge_cidx
    shape = (g.ne,) + x.shape[1:]
    Je = np.zeros(shape, dtype=np.complex128)
    Ji = np.zeros(shape, dtype=np.complex128)
    Me = np.zeros(shape, dtype=np.complex128)
    Je[L] = x[g.block("JL") + ci[L]]
    Ji[L] = -x[g.block("JL") + ci[L]]
    Me[L] = x[g.block("ML") + ci[L]]
    R = ~L
    Je[R] = x[g.block("JeR") + ci[R]]
    Ji[R] = x[g.block("JiR") + ci[R]]
    Me[R] = x[g.block("MR") + ci[R]]
    return Je, Ji, Me


def row_index(g: Geometry):
    """Row of each (edge, row type) pair; -1 where that row does not exist.

    Row types: 0 = tangential E (Eq. 1 on L edges, Eq. 3 on R edges),
    1 = tangential H (Eq. 2, L edges), 2 = Eq. 13 (R), 3 = Eq. 14 (R).
    """
    rows = -np.ones((g.ne, 4), dtype=np.int64)
    L = g.edge_class == 0
    ci = g.edge_cidx
    rows[L, 0] = g.block("JL") + ci[L]
    rows[L, 1] = g.block("ML") + ci[L]
    R = ~L
    rows[R, 0] = g.block("JeR") + ci[R]
    rows[R, 2] = g.block("JiR") + ci[R]
    rows[R, 3] = g.block("MR") + ci[R]
    return rows
