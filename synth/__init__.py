"""Seeded synthetic inputs shared by the oracle, the tests and the benchmark.

This module only *generates inputs*: closed triangle meshes (vertex
coordinates, triangle vertex indices, per-triangle region flags), seeded random
coefficient vectors, seeded random per-quadrature-point conductivities, and a
placement of the uniform grid around a mesh.  It holds none of the method's
arithmetic: no RWG edge tables, no quadrature, no Green's functions, no
operators.  Both the CUDA path and the oracle consume what it returns and derive
everything else on their own.

Units: lengths in micrometres.  Region flag 0 marks a plain PMCHW surface
(conductivity zero, the paper's "L" surfaces), 1 marks the surface-conductive
absorber ("R" surfaces), as in Sec. II of the paper.
"""

from __future__ import annotations

import dataclasses
import math

import numpy as np

__all__ = [
    "Mesh",
    "icosphere",
    "waveguide",
    "coupler",
    "complex_normal",
    "random_sigma_qpoints",
    "GridSpec",
    "grid_for_mesh",
]


@dataclasses.dataclass
class Mesh:
    """A closed, consistently outward-oriented triangle surface."""

    V: np.ndarray  # (nv, 3) float64 vertex coordinates [um]
    T: np.ndarray  # (nt, 3) int32 vertex indices, counter-clockwise seen from outside
    region: np.ndarray  # (nt,) int32: 0 = plain surface, 1 = absorber surface

    @property
    def nv(self) -> int:
        return int(self.V.shape[0])

    @property
    def nt(self) -> int:
        return int(self.T.shape[0])


def _orient_outward(V: np.ndarray, T: np.ndarray, inside: np.ndarray) -> np.ndarray:
    a, b, c = V[T[:, 0]], V[T[:, 1]], V[T[:, 2]]
    nrm = np.cross(b - a, c - a)
    out = (a + b + c) / 3.0 - inside
    flip = np.einsum("ij,ij->i", nrm, out) < 0
    T = T.copy()
    T[flip, 1], T[flip, 2] = T[flip, 2].copy(), T[flip, 1].copy()
    return T


def icosphere(level: int, radius: float = 1.0, center=(0.0, 0.0, 0.0)) -> Mesh:
    """Icosahedron subdivided ``level`` times, vertices pushed onto the sphere.

    level 2 gives 162 vertices / 320 triangles / 480 edges (the dielectric-sphere
    workload); each level multiplies the triangle count by four.
    """
    t = (1.0 + math.sqrt(5.0)) / 2.0
    V = [
        (-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0),
        (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
        (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1),
    ]
    F = [
        (0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11),
        (1, 5, 9), (5, 11, 4), (11, 10, 2), (10, 7, 6), (7, 1, 8),
        (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9),
        (4, 9, 5), (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1),
    ]
    verts = [np.array(v, dtype=np.float64) / np.linalg.norm(v) for v in V]
    faces = list(F)
    for _ in range(level):
        cache: dict[tuple[int, int], int] = {}

        def mid(i: int, j: int) -> int:
            key = (i, j) if i < j else (j, i)
            if key not in cache:
                m = verts[i] + verts[j]
                verts.append(m / np.linalg.norm(m))
                cache[key] = len(verts) - 1
            return cache[key]

        nf = []
        for (a, b, c) in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    Vn = np.array(verts) * radius + np.asarray(center, dtype=np.float64)
    Tn = np.array(faces, dtype=np.int32)
    Tn = _orient_outward(Vn, Tn, np.asarray(center, dtype=np.float64))
    return Mesh(Vn, Tn, np.zeros(len(Tn), dtype=np.int32))


def _box_surface(x, y, z):
    """Structured triangulation of the surface of the box x[0..nx] * y * z.

    ``x``, ``y``, ``z`` are the sorted node coordinates along each axis.  Each
    face quad is split along the same diagonal; triangles are oriented
    counter-clockwise seen from outside.
    """
    nx, ny, nz = len(x) - 1, len(y) - 1, len(z) - 1
    vid = -np.ones((nx + 1, ny + 1, nz + 1), dtype=np.int64)
    V = []
    for i in range(nx + 1):
        for j in range(ny + 1):
            for k in range(nz + 1):
                if i in (0, nx) or j in (0, ny) or k in (0, nz):
                    vid[i, j, k] = len(V)
                    V.append((x[i], y[j], z[k]))
    V = np.array(V, dtype=np.float64)
    tris = []

    def quads(idx):  # idx: (nu+1, nv+1) vertex ids with u x v = outward normal
        nu, nv = idx.shape[0] - 1, idx.shape[1] - 1
        for a in range(nu):
            for b in range(nv):
                p00, p10, p11, p01 = idx[a, b], idx[a + 1, b], idx[a + 1, b + 1], idx[a, b + 1]
                tris.append((p00, p10, p11))
                tris.append((p00, p11, p01))

    quads(vid[0, :, :].T)        # x = x0, outward -x: u = z, v = y
    quads(vid[nx, :, :])         # x = x1, outward +x: u = y, v = z
    quads(vid[:, 0, :])          # y = y0, outward -y: u = x, v = z
    quads(vid[:, ny, :].T)       # y = y1, outward +y: u = z, v = x
    quads(vid[:, :, 0].T)        # z = z0, outward -z: u = y, v = x
    quads(vid[:, :, nz])         # z = z1, outward +z: u = x, v = y
    return V, np.array(tris, dtype=np.int32)


def waveguide(
    length: float = 12.0,
    width: float = 0.5,
    height: float = 0.22,
    nx: int = 300,
    ny: int = 11,
    nz: int = 5,
    absorber_left: float = 4.0,
    absorber_right: float = 4.0,
    x0: float = 0.0,
) -> Mesh:
    """Straight rectangular guide along x with closed end caps.

    The guide spans x in [x0, x0+length], |y| <= width/2, |z| <= height/2.
    Triangles whose centroid lies within ``absorber_left`` of the left end or
    ``absorber_right`` of the right end get region flag 1 (absorber); this
    includes both end caps when the absorber lengths are positive.
    The defaults give the 12 um guide of 19,420 triangles with 4 um absorbers at
    both ends.
    """
    xs = x0 + np.linspace(0.0, length, nx + 1)
    ys = np.linspace(-width / 2, width / 2, ny + 1)
    zs = np.linspace(-height / 2, height / 2, nz + 1)
    V, T = _box_surface(xs, ys, zs)
    cx = V[T].mean(axis=1)[:, 0]
    region = np.zeros(len(T), dtype=np.int32)
    if absorber_left > 0:
        region[cx < x0 + absorber_left] = 1
    if absorber_right > 0:
        region[cx > x0 + length - absorber_right] = 1
    return Mesh(V, T, region)


def coupler(
    length: float = 40.0,
    width: float = 0.5,
    height: float = 0.22,
    gap: float = 0.2,
    nx: int = 1000,
    ny: int = 11,
    nz: int = 5,
    absorber: float = 4.0,
) -> Mesh:
    """Two parallel guides separated by ``gap`` along y (a directional coupler)."""
    off = (width + gap) / 2
    meshes = [waveguide(length, width, height, nx, ny, nz, absorber, absorber) for _ in range(2)]
    Vs, Ts, Rs, base = [], [], [], 0
    for m, dy in zip(meshes, (-off, off)):
        V = m.V.copy()
        V[:, 1] += dy
        Vs.append(V)
        Ts.append(m.T + base)
        Rs.append(m.region)
        base += len(V)
    return Mesh(np.concatenate(Vs), np.concatenate(Ts).astype(np.int32), np.concatenate(Rs))


def complex_normal(n: int, nrhs: int | None = None, seed: int = 0) -> np.ndarray:
    """Seeded standard complex normal vector (or n x nrhs matrix), complex128."""
    rng = np.random.default_rng(seed)
    shape = (n,) if nrhs is None else (n, nrhs)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def two_wave_samples(npts: int, t0: float, t1: float, alpha: float, beta: float, a: complex, c: complex,
                     noise: float = 0.0, seed: int = 0):
    """Samples t_k (uniform on [t0, t1]) and E_k = a exp(-g tau_k) + c exp(g tau_k) + noise, with
    g = alpha + j beta and tau measured from the midpoint of [t0, t1]; the noise is complex normal
    with standard deviation ``noise`` times the largest |E_k|."""
    t = np.linspace(t0, t1, npts)
    tau = t - 0.5 * (t0 + t1)
    g = alpha + 1j * beta
    E = a * np.exp(-g * tau) + c * np.exp(g * tau)
    if noise > 0:
        E = E + noise * np.max(np.abs(E)) * complex_normal(npts, seed=seed)
    return t, E


def random_sigma_qpoints(nt: int, q: int, region: np.ndarray, scale: float, seed: int = 0) -> np.ndarray:
    """Seeded non-negative conductivities [S], one per (triangle, quadrature point).

    Zero on plain (region 0) triangles, uniform in [0, scale] on absorber ones.
    """
    rng = np.random.default_rng(seed)
    s = rng.uniform(0.0, scale, size=(nt, q))
    s[np.asarray(region) == 0] = 0.0
    return s


@dataclasses.dataclass
class GridSpec:
    """Uniform grid: physical dims n (the FFT transform is 2n per axis)."""

    n: tuple[int, int, int]  # physical points per axis (x, y, z)
    h: float  # spacing [um]
    origin: tuple[float, float, float]  # coordinate of grid point (0,0,0)
    p: int  # stencil points per axis

    @property
    def padded(self) -> tuple[int, int, int]:
        return tuple(2 * v for v in self.n)


_OFFSETS = (0.2360679774997897, 0.3819660112501051, 0.1458980337503155)


def grid_for_mesh(V: np.ndarray, padded, p: int = 3, h: float | None = None) -> GridSpec:
    """Place a grid of transform size ``padded`` (physical = padded/2) around V.

    The spacing is the smallest that keeps every stencil inside the physical
    grid (unless ``h`` is given); the origin carries small irrational offsets
    so that no point of a structured mesh lands on a cell boundary.
    """
    n = tuple(int(v) // 2 for v in padded)
    lo, hi = V.min(axis=0), V.max(axis=0)
    ext = hi - lo
    if h is None:
        h = float(max(ext[a] / (n[a] - p - 1.5) for a in range(3)))
    mid = (lo + hi) / 2
    origin = tuple(float(mid[a] - h * ((n[a] - 1) / 2.0 - _OFFSETS[a])) for a in range(3))
    return GridSpec(n=n, h=h, origin=origin, p=p)
