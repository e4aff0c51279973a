"""Seeded test workloads shared by the parity tests, smoke() and bench.py.

Each case fixes a mesh (synth), media, grid, conductivity and excitation.  The
CUDA operator and the oracle are both built from exactly these inputs.
"""

from __future__ import annotations

import dataclasses

import numpy as np

import synth


@dataclasses.dataclass
class Case:
    name: str
    mesh: synth.Mesh
    media: tuple  # eps_i, mu_i, eps_e, mu_e, lambda0
    grid: synth.GridSpec
    q: int
    r_near: float
    sigma_segments: list | None = None
    sigma_scale: float = 0.0  # random per-point conductivity [S] when > 0
    seed: int = 0
    transverse: str = "auto"  # (y, z) convolution: "auto", "fft" planes or "direct" sums
    sigma_bspline: tuple | None = None  # (x0, L, axis, coef [S]): cubic B-spline profile


def sphere_mixed(level=2, padded=(32, 32, 32), p=3, q=6, r_near=0.5):
    """Dielectric sphere (r = 1 um, eps 2.25 in vacuum, 1.55 um) with an absorber cap x > 0.2."""
    m = synth.icosphere(level, 1.0)
    reg = (m.V[m.T].mean(1)[:, 0] > 0.2).astype(np.int32)
    m = synth.Mesh(m.V, m.T, reg)
    grid = synth.grid_for_mesh(m.V, padded, p=p)
    return Case("sphere_mixed", m, (2.25, 1.0, 1.0, 1.0, 1.55), grid, q, r_near, sigma_scale=0.003, seed=11)


def guide_small(nx=40, ny=6, nz=3, length=2.0, absorber=0.6, padded=(64, 32, 16), p=3, q=6, r_near=0.16, d=2):
    """Short silicon-like guide (eps 12.1 in 2.1) with monomial absorbers at both ends."""
    m = synth.waveguide(length, 0.5, 0.22, nx, ny, nz, absorber, absorber)
    grid = synth.grid_for_mesh(m.V, padded, p=p)
    s0 = 0.004
    segs = [
        (length - absorber, absorber, s0, d, 0, 1.0),
        (absorber, absorber, s0, d, 0, -1.0),
    ]
    return Case("guide_small", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, q, r_near, sigma_segments=segs, seed=12)


def guide_planes64():
    """guide_small on a 64 x 64 x 64 transform grid (64 x 64 cross-section planes)."""
    c = guide_small(padded=(64, 64, 64))
    c.name = "guide_planes64"
    return c


def guide_planes64_fft():
    """guide_planes64 with the (y, z) convolution forced onto the 64 x 64 FFT planes."""
    c = guide_planes64()
    c.name = "guide_planes64_fft"
    c.transverse = "fft"
    return c


def sphere_direct():
    """sphere_mixed with the (y, z) convolution forced to direct sums over its active columns."""
    c = sphere_mixed()
    c.name = "sphere_direct"
    c.transverse = "direct"
    return c


def plate_thin(padded=(32, 16, 8), p=2, q=3, r_near=0.3):
    """Flat thin box with a one-sided absorber: exercises p = 2 stencils and the 3-point rule."""
    m = synth.waveguide(1.5, 0.3, 0.1, 10, 3, 1, 0.4, 0.0)
    grid = synth.grid_for_mesh(m.V, padded, p=p)
    return Case("plate_thin", m, (4.0, 1.0, 1.5, 1.0, 1.3), grid, q, r_near, sigma_scale=0.002, seed=13)


def plate_p4_q7():
    """plate_thin with p = 4 stencils (64 points) and the 7-point rule (28 lanes per triangle)."""
    c = plate_thin(padded=(32, 16, 16), p=4, q=7, r_near=0.12)
    c.name = "plate_p4_q7"
    return c


def plate_q1():
    """plate_thin with p = 3 stencils and the 1-point rule (4 lanes per triangle)."""
    c = plate_thin(p=3, q=1)
    c.name = "plate_q1"
    return c


def guide_short(ncoef=16, sigma0=0.004, seed=1234):
    """A 1.6 um guide (416 triangles, N = 1,572) with 0.4 um absorber regions at both ends and a
    conductivity given as a cubic B-spline of ncoef coefficients over the whole guide, uniform in
    [0, 2 sigma0] (seeded); small enough for the oracle to assemble its grid operator column by
    column and solve it by LU."""
    m = synth.waveguide(1.6, 0.5, 0.22, 16, 4, 2, 0.4, 0.4)
    grid = synth.grid_for_mesh(m.V, (32, 16, 16), p=3)
    coef = np.random.default_rng(seed).uniform(0.0, 2 * sigma0, ncoef)
    return Case("guide_short", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, 6, 0.2, seed=14,
                sigma_bspline=(0.0, 1.6, 0, coef))


def guide_2k(ncoef=16, sigma0=0.004, seed=1234):
    """A 4 um guide of 1,952 triangles with 1 um absorber regions at both ends and a 16-coefficient
    cubic B-spline conductivity over the whole guide, uniform in [0, 2 sigma0] (seeded)."""
    m = synth.waveguide(4.0, 0.5, 0.22, 80, 4, 2, 1.0, 1.0)
    grid = synth.grid_for_mesh(m.V, (128, 16, 16), p=3)
    coef = np.random.default_rng(seed).uniform(0.0, 2 * sigma0, ncoef)
    return Case("guide_2k", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, 6, 2.05 * grid.h, seed=15,
                sigma_bspline=(0.0, 4.0, 0, coef))


def guide_full(p=3, q=6, r_near=None):
    """The 12 um guide: 0.5 x 0.22 um core (eps 12.1) in eps 2.1, 4 um absorbers
    sigma0 (x/L)^3 at both ends, 19,420 triangles, FFT grid 512 x 64 x 64."""
    m = synth.waveguide()
    grid = synth.grid_for_mesh(m.V, (512, 64, 64), p=p)
    if r_near is None:
        r_near = 2.05 * grid.h
    L = 4.0
    s0 = 0.002 * (4.0 / L) * 4  # (p+1) with p = d+1 = 3
    segs = [(12.0 - L, L, s0, 3, 0, 1.0), (L, L, s0, 3, 0, -1.0)]
    return Case("guide_12um", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, q, r_near, sigma_segments=segs, seed=0)


def coupler_full(p=3, q=6, r_near=None):
    """Two 40 um guides 0.2 um apart (a directional coupler) with 4 um absorbers sigma0 (x/L)^3 at
    all four ports, 128,440 triangles, FFT grid 1024 x 256 x 256 (the (y, z) convolution runs as
    direct sums over the active columns)."""
    m = synth.coupler()
    grid = synth.grid_for_mesh(m.V, (1024, 256, 256), p=p)
    if r_near is None:
        r_near = 2.05 * grid.h
    L, length = 4.0, 40.0
    s0 = 0.008
    segs = [(length - L, L, s0, 3, 0, 1.0), (L, L, s0, 3, 0, -1.0)]
    return Case("coupler_40um", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, q, r_near, sigma_segments=segs, seed=0)


def sigma_points(case: Case, qpts):
    """Conductivity [S] at the quadrature points (nt, q) for a case."""
    from oracle import sigma as osig  # the oracle evaluates the profile on its side

    if case.sigma_bspline is not None:
        x0, L, axis, coef = case.sigma_bspline
        return osig.bspline(qpts, x0, L, coef, axis)
    if case.sigma_segments:
        return osig.monomial(qpts, case.sigma_segments)
    if case.sigma_scale > 0:
        return synth.random_sigma_qpoints(case.mesh.nt, case.q, case.mesh.region, case.sigma_scale, case.seed)
    return np.zeros(qpts.shape[:2])
