"""Write transition_reflection.txt: the oracle's check of the power law of transition
reflection against absorber length (Sec. IV-B, Eqs. 43 and 45).

A straight guide (0.5 x 0.22 um core, eps 12.1 in eps 2.1, 1.55 um) has a 1.5 um plain section
and an absorber of length L at its right end, the absorber surface graded as
sigma(x) = sigma0 (s)^d, s = (x - 1.5 um) / L (Eq. 23), for d = 0, 1, 2.  The round-trip
reflection is held fixed the way Sec. IV-A asks: the decay rate is proportional to sigma in
the linear range, so the integral of sigma over the absorber, sigma0 L / (d + 1), is held at
K = 40 mS um, and sigma0 = K (d + 1) / L.  A complex-source beam launched at x = 0.3 um along +x
excites the guide; E(L) is the total interior field (three components) at five points of the
axis between x = 0.7 and 1.1 um.  For L = 3, 4, 6, 8 um the record holds the Eq. 45 measure
    m(L) = |E(2L) - E(L)|^2 / |E(L)|^2,
which falls as L^-(2d+2) once L is in the asymptotic range.

The absorbers are long (up to 16 um) so that sigma0 falls into the range where the decay rate
grows in proportion to sigma (below about 10 mS for this guide) while K stays large enough for
the round trip to sit below the measure; the mesh is correspondingly coarse (slices of 0.1 um,
a 2 x 1 cross-section: 12 triangles per slice).  A finer mesh (0.05 um slices, 4 x 2
cross-section) with L = 0.75 .. 2 um and K = 24 mS um gives the same ordering of the slopes but
has sigma0 up to 96 mS, far into the non-linear range, and its slopes are steeper than the law.

Each absorber length is its own closed mesh (six meshes: L = 3, 4, 6, 8, 12, 16 um; the
plain section's slices are the same in all of them).  The oracle's dense operator O1 is
assembled once per mesh for the three profiles (``operator.assemble_many``, rows split over a
pool of spawned worker processes) and solved by LU.  Calls only the oracle and the input
generators; runs for about six minutes on 8 cores.

    python tests/golden/make_transition_reflection.py
"""

import multiprocessing as mp
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import excitation, mesh, operator, post, sigma  # noqa: E402

X0 = 1.5  # interface between the plain section and the absorber [um]
DX = float(os.environ.get("TR_DX", "0.1"))  # slice width [um]
NY, NZ = int(os.environ.get("TR_NY", "2")), int(os.environ.get("TR_NZ", "1"))  # cross-section segments
K_MS_UM = float(os.environ.get("TR_K", "40.0"))  # held integral of sigma over the absorber [mS um]
DS = (0, 1, 2)
LS = tuple(float(v) for v in os.environ.get("TR_LS", "3,4,6,8").split(","))
OUT = os.environ.get("TR_OUT", "transition_reflection.txt")
MEDIA = (12.1, 1.0, 2.1, 1.0, 1.55)
SRC = dict(r0=(0.3, 0.0, 0.0), d=(1, 0, 0), b=0.07, p=(0, 1, 0))
PROBE_X = np.linspace(0.7, 1.1, 5)


def guide(La):
    length = X0 + La
    return synth.waveguide(length, 0.5, 0.22, int(round(length / DX)), NY, NZ, 0.0, La)


def profiles(g, La):
    """Per-point conductivity [S] of each d, sigma0 = K (d + 1) / L."""
    out = []
    for d in DS:
        s0 = K_MS_UM * 1e-3 * (d + 1) / La
        out.append(sigma.monomial(g.qpts, [(X0, La, s0, d, 0, 1)]))
    return out


def _rows_of(g, tris):
    rows = mesh.row_index(g)[g.tri_edge[tris]]
    return np.unique(rows[rows >= 0])


def _work(args):
    from threadpoolctl import threadpool_limits

    La, tris = args
    threadpool_limits(1)
    m = guide(La)
    g = mesh.build(m.V, m.T, m.region, q=6)
    rows = _rows_of(g, tris)
    mats = operator.assemble_many(g, operator.Media(*MEDIA), profiles(g, La), tris=tris, rows_out=rows)
    return rows, mats


def fields(pool, La):
    m = guide(La)
    g = mesh.build(m.V, m.T, m.region, q=6)
    groups = np.array_split(np.arange(g.nt), 48)
    As = [np.zeros((g.N, g.N), dtype=np.complex128) for _ in DS]
    for rows, mats in pool.imap_unordered(_work, [(La, grp) for grp in groups]):
        for A, Mt in zip(As, mats):
            A[rows] += Mt
    med = operator.Media(*MEDIA)
    ki, zi = med.k[1], med.z[1]
    pts = np.stack([PROBE_X, np.full_like(PROBE_X, 0.01), np.full_like(PROBE_X, -0.005)], 1)
    e_inc = excitation.beam(pts, ki, zi, SRC["r0"], SRC["d"], SRC["b"], SRC["p"])[0]
    out = []
    for A, sg in zip(As, profiles(g, La)):
        b = excitation.rhs(g, med, sg, "i", "beam", **SRC)
        x = np.linalg.solve(A, b)
        out.append((post.radiated(g, x, pts, ki, zi, "i") + e_inc).reshape(-1))
    return g, out


def main():
    t0 = time.time()
    Ea = {}
    info = {}
    ctx = mp.get_context("spawn")
    with ctx.Pool(min(8, os.cpu_count() or 1)) as pool:
        for La in sorted(set(LS) | {2 * L for L in LS}):
            g, E = fields(pool, La)
            for d, e in zip(DS, E):
                Ea[(d, La)] = e
            info[La] = (g.nt, g.N)
            print(f"L = {La}: {g.nt} triangles, N = {g.N}, {time.time() - t0:.0f} s", flush=True)
    with open(os.path.join(HERE, OUT), "w") as f:
        f.write("# Transition reflection against absorber length (Sec. IV-B, Eq. 45 of Zhang et al.,\n"
                "# arXiv 1004.5076), from the oracle; written by make_transition_reflection.py.\n"
                "# guide: 1.5 um plain + absorber L, 0.5 x 0.22 um core eps 12.1 in eps 2.1, lambda 1.55 um,\n"
                f"# slices {DX} um, cross-section {NY} x {NZ} segments, sigma = sigma0 s^d, "
                f"sigma0 L / (d + 1) = {K_MS_UM} mS um;\n"
                "# meshes: " + ", ".join(f"L={k}: {v[0]} tri / N={v[1]}" for k, v in sorted(info.items())) + "\n"
                "# columns: d  L_um  m45 = |E(2L)-E(L)|^2/|E(L)|^2  |E(L)|^2\n")
        for d in DS:
            for L in LS:
                e1, e2 = Ea[(d, L)], Ea[(d, 2 * L)]
                n1 = np.vdot(e1, e1).real
                f.write("%d  %5.2f  %.6e  %.6e\n" % (d, L, np.vdot(e2 - e1, e2 - e1).real / n1, n1))
    print(f"done in {time.time() - t0:.0f} s")


if __name__ == "__main__":
    main()
