"""Write mie_refinement.txt: the far-field error of the oracle's dense PMCHW solution of the
dielectric sphere (r = 1 um, eps 2.25 in vacuum, 1.55 um, x-polarised plane wave along z) against
the Mie series, on icospheres of 80, 320 and 1280 triangles, for plain PMCHW and for the
all-absorber rows with a conducting sheet (sigma = 1/eta0 S).  The error is the larger of the
relative l2 errors of |F_theta| (phi = 0) and |F_phi| (phi = 90 deg) over 25 angles.  Calls only
the oracle and the input generators; about five minutes on one core.

    python tests/golden/make_mie_refinement.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import ETA0, excitation, mesh, mie, operator, post  # noqa: E402


def far_error(level, region_R, sigma_S):
    m = synth.icosphere(level, 1.0)
    reg = np.ones(m.nt, int) if region_R else m.region
    g = mesh.build(m.V, m.T, reg, q=6)
    med = operator.Media(2.25, 1.0, 1.0, 1.0, 1.55)
    sig = np.full((g.nt, g.q), sigma_S)
    x = np.linalg.solve(operator.assemble(g, med, sig),
                        excitation.rhs(g, med, sig, "e", "planewave", d=[0, 0, 1], e=[1, 0, 0]))
    ke, ze = med.k[0], med.z[0]
    th = np.linspace(0.01, np.pi - 0.01, 25)
    r0 = np.stack([np.sin(th), 0 * th, np.cos(th)], 1)
    r90 = np.stack([0 * th, np.sin(th), np.cos(th)], 1)
    thh = np.stack([np.cos(th), 0 * th, -np.sin(th)], 1)
    f_th = np.abs(np.sum(post.far_field(g, x, ke, ze, r0) * thh, 1))
    f_ph = np.abs(post.far_field(g, x, ke, ze, r90)[:, 0])
    S1, S2 = mie.amplitudes(1.5, ke * 1.0, th, s=sigma_S * ETA0 * ze)
    e2 = np.linalg.norm(f_th - np.abs(S2) / ke) / np.linalg.norm(np.abs(S2) / ke)
    e1 = np.linalg.norm(f_ph - np.abs(S1) / ke) / np.linalg.norm(np.abs(S1) / ke)
    return g.nt, g.N, max(e1, e2)


def main():
    rows = []
    for level in (1, 2, 3):
        for name, region_R, s in (("plain", False, 0.0), ("sheet", True, 1.0 / ETA0)):
            nt, N, err = far_error(level, region_R, s)
            rows.append((level, nt, N, name, err))
            print(level, nt, N, name, err, flush=True)
    with open(os.path.join(HERE, "mie_refinement.txt"), "w") as f:
        f.write("# Far-field error of the oracle's dense PMCHW solution of the dielectric sphere against the\n"
                "# Mie series under mesh refinement; written by make_mie_refinement.py.\n"
                "# columns: level  triangles  unknowns  rows(plain|sheet)  max_rel_far_field_error\n")
        for r in rows:
            f.write("%d  %5d  %5d  %s  %.5f\n" % r)


if __name__ == "__main__":
    main()
