"""Write decay_rate_vs_sigma.txt: the oracle's decay rate of the guided field under a uniform
surface conductivity, for a range of conductivities (the study of Sec. III).

A 2.4 um guide (0.5 x 0.22 um core, eps 12.1 in eps 2.1, 1.55 um) whose surface is absorber
everywhere except the far end cap carries a complex-source beam launched at x = 0.3 um.  For every
sigma the oracle's dense operator (O1, assembled once at sigma = 0 and once at sigma = 1/eta0 S;
the operator is affine in sigma) is solved by LU, the interior field E_y is evaluated at 33 points
of the axis between x = 0.6 and 1.4 um, and the decay-rate fit of Sec. III
(a exp(-g tau) + c exp(g tau), g = alpha + j beta) is taken over alpha in [0, 12] /um (step 0.1)
and beta in [4, 16] rad/um (step 0.2).  The decay rate by Poynting's theorem (Sec. III-B) is taken
at the cross-section x = 1.025 um (the middle of one mesh slice) over the box |y| <= 0.6,
|z| <= 0.5 um.  Calls only the oracle and the input generators; runs for about seven minutes.

    python tests/golden/make_decay_rate_vs_sigma.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle import ETA0, excitation, mesh, operator, post  # noqa: E402

SIGMAS_MS = [0.0, 0.5, 1.0, 2.0, 4.0, 8.0, 16.0, 32.0, 64.0, 128.0, 256.0, 1024.0]


def main():
    m = synth.waveguide(2.4, 0.5, 0.22, 48, 4, 2, 2.4, 0.0)
    g = mesh.build(m.V, m.T, m.region, q=6)
    med = operator.Media(12.1, 1.0, 2.1, 1.0, 1.55)
    z0 = np.zeros((g.nt, g.q))
    A0 = operator.assemble(g, med, z0)
    A1 = operator.assemble(g, med, z0 + 1.0 / ETA0) - A0
    ki, zi = med.k[1], med.z[1]
    src = dict(r0=(0.3, 0.0, 0.0), d=(1, 0, 0), b=0.07, p=(0, 1, 0))
    ts = np.linspace(0.6, 1.4, 33)
    pts = np.stack([ts, np.full_like(ts, 0.01), np.full_like(ts, -0.005)], 1)
    e_inc = excitation.beam(pts, ki, zi, src["r0"], src["d"], src["b"], src["p"])[0][:, 1]
    rows = []
    for s_ms in SIGMAS_MS:
        s = s_ms * 1e-3
        x = np.linalg.solve(A0 + (s * ETA0) * A1, excitation.rhs(g, med, z0 + s, "i", "beam", **src))
        E = post.radiated(g, x, pts, ki, zi, "i")[:, 1] + e_inc
        al, bt, res, a, c = post.fit_decay(ts, E, np.linspace(0.0, 12.0, 121), np.linspace(4.0, 16.0, 61))
        ap = post.poynting_decay_rate(g, x, med, s, 1.025, (0.25, 0.11), (0.6, 0.5), 0.025,
                                      inc=lambda q: excitation.beam(q, ki, zi, src["r0"], src["d"], src["b"],
                                                                    src["p"]), n=8)[0]
        rows.append((s_ms, al, ap, bt, res, abs(c / a)))
    with open(os.path.join(HERE, "decay_rate_vs_sigma.txt"), "w") as f:
        f.write("# Decay rate of the field in a guide with uniform surface conductivity (Sec. III of Zhang\n"
                "# et al., arXiv 1004.5076), from the oracle; written by make_decay_rate_vs_sigma.py.\n"
                f"# guide 2.4 um, 0.5 x 0.22 um core eps 12.1 in eps 2.1, lambda 1.55 um, {g.nt} triangles, "
                f"N = {g.N}\n"
                "# columns: sigma_mS  alpha_fit_per_um  alpha_poynting_per_um  beta_rad_per_um  "
                "fit_rel_residual  |c/a|\n")
        for r in rows:
            f.write("%9.2f  %6.2f  %7.3f  %6.2f  %.4f  %.4f\n" % r)


if __name__ == "__main__":
    main()
