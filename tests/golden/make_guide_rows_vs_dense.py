"""Write guide_rows_vs_dense.txt: the grid operator's definition (O2) against the exact dense
operator (O1) on every plain-surface row of the 12 um guide's periodic section.

The guide of the benchmark (19,420 triangles; x in [4, 8] um carries no absorber) has 100 regular
slices of 192 unknowns there.  O1 restricted to them is block Toeplitz (Appendix B): two block rows
of O1 entries give every block (oracle/toeplitz.py), and the product with a seeded x supported on
those slices gives the exact rows.  O2 (oracle/pfft.py) is evaluated on the same targets at the
benchmark's near radius (2.05 grid steps) and at 3.05.  The CUDA operator equals O2 to 1e-5
(complex64), so these are the benchmark operator's errors against the exact one on all 19,200
rows.  Calls only the oracle and the input generators; about 45 minutes on one host.

    python tests/golden/make_guide_rows_vs_dense.py
"""

import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)
sys.path.insert(0, os.path.dirname(HERE))

import cases  # noqa: E402
import synth  # noqa: E402
from oracle import mesh, operator, pfft, toeplitz  # noqa: E402


def main():
    case = cases.guide_full()
    g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
    sig = cases.sigma_points(case, g.qpts)
    med = operator.Media(*case.media)
    lay = toeplitz.SliceLayout(g, 0.0, 12.0 / 300, 300, first=100, count=100)
    T = toeplitz.blocks(g, med, sig, lay)
    xs = synth.complex_normal(lay.count * lay.m, seed=21).reshape(lay.count, lay.m)
    x = np.zeros(g.N, dtype=np.complex128)
    for k in range(lay.count):
        idx, sg = lay.unknowns(g, k)
        x[idx] = sg * xs[k]
    ys = toeplitz.apply(T, xs)
    tris = np.unique(np.concatenate([g.edge_t[e].reshape(-1) for e in lay.edges]))
    out = []
    for fh in (2.05, 3.05):
        y2 = pfft.PFFT(g, med, case.grid, fh * case.grid.h).apply(x, sig, targets=tris)
        num = den = worst = 0.0
        for k in range(lay.count):
            idx, sg = lay.unknowns(g, k)
            d = sg * y2[idx] - ys[k]
            num += np.vdot(d, d).real
            den += np.vdot(ys[k], ys[k]).real
            worst = max(worst, np.abs(d).max())
        amax = max(np.abs(v).max() for v in ys)
        out.append((fh, lay.count * lay.m, np.sqrt(num / den), worst / amax))
    with open(os.path.join(HERE, "guide_rows_vs_dense.txt"), "w") as f:
        f.write("# O2 (grid operator definition) against O1 (exact, block-Toeplitz product) on every plain-\n"
                "# surface row of the 12 um guide's periodic section (x in [4, 8] um), p = 3, q = 6, x random on\n"
                "# those slices; written by make_guide_rows_vs_dense.py.\n"
                "# columns: near_radius_in_grid_steps  rows  rel_l2_error  max_entry_error_over_max_entry\n")
        for r in out:
            f.write("%.2f  %d  %.4e  %.4e\n" % r)


if __name__ == "__main__":
    main()
