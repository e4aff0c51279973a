"""The GPU operator against the exact operator on every row of a periodic section.

On a straight extruded guide the plain-surface block A_LL of the exact
operator O1 is block Toeplitz over the regular slices (Appendix B); the
oracle's block-Toeplitz product (two block rows of O1 entries, circulant
embedding) gives its exact rows for a vector supported on those slices.  The
GPU's grid operator is compared with them on every row of the plain section
of a short guide with absorbers at both ends: its error there is the grid
method's discretisation error, the same as that of the oracle's grid operator
O2 (which the GPU matches to 1e-10 in complex128 and 1e-5 in complex64).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth
import paper_1004_5076_gb300 as sc
from oracle import mesh, operator, toeplitz
from oracle import sigma as osig

pytestmark = pytest.mark.gpu

NX, LEN = 20, 2.0


@pytest.fixture(scope="module")
def periodic():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m = synth.waveguide(LEN, 0.5, 0.22, NX, 4, 2, 0.5, 0.5)
    g = mesh.build(m.V, m.T, m.region, q=6)
    med = operator.Media(12.1, 1.0, 2.1, 1.0, 1.55)
    segs = [(1.5, 0.5, 0.004, 2, 0, 1.0), (0.5, 0.5, 0.004, 2, 0, -1.0)]
    sig = osig.monomial(g.qpts, segs)
    # the plain section is x in [0.5, 1.5] um: slices 5 .. 14; 6 .. 13 join plain triangles only
    lay = toeplitz.SliceLayout(g, 0.0, LEN / NX, NX, first=6, count=8)
    T = toeplitz.blocks(g, med, sig, lay)
    xs = synth.complex_normal(lay.count * lay.m, seed=33).reshape(lay.count, lay.m)
    x = np.zeros(g.N, dtype=np.complex128)
    for k in range(lay.count):
        idx, sgn = lay.unknowns(g, k)
        x[idx] = sgn * xs[k]
    ys = toeplitz.apply(T, xs)
    grid = synth.grid_for_mesh(m.V, (64, 16, 16), p=3)
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    yield m, g, med, sig, segs, lay, x, ys, grid, mh
    sc.scabem_mesh_destroy(mh)


def _rows(lay, g, y):
    return [lay.unknowns(g, k)[1] * y[lay.unknowns(g, k)[0]] for k in range(lay.count)]


_err = {}


@pytest.mark.parametrize("near_h", [2.05, 3.05])
@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_gpu_operator_on_every_row_of_the_periodic_section(periodic, near_h, prec):
    """Relative error of the GPU operator on all 576 rows of the regular slices against the exact
    rows: below 10% at a near radius of 2.05 grid steps and 5% at 3.05 (the oracle's own grid
    operator O2 measures 7.0% and 3.6% on this case), smaller at the larger radius, and the same
    in complex64 and complex128 (it is the grid method's error, not rounding)."""
    m, g, med, sig, segs, lay, x, ys, grid, mh = periodic
    r_near = near_h * grid.h
    op = sc.scabem_op_create(mh, (12.1, 1.0, 2.1, 1.0, 1.55), grid.n, grid.h, grid.origin, 3, 6, r_near, 3)
    sc.scabem_set_sigma(op, segments=segs)
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    xt = torch.as_tensor(x).to(dt).cuda().contiguous()
    yt = torch.empty_like(xt)
    sc.scabem_apply(op, xt, yt, prec=prec)
    torch.cuda.synchronize()
    y = yt.cpu().numpy().astype(np.complex128)
    sc.scabem_op_destroy(op)
    gpu, exact = np.concatenate(_rows(lay, g, y)), np.concatenate(ys)
    assert len(exact) == lay.count * lay.m == 576  # every row of the regular slices
    err = np.linalg.norm(gpu - exact) / np.linalg.norm(exact)
    _err[(near_h, prec)] = err
    assert err < (0.1 if near_h < 3 else 0.05), err
    if (2.05, prec) in _err and (3.05, prec) in _err:
        assert _err[(3.05, prec)] < _err[(2.05, prec)]
    other = sc.SCABEM_C64 if prec == sc.SCABEM_C128 else sc.SCABEM_C128
    if (near_h, other) in _err:
        assert abs(_err[(near_h, other)] - err) <= 1e-4 * err
