"""Conductivity profiles on the GPU: the cubic B-spline kind (Eq. 23 in a
smooth basis) evaluated by the CUDA set-up against the oracle's profile."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import mesh, operator, pfft
from oracle import sigma as osig

pytestmark = pytest.mark.gpu

TOL64 = 1e-10


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _apply(op, x, prec=sc.SCABEM_C128):
    xt = torch.as_tensor(x).to(torch.complex128).cuda().contiguous()
    yt = torch.empty_like(xt)
    sc.scabem_apply(op, xt, yt, prec=prec)
    torch.cuda.synchronize()
    return yt.cpu().numpy()


def test_bspline_profile_matches_oracle_values_and_operator():
    """BSPLINE on the device equals PER_QPOINT with the oracle's B-spline
    values (to rounding), and the resulting operator matches O2."""
    case = cases.guide_small()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 2)
    try:
        g = mesh.build(m.V, m.T, m.region, q=case.q)
        coef = np.random.default_rng(1234).uniform(0.0, 2 * 0.004, 16)
        x0, L = float(m.V[:, 0].min()), float(np.ptp(m.V[:, 0]))
        sig = osig.bspline(g.qpts, x0, L, coef, axis=0)
        assert sig.max() > 0.0
        x = cases.synth.complex_normal(g.N, seed=77)
        sc.scabem_set_sigma(op, bspline=(x0, L, 0, coef))
        y_spline = _apply(op, x)
        sc.scabem_set_sigma(op, per_qpoint=sig.reshape(-1))
        y_values = _apply(op, x)
        scale = np.max(np.abs(y_values))
        assert np.max(np.abs(y_spline - y_values)) <= 1e-13 * scale
        med = operator.Media(*case.media)
        y_or = pfft.PFFT(g, med, case.grid, case.r_near).apply(x, sig)
        assert np.max(np.abs(y_spline - y_or)) <= TOL64 * np.max(np.abs(y_or))
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)


def test_bspline_profile_rejects_bad_arguments():
    case = cases.plate_thin()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 1)
    try:
        for bad in [(0.0, 1.0, 0, [1.0, 1.0, 1.0]),          # too few coefficients
                    (0.0, 0.0, 0, [1.0] * 8),                 # L = 0
                    (0.0, 1.0, 3, [1.0] * 8),                 # bad axis
                    (0.0, 1.0, 0, [1.0] * 7 + [-1.0])]:       # negative coefficient
            with pytest.raises(sc.ScabemError):
                sc.scabem_set_sigma(op, bspline=bad)
        with pytest.raises(sc.ScabemError):
            sc.scabem_set_sigma(op, bspline=(0.0, 1.0, 0, [1.0] * 7 + [float("nan")]))
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)
