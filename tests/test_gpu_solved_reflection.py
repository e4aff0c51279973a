"""Solved systems against the oracle's direct solution.

The oracle assembles its grid operator O2 (the plain definition of the
precorrected-FFT product) column by column and solves it by LU; the CUDA
path solves the same system with GMRES (complex128 operator, and complex64
operator with FP64 iterative refinement).  The solutions
and the reflection fitted from them (Sec. I, Table 1: two-wave fit of the
axis field) must agree to 1e-8 relative; the solves are run to a relative
residual of 1e-12 so that the conditioning of the system does not eat the
margin.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import excitation, mesh, operator, pfft, post

from test_gpu_parity import oracle_op

pytestmark = pytest.mark.gpu

TOL = 1e-8


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


_cache = {}
_dense = {}  # the oracle's O2 matrices, kept for the gradient tests


def setup(case, src_kw, side):
    """GPU operator, oracle geometry, conductivity, right-hand side and the
    oracle's LU solution of the O2 system."""
    if case.name in _cache:
        return _cache[case.name]
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3, transverse=case.transverse)
    g = mesh.build(m.V, m.T, m.region, q=case.q)
    sig = cases.sigma_points(case, g.qpts)
    if case.sigma_bspline is not None:
        sc.scabem_set_sigma(op, bspline=case.sigma_bspline)
    elif case.sigma_segments:
        sc.scabem_set_sigma(op, segments=case.sigma_segments)
    else:
        sc.scabem_set_sigma(op, per_qpoint=sig.reshape(-1))
    med = operator.Media(*case.media)
    A = pfft.dense(oracle_op(case, g, med), sig, chunk=64)
    b = excitation.rhs(g, med, sig, side, src_kw["kind"], **src_kw["oracle"])
    x = np.linalg.solve(A, b)
    _cache[case.name] = (mh, op, g, med, sig, b, x)
    _dense[case.name] = A
    return _cache[case.name]


def gpu_solve(op, b_or, prec):
    """GMRES through the C-ABI on the oracle's right-hand side."""
    b = torch.as_tensor(b_or).cuda().contiguous()
    x = torch.zeros_like(b)
    info = sc.scabem_solve(op, b, x, tol=1e-10 if prec == sc.SCABEM_C128 else 1e-5, restart=120, maxit=20000,
                           refine_tol=1e-12, max_refine=20, prec=prec)[0]
    assert info["status"] == 0 and info["relres"] <= 1e-12, info
    return x


SPHERE_SRC = {"kind": "planewave", "gpu": dict(dir=(0, 0, 1), pol=(1, 0, 0)),
              "oracle": dict(d=(0, 0, 1), e=(1, 0, 0))}
GUIDE_SRC = {"kind": "beam", "gpu": dict(pos=(0.5, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07),
             "oracle": dict(r0=(0.5, 0.0, 0.0), d=(1, 0, 0), b=0.07, p=(0, 1, 0))}


def guide_short():
    return cases.guide_short()


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64_refined"])
def test_sphere_solution_matches_oracle_lu(prec):
    """Plane wave on the sphere with a random-conductivity absorber cap: x against LU of O2."""
    case = cases.sphere_mixed()
    mh, op, g, med, sig, b, x_or = setup(case, SPHERE_SRC, "e")
    x = gpu_solve(op, b, prec).cpu().numpy()
    assert np.linalg.norm(x - x_or) <= TOL * np.linalg.norm(x_or)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64_refined"])
def test_guide_solution_and_reflection_match_oracle_lu(prec):
    """Beam in the short guide with a B-spline absorber profile: the solution, the
    interior field on the axis and the fitted reflection of the right absorber
    against the oracle's LU solution and its own field and fit."""
    case = guide_short()
    mh, op, g, med, sig, b, x_or = setup(case, GUIDE_SRC, "i")
    xt = gpu_solve(op, b, prec)
    x = xt.cpu().numpy()
    assert np.linalg.norm(x - x_or) <= TOL * np.linalg.norm(x_or)
    s = sc.make_source("beam", "i", **GUIDE_SRC["gpu"])
    ke, ki = med.k
    ze, zi = med.z
    t0, t1, npts = 0.7, 1.15, 24
    betas = np.linspace(8.0, 14.0, 601)
    out = sc.scabem_reflection(op, xt, 0, 1, (0.0, 0.01, -0.005), t0, t1, npts, betas[0], betas[-1], len(betas),
                               inc=s)[0]
    ts = np.linspace(t0, t1, npts)
    pts = np.stack([ts, np.full(npts, 0.01), np.full(npts, -0.005)], 1)
    E_or = post.radiated(g, x_or, pts, ki, zi, "i") + excitation.beam(pts, ki, zi, **GUIDE_SRC["oracle"])[0]
    r_or, beta_or, res_or = post.fit_reflection(ts, E_or[:, 1], betas=betas)
    assert abs(out[2] - beta_or) < 1e-9
    assert abs(complex(out[0], out[1]) - r_or) <= TOL * max(1.0, abs(r_or))
    assert abs(out[3] - res_or) <= TOL
