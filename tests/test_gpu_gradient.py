"""Adjoint solves and conductivity gradients on the GPU.

- transposed GMRES reaches its FP64 residual with the transposed operator;
- the per-point sensitivity d(lam^T (A x - b))/d sigma_p matches the oracle's
  exact affine difference (O2 and the oracle's right-hand side);
- the autograd gradient of a real objective through absorber_solve matches
  central finite differences of the same GPU solves.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import excitation, mesh, operator, pfft
from oracle import sigma as osig

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _op(case, prec_mask=3):
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, prec_mask)
    return mh, op


def _spline(case):
    V = case.mesh.V
    return float(V[:, 0].min()), float(np.ptp(V[:, 0])), 0


BEAM = dict(kind="beam", pos=(1.0, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64_refined"])
def test_transposed_solve(prec):
    case = cases.guide_small()
    mh, op = _op(case)
    try:
        sc.scabem_set_sigma(op, segments=case.sigma_segments)
        N = sc.scabem_mesh_info(mh)[2]
        r = torch.as_tensor(cases.synth.complex_normal(N, seed=5)).cuda()
        lam = torch.zeros_like(r)
        info = sc.scabem_solve(op, r, lam, tol=1e-6 if prec == sc.SCABEM_C64 else 1e-10, restart=100, maxit=6000,
                               refine_tol=1e-9, max_refine=10, prec=prec, transpose=True)[0]
        chk = torch.empty_like(r)
        sc.scabem_apply_adjoint(op, lam, chk, prec=sc.SCABEM_C128)
        torch.cuda.synchronize()
        rel = float((chk - r).abs().norm() / r.abs().norm())
        assert rel <= 1e-8, (rel, info)
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)


DIPOLE = dict(pos=(0.7, 0.01, 0.0), pol=(0.3, 1.0, 0.2))


def test_sigma_sensitivity_matches_oracle_difference():
    case = cases.plate_thin()
    mh, op = _op(case, prec_mask=2)
    try:
        g = mesh.build(case.mesh.V, case.mesh.T, case.mesh.region, q=case.q)
        x0, L, axis = _spline(case)
        coef = np.random.default_rng(21).uniform(0.0, 0.008, 12)
        sig = osig.bspline(g.qpts, x0, L, coef, axis)
        sc.scabem_set_sigma(op, bspline=(x0, L, axis, coef))
        x = cases.synth.complex_normal(g.N, seed=31)
        lam = cases.synth.complex_normal(g.N, seed=32)
        src = sc.make_source("dipole", "i", pos=DIPOLE["pos"], pol=DIPOLE["pol"])
        h = sc.scabem_sigma_gradient(op, x, lam, [src], per_qpoint=True)
        med = operator.Media(*case.media)
        o2 = pfft.PFFT(g, med, case.grid, case.r_near)
        kw = dict(rs=DIPOLE["pos"], p=DIPOLE["pol"])
        base = lam @ (o2.apply(x, sig) - excitation.rhs(g, med, sig, "i", "dipole", **kw))
        absorber = np.nonzero(case.mesh.region == 1)[0]
        rng = np.random.default_rng(41)
        scale = np.max(np.abs(h))
        for t in rng.choice(absorber, 4, replace=False):
            p = int(t) * case.q + int(rng.integers(case.q))
            s2 = sig.copy().reshape(-1)
            s2[p] += 1.0  # A and b are affine in sigma: the difference is the derivative
            s2 = s2.reshape(sig.shape)
            ref = lam @ (o2.apply(x, s2) - excitation.rhs(g, med, s2, "i", "dipole", **kw)) - base
            assert abs(h[p] - ref) <= 1e-9 * scale, (p, h[p], ref)
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)


def test_autograd_gradient_matches_finite_differences():
    from paper_1004_5076_gb300.autograd import absorber_solve

    case = cases.guide_small()
    mh, op = _op(case, prec_mask=2)
    try:
        N = sc.scabem_mesh_info(mh)[2]
        spline = _spline(case)
        src = [sc.make_source("beam", "i", pos=BEAM["pos"], dir=BEAM["dir"], pol=BEAM["pol"], b=BEAM["b"])]
        v = torch.as_tensor(cases.synth.complex_normal(N, seed=51)).cuda()
        kw = dict(tol=1e-12, restart=120, maxit=20000, refine_tol=1e-12, max_refine=8, prec=sc.SCABEM_C128)

        def J(c):
            x = absorber_solve(c, op, N, spline, src, **kw)
            return (v * x).sum().real

        c0 = torch.tensor(np.random.default_rng(61).uniform(0.0, 0.008, 12), dtype=torch.float64,
                          requires_grad=True)
        J(c0).backward()
        grad = c0.grad.numpy()
        for k in (2, 6, 9):
            hk = 1e-4 * 0.008
            cp, cm = c0.detach().clone(), c0.detach().clone()
            cp[k] += hk
            cm[k] -= hk
            fd = (float(J(cp)) - float(J(cm))) / (2 * hk)
            assert abs(grad[k] - fd) <= 1e-5 * max(abs(fd), np.max(np.abs(grad))), (k, grad[k], fd)
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)
