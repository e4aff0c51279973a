"""Gradient of the reflection |r|^2 with respect to the absorber's B-spline coefficients.

The absorber conductivity is a cubic B-spline of 16 coefficients (uniform in
[0, 2 sigma0], seeded), and the objective is J = |r|^2 with r = c / a the
two-wave split (Sec. I, Table 1) of the interior field E_y on probe points of
the axis at a fixed propagation constant: [a, c] = P E_y, P the pseudo-inverse
of [exp(-j beta t), exp(j beta t)].  E_y = E_inc + F x is linear in the
solution x, F the field map of the interior currents (Eq. 8).  The GPU
gradient runs through the autograd wrapper: the forward GMRES solve, the
adjoint (transposed) solve A^T lam = conj(v) and the conductivity sensitivity
of lam^T (A x - b); J is built in torch from F (the library's field
evaluation applied to the columns of the identity).

- On the short guide (416 triangles) it matches the oracle's FP64 adjoint
  gradient: the oracle's grid operator O2 assembled and solved by LU for x
  and lam, F from the oracle's own field evaluation, and the derivative of
  lam^T (A x - b) by the exact affine difference in each coefficient (A and b
  are affine in sigma).
- On a 1,952-triangle guide it matches central finite differences
  (h = 1e-4 of the coefficient range) of the same GPU solves, with the
  complex64 operator inside GMRES and FP64 refinement, the precision the
  gradient workload uses.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import excitation, mesh, operator, post

from test_gpu_parity import oracle_op
from test_gpu_solved_reflection import GUIDE_SRC, _dense, setup

pytestmark = pytest.mark.gpu

BETA = 10.0  # rad/um, the guided wave's propagation constant (fit of the Sec. III study)


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _probe(t0, t1, n):
    ts = np.linspace(t0, t1, n)
    return ts, np.stack([ts, np.full(n, 0.01), np.full(n, -0.005)], 1)


def _split(ts):
    """P: [a, c] = P E for E = a exp(-j beta t) + c exp(j beta t) (least squares)."""
    M = np.stack([np.exp(-1j * BETA * ts), np.exp(1j * BETA * ts)], 1)
    return np.linalg.pinv(M)


def _gpu_field_map(op, N, pts):
    """F (npts x N): E_y at the points from the interior currents of each unit vector."""
    eye = torch.eye(N, dtype=torch.complex128, device="cuda")
    E = sc.scabem_fields(op, eye, pts, nrhs=N, ld=N)  # (N, npts, 3)
    return torch.as_tensor(E[:, :, 1].T.copy()).cuda()


def _gpu_gradient(op, case, N, src_kw, pts, ts, solve_kw):
    from paper_1004_5076_gb300.autograd import absorber_solve

    x0, L, axis, coef = case.sigma_bspline
    src = [sc.make_source("beam", "i", **src_kw)]
    F = _gpu_field_map(op, N, pts)
    ki = 2 * np.pi * np.sqrt(case.media[0] * case.media[1]) / case.media[4]
    zi = np.sqrt(case.media[1] / case.media[0])
    e_inc = excitation.beam(pts, ki, zi, src_kw["pos"], src_kw["dir"], src_kw["b"], src_kw["pol"])[0][:, 1]
    P = torch.as_tensor(_split(ts)).cuda()
    einc = torch.as_tensor(e_inc).cuda()

    def J(c):
        x = absorber_solve(c, op, N, (x0, L, axis), src, **solve_kw)
        ac = P @ (einc + F @ x)
        r = ac[1] / ac[0]
        return (r * r.conj()).real

    c0 = torch.tensor(coef, dtype=torch.float64, requires_grad=True)
    j0 = J(c0)
    j0.backward()
    return float(j0), c0.grad.numpy().copy(), J


def test_reflection_gradient_matches_oracle_adjoint():
    case = cases.guide_short()
    mh, op, g, med, sig, b, x_or = setup(case, GUIDE_SRC, "i")
    A = _dense[case.name]
    N = g.N
    ts, pts = _probe(0.7, 1.15, 16)
    kw = dict(tol=1e-12, restart=120, maxit=20000, refine_tol=1e-12, max_refine=10, prec=sc.SCABEM_C128)
    j_gpu, grad_gpu, _ = _gpu_gradient(op, case, N, GUIDE_SRC["gpu"], pts, ts, kw)
    # the oracle's adjoint gradient
    ke, ki = med.k
    ze, zi = med.z
    so = GUIDE_SRC["oracle"]
    F = post.radiated(g, np.eye(N, dtype=np.complex128), pts, ki, zi, "i")[:, 1, :]  # (npts, N)
    e_inc = excitation.beam(pts, ki, zi, so["r0"], so["d"], so["b"], so["p"])[0][:, 1]
    P = _split(ts)
    a, c = P @ (e_inc + F @ x_or)
    r = c / a
    assert abs(abs(r) ** 2 - j_gpu) <= 1e-7 * max(j_gpu, 1e-12)
    w = 2 * np.conj(r) * (P[1] - r * P[0]) / a  # dJ = Re(w F dx)
    lam = np.linalg.solve(A.T, w @ F)
    x0, L, axis, coef = case.sigma_bspline
    o2 = oracle_op(case, g, med)
    zero = np.zeros_like(sig)
    base = o2.apply(x_or, zero) - excitation.rhs(g, med, zero, "i", "beam", **so)
    grad_or = np.zeros(len(coef))
    from oracle import sigma as osig

    for i in range(len(coef)):
        e = np.zeros(len(coef))
        e[i] = 1.0
        si = osig.bspline(g.qpts, x0, L, e, axis)
        di = o2.apply(x_or, si) - excitation.rhs(g, med, si, "i", "beam", **so) - base
        grad_or[i] = -np.real(lam @ di)
    scale = np.max(np.abs(grad_or))
    assert scale > 0
    assert np.max(np.abs(grad_gpu - grad_or)) <= 1e-6 * scale, (grad_gpu, grad_or)


def test_reflection_gradient_matches_finite_differences_on_2k_triangles():
    case = cases.guide_2k()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3)
    try:
        N = sc.scabem_mesh_info(mh)[2]
        assert m.nt == 1952
        src_kw = dict(pos=(1.2, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)
        ts, pts = _probe(1.5, 2.6, 24)
        kw = dict(tol=1e-6, restart=120, maxit=40000, refine_tol=1e-12, max_refine=20, prec=sc.SCABEM_C64)
        j0, grad, J = _gpu_gradient(op, case, N, src_kw, pts, ts, kw)
        coef = case.sigma_bspline[3]
        h = 1e-4 * 0.008
        scale = np.max(np.abs(grad))
        for k in (3, 8, 12):
            cp, cm = torch.tensor(coef), torch.tensor(coef)
            cp[k] += h
            cm[k] -= h
            fd = (float(J(cp)) - float(J(cm))) / (2 * h)
            assert abs(grad[k] - fd) <= 1e-4 * scale, (k, grad[k], fd, scale)
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)
