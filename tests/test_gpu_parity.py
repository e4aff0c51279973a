"""Parity of the CUDA path (through the C-ABI) with the FP64 oracle.

Tolerances (stated by the target and used verbatim): complex128 operator
1e-10 relative, complex64 operator 1e-5 relative, solved systems 1e-8
relative residual after refinement.  Element-wise checks scale by the largest
oracle entry (|y_gpu - y_orc|_inf <= tol * |y_orc|_inf) so tiny entries with
cancellation are measured against the row scale of the operator.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import excitation, mesh, operator, pfft, post

pytestmark = pytest.mark.gpu

TOL64 = 1e-10
TOL32 = 1e-5


def _gpu_ok():
    return torch.cuda.is_available()


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not _gpu_ok():
        pytest.skip("no CUDA device")


_cache = {}


def build(case, prec_mask=3):
    key = (case.name, prec_mask, case.grid.n, case.grid.p, case.q, case.r_near, case.transverse)
    if key in _cache:
        return _cache[key]
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, prec_mask, transverse=case.transverse)
    if case.transverse != "auto":
        assert sc.scabem_op_grid_info(op)["transverse_direct"] == (case.transverse == "direct")
    g = mesh.build(m.V, m.T, m.region, q=case.q)
    sig = cases.sigma_points(case, g.qpts)
    if case.sigma_segments:
        sc.scabem_set_sigma(op, segments=case.sigma_segments)
    else:
        sc.scabem_set_sigma(op, per_qpoint=sig.reshape(-1))
    med = operator.Media(*case.media)
    _cache[key] = (mh, op, g, med, sig)
    return _cache[key]


def gpu_apply(op, x, prec):
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    xt = torch.as_tensor(x).to(dt).cuda().contiguous()
    yt = torch.empty_like(xt)
    sc.scabem_apply(op, xt, yt, nrhs=1, ld=xt.shape[0], prec=prec)
    torch.cuda.synchronize()
    return yt.cpu().numpy().astype(np.complex128)


_oracle_y = {}
_oracle_ops = {}


def oracle_op(case, g, med):
    """The oracle's grid operator O2 of a case, built once per test session (it keeps its
    whole-mesh near corrections, the costly part, after the first full apply)."""
    key = (case.name, case.grid.n, case.grid.p, case.q, case.r_near, case.grid.h)
    if key not in _oracle_ops:
        _oracle_ops[key] = pfft.PFFT(g, med, case.grid, case.r_near)
    return _oracle_ops[key]


def oracle_apply(case, g, med, sig, x, key):
    if key not in _oracle_y:
        _oracle_y[key] = oracle_op(case, g, med).apply(x, sig)
    return _oracle_y[key]


CASES = [cases.sphere_mixed, cases.guide_small, cases.plate_thin, cases.guide_planes64, cases.guide_planes64_fft,
         cases.sphere_direct, cases.plate_p4_q7, cases.plate_q1]


@pytest.mark.parametrize("mk", CASES, ids=lambda f: f.__name__)
def test_apply_complex128_matches_oracle(mk):
    case = mk()
    mh, op, g, med, sig = build(case)
    x = cases.synth.complex_normal(g.N, seed=case.seed + 100)
    y_or = oracle_apply(case, g, med, sig, x, (case.name, "x0"))
    y = gpu_apply(op, x, sc.SCABEM_C128)
    rel = np.linalg.norm(y - y_or) / np.linalg.norm(y_or)
    assert rel < TOL64, rel
    assert np.max(np.abs(y - y_or)) <= TOL64 * np.max(np.abs(y_or))


@pytest.mark.parametrize("mk", CASES, ids=lambda f: f.__name__)
def test_apply_complex64_matches_oracle(mk):
    case = mk()
    mh, op, g, med, sig = build(case)
    x = cases.synth.complex_normal(g.N, seed=case.seed + 100)
    y_or = oracle_apply(case, g, med, sig, x, (case.name, "x0"))
    y = gpu_apply(op, x, sc.SCABEM_C64)
    rel = np.linalg.norm(y - y_or) / np.linalg.norm(y_or)
    assert rel < TOL32, rel
    assert np.max(np.abs(y - y_or)) <= TOL32 * np.max(np.abs(y_or))


def test_apply_empty_batch_and_zero_input():
    """nrhs = 0 touches nothing; x = 0 gives exactly 0 in both directions and precisions (every
    stage is linear, and the row sums add exact zeros)."""
    case = cases.plate_thin()
    mh, op, g, med, sig = build(case)
    N = g.N
    y = torch.full((N,), complex(float("nan"), 0.0), dtype=torch.complex64, device="cuda")
    x = torch.zeros(N, dtype=torch.complex64, device="cuda")
    sc.scabem_apply(op, x, y, nrhs=0, ld=N, prec=sc.SCABEM_C64)
    sc.scabem_apply_adjoint(op, x, y, nrhs=0, ld=N, prec=sc.SCABEM_C64)
    torch.cuda.synchronize()
    assert torch.isnan(y.real).all()
    for prec, dt in ((sc.SCABEM_C64, torch.complex64), (sc.SCABEM_C128, torch.complex128)):
        x = torch.zeros(N, dtype=dt, device="cuda")
        for fn in (sc.scabem_apply, sc.scabem_apply_adjoint):
            y = torch.full_like(x, 1.0 + 1.0j)
            fn(op, x, y, prec=prec)
            torch.cuda.synchronize()
            assert int(torch.count_nonzero(y)) == 0, (fn.__name__, prec)


def test_apply_batched_columns_and_host_buffers():
    """nrhs > 1 with ld > N, from host (pinned-less numpy) buffers: same as column by column.

    The row sums add two terms per row with atomics (order-independent), so
    the columns agree with single-column applies to rounding of the staging
    path at most."""
    case = cases.sphere_mixed()
    mh, op, g, med, sig = build(case)
    N = g.N
    ld = N + 7
    X = np.zeros((3, ld), np.complex128)
    for c in range(3):
        X[c, :N] = cases.synth.complex_normal(N, seed=200 + c)
    Y = np.zeros_like(X)
    sc.scabem_apply(op, X, Y, nrhs=3, ld=ld, prec=sc.SCABEM_C128)
    for c in range(3):
        yc = gpu_apply(op, X[c, :N], sc.SCABEM_C128)
        assert np.linalg.norm(Y[c, :N] - yc) <= 1e-13 * np.linalg.norm(yc)
        assert np.all(Y[c, N:] == 0)


@pytest.mark.parametrize(
    "mk,src,side",
    [
        (cases.guide_small, dict(kind="beam", pos=(1.0, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07), "i"),
        (cases.sphere_mixed, dict(kind="planewave", dir=(0, 0, 1), pol=(1, 0, 0)), "e"),
        (cases.plate_thin, dict(kind="dipole", pos=(0.7, 0.01, 0.0), pol=(0.3, 1.0, 0.2)), "i"),
    ],
    ids=["beam_interior", "planewave_exterior", "dipole_interior"],
)
def test_rhs_matches_oracle(mk, src, side):
    case = mk()
    mh, op, g, med, sig = build(case)
    kind = src.pop("kind")
    s = sc.make_source(kind, side, **src)
    b = torch.zeros(g.N, dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, [s], b, prec=sc.SCABEM_C128)
    torch.cuda.synchronize()
    kw = {"planewave": dict(d=src.get("dir"), e=src.get("pol")),
          "dipole": dict(rs=src.get("pos"), p=src.get("pol")),
          "beam": dict(r0=src.get("pos"), d=src.get("dir"), b=src.get("b"), p=src.get("pol"))}[kind]
    b_or = excitation.rhs(g, med, sig, side, kind, **kw)
    b = b.cpu().numpy()
    assert np.linalg.norm(b - b_or) <= TOL64 * np.linalg.norm(b_or)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64_refined"])
def test_solve_reaches_oracle_residual(prec):
    """GMRES (complex64 or complex128 inner operator, FP64 refinement) solves the oracle's system."""
    case = cases.sphere_mixed()
    mh, op, g, med, sig = build(case)
    s = sc.make_source("planewave", "e", dir=(0, 0, 1), pol=(1, 0, 0))
    b = torch.zeros(g.N, dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, [s], b, prec=sc.SCABEM_C128)
    x = torch.zeros_like(b)
    info = sc.scabem_solve(op, b, x, tol=1e-9 if prec == sc.SCABEM_C128 else 1e-5, restart=80, maxit=3000,
                           refine_tol=1e-10, max_refine=12, prec=prec)
    assert info[0]["status"] == 0 and info[0]["relres"] < 1e-8, info
    xn = x.cpu().numpy()
    bn = b.cpu().numpy()
    r = bn - oracle_op(case, g, med).apply(xn, sig)
    assert np.linalg.norm(r) / np.linalg.norm(bn) < 1e-8


@pytest.mark.parametrize("prec,transverse", [(sc.SCABEM_C64, "auto"), (sc.SCABEM_C128, "auto"), (sc.SCABEM_C64, "fft")],
                         ids=["c64", "c128", "c64_fft_planes"])
def test_full_size_guide_sampled_rows(prec, transverse):
    """The 12 um guide on the 512 x 64 x 64 grid, in the launch configuration
    bench.py times (automatic choice: direct (y, z) sums), and with the FFT
    planes: every row of 24 random edges (both triangles of each edge as
    targets) against the oracle's grid operator at those rows."""
    case = cases.guide_full()
    case.transverse = transverse
    mask = 1 if prec == sc.SCABEM_C64 else 3
    mh, op, g, med, sig = build(case, prec_mask=mask)
    x = cases.synth.complex_normal(g.N, seed=4242)
    y = gpu_apply(op, x, prec)
    rng = np.random.default_rng(9)
    edges = rng.choice(g.ne, 24, replace=False)
    targets = np.unique(g.edge_t[edges].reshape(-1))
    key = (case.name, "sampled")
    if key not in _oracle_y:
        _oracle_y[key] = pfft.PFFT(g, med, case.grid, case.r_near).apply(x, sig, targets=targets)
    y_or = _oracle_y[key]
    rows = mesh.row_index(g)[edges]
    rows = rows[rows >= 0]
    tol = TOL32 if prec == sc.SCABEM_C64 else TOL64
    d = y[rows] - y_or[rows]
    assert np.linalg.norm(d) <= tol * np.linalg.norm(y_or[rows])
    assert np.max(np.abs(d)) <= tol * np.max(np.abs(y_or[rows]))


def test_fields_and_reflection_match_oracle():
    case = cases.guide_small()
    mh, op, g, med, sig = build(case)
    x = cases.synth.complex_normal(g.N, seed=77) * 1e-2
    xt = torch.as_tensor(x).cuda()
    src = sc.make_source("beam", "i", pos=(0.8, 0, 0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)
    pts = np.stack([np.linspace(0.9, 1.3, 12), np.full(12, 0.01), np.full(12, -0.005)], 1)
    E = sc.scabem_fields(op, xt, pts, inc=src)[0]
    ke, ki = med.k
    ze, zi = med.z
    E_or = post.radiated(g, x, pts, ki, zi, "i") + excitation.beam(pts, ki, zi, (0.8, 0, 0), (1, 0, 0), 0.07,
                                                                   (0, 1, 0))[0]
    assert np.linalg.norm(E - E_or) <= 1e-10 * np.linalg.norm(E_or)
    out = sc.scabem_reflection(op, xt, 0, 1, (0.0, 0.01, -0.005), 0.9, 1.3, 12, 10.0, 16.0, 601, inc=src)[0]
    r_or, beta_or, res_or = post.fit_reflection(pts[:, 0], E_or[:, 1], betas=np.linspace(10.0, 16.0, 601))
    assert abs(out[2] - beta_or) < 1e-9
    assert abs(complex(out[0], out[1]) - r_or) < 1e-8 * max(1.0, abs(r_or))


def test_invalid_arguments_are_rejected():
    case = cases.sphere_mixed()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    # stencils outside the grid: origin far away
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, (5.0, 5.0, 5.0), 3, 6, 0.3, 3)
    assert e.value.code == -1
    with pytest.raises(sc.ScabemError):
        sc.scabem_op_create(mh, case.media, (15, 16, 16), case.grid.h, case.grid.origin, 3, 6, 0.3, 3)
    _, op, g, _, _ = build(case)
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_set_sigma(op, per_qpoint=np.full(g.nt * g.q, np.nan))
    assert e.value.code == -7
    sc.scabem_mesh_destroy(mh)
