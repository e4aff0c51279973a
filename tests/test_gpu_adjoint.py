"""The transposed operator x = A^T y (scabem_apply_adjoint) on the GPU.

Checked against the oracle's transposed O2 matrix on a small mesh, and by
the dot-product identity y . (A x) = (A^T y) . x against the forward apply
(itself parity-checked against O2) on every parity case, both (y, z)
convolution paths and the full-size guide.  Tolerances: complex128 1e-10
against the oracle and 1e-12 for the identity; complex64 1e-5.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import pfft
from test_gpu_parity import CASES, build

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _run(fn, op, v, prec):
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    vt = torch.as_tensor(v).to(dt).cuda().contiguous()
    out = torch.empty_like(vt)
    fn(op, vt, out, prec=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy().astype(np.complex128)


def _dot_gap(op, N, prec, seed):
    rng = np.random.default_rng(seed)
    x = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    y = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    Ax = _run(sc.scabem_apply, op, x, prec)
    ATy = _run(sc.scabem_apply_adjoint, op, y, prec)
    lhs, rhs = y @ Ax, ATy @ x
    return abs(lhs - rhs) / (np.linalg.norm(y) * np.linalg.norm(Ax))


@pytest.mark.parametrize("mk", CASES, ids=lambda f: f.__name__)
@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_adjoint_dot_product_identity(mk, prec):
    case = mk()
    mh, op, g, med, sig = build(case)
    gap = _dot_gap(op, g.N, prec, case.seed + 7)
    assert gap < (1e-12 if prec == sc.SCABEM_C128 else 1e-5), gap


def test_adjoint_matches_oracle_transpose():
    case = cases.plate_thin()
    mh, op, g, med, sig = build(case)
    y = cases.synth.complex_normal(g.N, seed=99)
    ref = pfft.apply_transpose(pfft.PFFT(g, med, case.grid, case.r_near), y, sig)
    got = _run(sc.scabem_apply_adjoint, op, y, sc.SCABEM_C128)
    assert np.max(np.abs(got - ref)) <= 1e-10 * np.max(np.abs(ref))
    got32 = _run(sc.scabem_apply_adjoint, op, y, sc.SCABEM_C64)
    assert np.max(np.abs(got32 - ref)) <= 1e-5 * np.max(np.abs(ref))


@pytest.mark.parametrize("prec", [sc.SCABEM_C64, sc.SCABEM_C128], ids=["c64", "c128"])
def test_adjoint_full_size_guide(prec):
    """The 12 um guide (direct (y, z) sums, 706k near pairs): dot-product identity."""
    case = cases.guide_full()
    mh, op, g, med, sig = build(case, prec_mask=1 if prec == sc.SCABEM_C64 else 3)
    gap = _dot_gap(op, g.N, prec, 5)
    assert gap < (1e-12 if prec == sc.SCABEM_C128 else 1e-5), gap


def test_adjoint_host_buffers_and_batch():
    """Host staging and several right-hand sides in one call give the same columns."""
    case = cases.sphere_mixed()
    mh, op, g, med, sig = build(case)
    N = g.N
    Y = np.stack([cases.synth.complex_normal(N, seed=300 + c) for c in range(3)])
    Yd = torch.as_tensor(Y).cuda().contiguous()
    Xd = torch.empty_like(Yd)
    sc.scabem_apply_adjoint(op, Yd, Xd, nrhs=3, ld=N, prec=sc.SCABEM_C128)
    torch.cuda.synchronize()
    Xh = np.empty_like(Y)
    sc.scabem_apply_adjoint(op, np.ascontiguousarray(Y), Xh, nrhs=3, ld=N, prec=sc.SCABEM_C128)
    for c in range(3):
        one = _run(sc.scabem_apply_adjoint, op, Y[c], sc.SCABEM_C128)
        assert np.max(np.abs(Xd.cpu().numpy()[c] - one)) <= 1e-13 * np.max(np.abs(one))
        assert np.max(np.abs(Xh[c] - one)) <= 1e-13 * np.max(np.abs(one))
