"""Batched apply: many right-hand sides in one scabem_apply call.

Up to eight columns go through every stage together, and the point kernel
reads each target's near records once for all of them.  Every column must
equal a single-column apply of the same vector to rounding (the arithmetic of
a column is the same, in the same order, and the row sums add two terms onto
zero; only the compiler's instruction choice in the two kernels may differ) and
the oracle's grid operator O2 within the parity tolerances (complex128 1e-10,
complex64 1e-5), for batches that fill the eight columns and for a ragged last
batch, with a leading dimension larger than N.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import mesh, pfft

from test_gpu_parity import TOL32, TOL64, build, gpu_apply, oracle_op

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


CASES = [cases.guide_small, cases.sphere_direct, cases.plate_p4_q7, cases.plate_q1]
_yor = {}


@pytest.mark.parametrize("mk", CASES, ids=lambda f: f.__name__)
@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_batched_columns_match_single_applies_and_oracle(mk, prec):
    case = mk()
    mh, op, g, med, sig = build(case)
    N = g.N
    nrhs, ld = 11, N + 5  # one batch of 8 and a ragged batch of 3
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    X = np.zeros((nrhs, ld), np.complex128)
    for c in range(nrhs):
        X[c, :N] = cases.synth.complex_normal(N, seed=500 + c)
    Xd = torch.as_tensor(X).to(dt).cuda().contiguous()
    Yd = torch.full_like(Xd, complex(3.0, -1.0))
    sc.scabem_apply(op, Xd, Yd, nrhs=nrhs, ld=ld, prec=prec)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.complex128)
    assert np.all(Y[:, N:] == complex(3.0, -1.0))  # the padding between columns is untouched
    if case.name not in _yor:
        _yor[case.name] = oracle_op(case, g, med).apply(X[:, :N].T, sig).T
    Y_or = _yor[case.name]
    tol = TOL64 if prec == sc.SCABEM_C128 else TOL32
    same = 1e-14 if prec == sc.SCABEM_C128 else 1e-6
    for c in range(nrhs):
        single = gpu_apply(op, X[c, :N], prec)
        assert np.max(np.abs(Y[c, :N] - single)) <= same * np.max(np.abs(single)), c
        d = Y[c, :N] - Y_or[c]
        assert np.linalg.norm(d) <= tol * np.linalg.norm(Y_or[c]), c
        assert np.max(np.abs(d)) <= tol * np.max(np.abs(Y_or[c])), c


def test_batched_full_size_guide_sampled_rows():
    """The 12 um guide with eight columns in one call (the batched launch configuration the
    benchmark times): every column equals its single-column apply to rounding, and the rows of
    12 random edges of two columns match the oracle's grid operator."""
    case = cases.guide_full()
    mh, op, g, med, sig = build(case, prec_mask=1)
    N = g.N
    nrhs = 8
    X = np.stack([cases.synth.complex_normal(N, seed=900 + c) for c in range(nrhs)])
    Xd = torch.as_tensor(X).to(torch.complex64).cuda().contiguous()
    Yd = torch.empty_like(Xd)
    sc.scabem_apply(op, Xd, Yd, nrhs=nrhs, ld=N, prec=sc.SCABEM_C64)
    torch.cuda.synchronize()
    Y = Yd.cpu().numpy().astype(np.complex128)
    for c in range(nrhs):
        single = gpu_apply(op, X[c], sc.SCABEM_C64)
        assert np.max(np.abs(Y[c] - single)) <= 1e-6 * np.max(np.abs(single)), c
    rng = np.random.default_rng(17)
    edges = rng.choice(g.ne, 12, replace=False)
    targets = np.unique(g.edge_t[edges].reshape(-1))
    rows = mesh.row_index(g)[edges]
    rows = rows[rows >= 0]
    y_or = pfft.PFFT(g, med, case.grid, case.r_near).apply(X[[0, 7]].T, sig, targets=targets).T
    for c, yo in zip((0, 7), y_or):
        d = Y[c, rows] - yo[rows]
        assert np.linalg.norm(d) <= TOL32 * np.linalg.norm(yo[rows]), c
