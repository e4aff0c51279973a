"""Circulant preconditioner of Appendix B on the GPU.

On a short guide with absorbers at both ends, the plain section's regular
slices carry a block circulant approximation of A_LL built from the
operator's own columns: Strang's (the middle slice's columns) or T. Chan's
optimal one (the first and the last slice's columns).  The preconditioner's
apply on those unknowns must equal the oracle's circulant solve (block DFT
over the slices, one dense solve per frequency) built from the same columns
of the oracle's grid operator O2, and leave every other unknown to the
block-diagonal preconditioner; GMRES with it must reach the same solution as
with the block-diagonal one.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
import synth
from oracle import toeplitz

from test_gpu_parity import build, oracle_op

pytestmark = pytest.mark.gpu

NX, LEN, FIRST, COUNT = 20, 2.0, 6, 8


def periodic_case():
    m = synth.waveguide(LEN, 0.5, 0.22, NX, 4, 2, 0.5, 0.5)
    grid = synth.grid_for_mesh(m.V, (64, 32, 32), p=3)
    segs = [(1.5, 0.5, 0.004, 2, 0, 1.0), (0.5, 0.5, 0.004, 2, 0, -1.0)]
    return cases.Case("guide_periodic", m, (12.1, 1.0, 2.1, 1.0, 1.55), grid, 6, 2.05 * grid.h, sigma_segments=segs,
                      seed=16)


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = periodic_case()
    mh, op, g, med, sig = build(case)
    lay = toeplitz.SliceLayout(g, 0.0, LEN / NX, NX, first=FIRST, count=COUNT)
    return case, mh, op, g, med, sig, lay


_cols = {}


def _oracle_blocks(case, g, med, sig, lay, slices):
    """T[d] from the oracle's O2 columns of the given regular slices (signed unit vectors).  An
    offset that two slices both give keeps the first slice's block: Chan's c_0 = T[0] is the
    diagonal block of the first block column (the operator is Toeplitz only up to the absorbers
    and the grid, so the last slice's diagonal block differs slightly)."""
    T = {}
    for k0 in slices:
        if k0 not in _cols:
            idx0, sg0 = lay.unknowns(g, k0)
            E = np.zeros((g.N, lay.m), dtype=np.complex128)
            E[idx0, np.arange(lay.m)] = sg0
            _cols[k0] = oracle_op(case, g, med).apply(E, sig)
        for k in range(lay.count):
            idx, sg = lay.unknowns(g, k)
            T.setdefault(k - k0, sg[:, None] * _cols[k0][idx])
    return T


@pytest.mark.parametrize("kind", ["strang", "chan"])
def test_circulant_apply_matches_oracle(setup, kind):
    case, mh, op, g, med, sig, lay = setup
    R, m = lay.count, lay.m
    if kind == "strang":  # the middle slice's columns
        c = toeplitz.strang(_oracle_blocks(case, g, med, sig, lay, [R // 2]), R)
    else:  # the first and the last slice's columns give every offset
        c = toeplitz.chan(_oracle_blocks(case, g, med, sig, lay, [0, R - 1]), R)
    v = cases.synth.complex_normal(g.N, seed=71)
    vt = torch.as_tensor(v).cuda()
    z_bd = torch.empty_like(vt)
    sc.scabem_precond_apply(op, vt, z_bd)  # block diagonal only
    sc.scabem_set_precond_circulant(op, mh, axis=0, x0=0.0, dx=LEN / NX, first=FIRST, count=COUNT, kind=kind)
    try:
        z = torch.empty_like(vt)
        sc.scabem_precond_apply(op, vt, z)
        torch.cuda.synchronize()
        z, z_bd = z.cpu().numpy(), z_bd.cpu().numpy()
        vs = np.stack([lay.unknowns(g, k)[1] * v[lay.unknowns(g, k)[0]] for k in range(R)])
        xs = toeplitz.circulant_solve(c, vs)
        per = np.zeros(g.N, dtype=bool)
        for k in range(R):
            idx, sg = lay.unknowns(g, k)
            per[idx] = True
            assert np.linalg.norm(sg * z[idx] - xs[k]) <= 1e-9 * np.linalg.norm(xs), k
        assert per.sum() == R * m
        assert np.array_equal(z[~per], z_bd[~per])
        # transposed solves keep the block-diagonal preconditioner
        zt = torch.empty_like(vt)
        sc.scabem_precond_apply(op, vt, zt, transpose=True)
        zt_bd = torch.empty_like(vt)
        sc.scabem_set_precond_circulant(op, mh, count=0)
        sc.scabem_precond_apply(op, vt, zt_bd, transpose=True)
        torch.cuda.synchronize()
        assert torch.equal(zt, zt_bd)
    finally:
        sc.scabem_set_precond_circulant(op, mh, count=0)


@pytest.mark.parametrize("kind", ["strang", "chan"])
def test_gmres_with_the_circulant_reaches_the_same_solution(setup, kind):
    """The preconditioned solve reaches the block-diagonal one's solution; the iteration counts
    are printed.  A circulant closes the plain section into a ring without absorbers, whose guided
    resonances make it a poor model of A_LL for a guided wave, so fewer iterations are not asked."""
    case, mh, op, g, med, sig, lay = setup
    src = [sc.make_source("beam", "i", pos=(0.6, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)]
    b = torch.zeros(g.N, dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, src, b, prec=sc.SCABEM_C128)
    kw = dict(tol=1e-5, restart=60, maxit=40000, refine_tol=1e-10, max_refine=10, prec=sc.SCABEM_C64)
    x_bd = torch.zeros_like(b)
    info_bd = sc.scabem_solve(op, b, x_bd, **kw)[0]
    sc.scabem_set_precond_circulant(op, mh, axis=0, x0=0.0, dx=LEN / NX, first=FIRST, count=COUNT, kind=kind)
    try:
        x_c = torch.zeros_like(b)
        info_c = sc.scabem_solve(op, b, x_c, **kw)[0]
    finally:
        sc.scabem_set_precond_circulant(op, mh, count=0)
    assert info_bd["status"] == 0 and info_c["status"] == 0, (info_bd, info_c)
    rel = float((x_c - x_bd).abs().norm() / x_bd.abs().norm())
    assert rel <= 1e-7, (rel, info_bd, info_c)
    print(f"iterations: block diagonal {info_bd['iters']}, {kind} circulant {info_c['iters']}")
