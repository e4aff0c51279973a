"""The autotuner: it times the operator's runtime shapes (the (y, z) mode
where both fit, the axis-0 lines per CTA) and keeps the fastest; the operator
it leaves behind is the same linear operator, so the parity with the oracle's
grid operator must hold after tuning, in both precisions and for a batch."""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import mesh, operator

from test_gpu_parity import TOL32, TOL64, oracle_apply

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("prec,nrhs", [(sc.SCABEM_C64, 1), (sc.SCABEM_C128, 1), (sc.SCABEM_C64, 8)],
                         ids=["c64", "c128", "c64_batch8"])
def test_autotuned_operator_matches_oracle(prec, nrhs):
    case = cases.guide_planes64()  # 64 x 64 planes: both (y, z) modes fit
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3)
    try:
        sc.scabem_set_sigma(op, segments=case.sigma_segments)
        res = sc.scabem_autotune(op, prec=prec, nrhs=nrhs)
        assert 0 < res["ms"] <= res["ms_initial"] * 1.0001, res
        assert res["axis0_lines"] in (0, 1, 2, 4, 8, 16)
        assert sc.scabem_op_grid_info(op)["transverse_direct"] == res["direct"]
        g = mesh.build(m.V, m.T, m.region, q=case.q)
        sig = cases.sigma_points(case, g.qpts)
        med = operator.Media(*case.media)
        x = cases.synth.complex_normal(g.N, seed=case.seed + 100)
        y_or = oracle_apply(case, g, med, sig, x, (case.name, "x0"))
        dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
        X = torch.as_tensor(np.tile(x, (nrhs, 1))).to(dt).cuda().contiguous()
        Y = torch.empty_like(X)
        sc.scabem_apply(op, X, Y, nrhs=nrhs, ld=g.N, prec=prec)
        torch.cuda.synchronize()
        tol = TOL64 if prec == sc.SCABEM_C128 else TOL32
        for c in range(nrhs):
            y = Y[c].cpu().numpy().astype(np.complex128)
            assert np.linalg.norm(y - y_or) <= tol * np.linalg.norm(y_or), (c, res)
    finally:
        sc.scabem_op_destroy(op)
        sc.scabem_mesh_destroy(mh)
