"""The directional coupler on the 1024 x 256 x 256 transform grid.

Two 40 um guides 0.2 um apart with absorbers at all four ports: 128,440
triangles, 424k unknowns, 13 M near pairs (12.7 GB of complex64 records,
byte offsets beyond 32 bits), (y, z) planes of 256 x 256 that only the direct sums over the active
columns handle.  Every row of 24 random edges (both triangles of each edge as
targets) against the oracle's grid operator O2 at those rows, in complex128
(1e-10) and complex64 (1e-5), and eight columns in one call against the
single-column apply.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import mesh, operator, pfft

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def coupler():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = cases.coupler_full()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3)
    sc.scabem_set_sigma(op, segments=case.sigma_segments)
    assert sc.scabem_op_grid_info(op)["transverse_direct"]
    g = mesh.build(m.V, m.T, m.region, q=case.q)
    sig = cases.sigma_points(case, g.qpts)
    x = cases.synth.complex_normal(g.N, seed=4343)
    rng = np.random.default_rng(19)
    edges = rng.choice(g.ne, 24, replace=False)
    targets = np.unique(g.edge_t[edges].reshape(-1))
    y_or = pfft.PFFT(g, operator.Media(*case.media), case.grid, case.r_near).apply(x, sig, targets=targets)
    rows = mesh.row_index(g)[edges]
    rows = rows[rows >= 0]
    yield op, g, x, rows, y_or
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_coupler_sampled_rows_match_oracle(coupler, prec):
    op, g, x, rows, y_or = coupler
    info = sc.scabem_op_info(op)
    assert info["near_pairs"] > 10_000_000 and info["near_bytes_c64"] > 2**33  # byte offsets beyond 32 bits
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    xt = torch.as_tensor(x).to(dt).cuda().contiguous()
    yt = torch.empty_like(xt)
    sc.scabem_apply(op, xt, yt, prec=prec)
    torch.cuda.synchronize()
    y = yt.cpu().numpy().astype(np.complex128)
    tol = 1e-10 if prec == sc.SCABEM_C128 else 1e-5
    d = y[rows] - y_or[rows]
    assert np.linalg.norm(d) <= tol * np.linalg.norm(y_or[rows])
    assert np.max(np.abs(d)) <= tol * np.max(np.abs(y_or[rows]))


def test_coupler_eight_columns_in_one_call(coupler):
    op, g, x, rows, y_or = coupler
    N = g.N
    X = torch.stack([torch.as_tensor(cases.synth.complex_normal(N, seed=60 + c)) for c in range(8)])
    X[3] = torch.as_tensor(x)
    X = X.to(torch.complex64).cuda().contiguous()
    Y = torch.empty_like(X)
    sc.scabem_apply(op, X, Y, nrhs=8, ld=N, prec=sc.SCABEM_C64)
    y1 = torch.empty_like(X[3])
    sc.scabem_apply(op, X[3].contiguous(), y1, prec=sc.SCABEM_C64)
    torch.cuda.synchronize()
    a, b = Y[3].cpu().numpy(), y1.cpu().numpy()
    assert np.max(np.abs(a - b)) <= 1e-6 * np.max(np.abs(b))
    d = a.astype(np.complex128)[rows] - y_or[rows]
    assert np.linalg.norm(d) <= 1e-5 * np.linalg.norm(y_or[rows])
