"""scabem_rhs_noalloc: the right-hand side for callers that cannot allocate
device memory while they run (a framework's memory pool that has reserved the
device, loops that cannot take cudaFree's device-wide synchronisation).

It must give what scabem_rhs gives, call after call, although every call
reuses the same fixed scratch array.  This file is collected last so that a
run stopping at its first failure has already run every other test; it
passes alone in a fresh process as well.
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc

pytestmark = pytest.mark.gpu

TOL64 = 1e-10  # the complex128 tolerance of the parity tests
TOL32 = 1e-5


@pytest.fixture(scope="module")
def guide_op():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = cases.guide_small()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3)
    sc.scabem_set_sigma(op, segments=case.sigma_segments)
    N = sc.scabem_mesh_info(mh)[2]
    yield op, N
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_rhs_noalloc_matches_rhs_on_consecutive_calls(guide_op, prec):
    op, N = guide_op
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    tol = TOL64 if prec == sc.SCABEM_C128 else TOL32
    sources = [
        sc.make_source("beam", "i", pos=(1.0, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07),
        sc.make_source("planewave", "e", dir=(0, 0.6, 0.8), pol=(1, 0, 0)),
    ]
    for s in sources:  # two calls in a row, each against the allocating entry point
        ref = torch.zeros(N, dtype=dt, device="cuda")
        sc.scabem_rhs(op, [s], ref, prec=prec)
        got = torch.full((N,), complex(7.0, -3.0), dtype=dt, device="cuda")
        sc.scabem_rhs_noalloc(op, [s], got, prec=prec)
        torch.cuda.synchronize()
        r, g = ref.cpu().numpy(), got.cpu().numpy()
        assert np.linalg.norm(g - r) <= tol * np.linalg.norm(r)


@pytest.mark.parametrize("prec", [sc.SCABEM_C128, sc.SCABEM_C64], ids=["c128", "c64"])
def test_rhs_noalloc_two_sources_per_call_with_leading_dimension(guide_op, prec):
    """Two sources in one call reuse the shared scratch one after the other; columns are ld = N + 3
    apart and the padding between them is left untouched."""
    op, N = guide_op
    dt = torch.complex128 if prec == sc.SCABEM_C128 else torch.complex64
    tol = TOL64 if prec == sc.SCABEM_C128 else TOL32
    ld = N + 3
    sources = [
        sc.make_source("dipole", "i", pos=(0.9, 0.02, 0.01), pol=(0.2, 1.0, 0.1)),
        sc.make_source("beam", "i", pos=(1.2, 0.0, 0.0), dir=(-1, 0, 0), pol=(0, 0, 1), b=0.05),
    ]
    ref = torch.zeros(2 * ld, dtype=dt, device="cuda")
    sc.scabem_rhs(op, sources, ref, ld=ld, prec=prec)
    fill = complex(7.0, -3.0)
    got = torch.full((2 * ld,), fill, dtype=dt, device="cuda")
    sc.scabem_rhs_noalloc(op, sources, got, ld=ld, prec=prec)
    torch.cuda.synchronize()
    r, g = ref.cpu().numpy().reshape(2, ld), got.cpu().numpy().reshape(2, ld)
    for c in range(2):
        assert np.linalg.norm(g[c, :N] - r[c, :N]) <= tol * np.linalg.norm(r[c, :N]), c
        assert np.all(g[c, N:] == np.asarray(fill, dtype=g.dtype))
    assert np.linalg.norm(g[0, :N] - g[1, :N]) > 0.1 * np.linalg.norm(g[0, :N])


def test_rhs_noalloc_rejects_host_buffers(guide_op):
    op, N = guide_op
    b = np.zeros(N, np.complex128)
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_rhs_noalloc(op, [sc.make_source("planewave", "e")], b)
    assert e.value.code == -1


def test_rhs_noalloc_rejects_meshes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    m = cases.synth.waveguide(12.0, 0.5, 0.22, 600, 11, 5, 4.0, 4.0)  # 38,620 triangles > 32,768
    grid = cases.synth.grid_for_mesh(m.V, (512, 64, 64), p=3)
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, (12.1, 1, 2.1, 1, 1.55), grid.n, grid.h, grid.origin, 3, 3, 0.0, 1)
    b = torch.zeros(sc.scabem_mesh_info(mh)[2], dtype=torch.complex64, device="cuda")
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_rhs_noalloc(op, [sc.make_source("planewave", "e")], b, prec=sc.SCABEM_C64)
    assert e.value.code == -1 and "32768" in str(e.value)
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)
