"""Fields off the surface and the decay rate by Poynting's theorem (Sec. III-B) on the GPU.

- scabem_fields_eh: E and H of the interior current set (with the incident
  beam) inside the core and of the exterior set outside, against the
  oracle's post.radiated_fields (the operators of Eqs. 15-16 by the same
  point quadrature), complex128, 1e-10 relative.
- scabem_poynting_rate: the loss around the perimeter, the side flux, the
  cross-section flux and alpha against the oracle's
  post.poynting_decay_rate on the same solution, with a uniform surface
  conductivity, at a cross-section inside an absorber region (1e-9).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from oracle import excitation, mesh, operator, post

pytestmark = pytest.mark.gpu

SIGMA_S = 0.002
BEAM = dict(pos=(0.2, 0.0, 0.0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)


@pytest.fixture(scope="module")
def solved():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    case = cases.guide_small()
    m = case.mesh
    mh = sc.scabem_mesh_create(m.V, m.T, m.region)
    op = sc.scabem_op_create(mh, case.media, case.grid.n, case.grid.h, case.grid.origin, case.grid.p, case.q,
                             case.r_near, 3)
    g = mesh.build(m.V, m.T, m.region, q=case.q)
    sc.scabem_set_sigma(op, per_qpoint=np.full(g.nt * g.q, SIGMA_S))
    src = sc.make_source("beam", "i", **BEAM)
    b = torch.zeros(g.N, dtype=torch.complex128, device="cuda")
    sc.scabem_rhs(op, [src], b, prec=sc.SCABEM_C128)
    x = torch.zeros_like(b)
    sc.scabem_solve(op, b, x, tol=1e-6, restart=100, maxit=20000, refine_tol=1e-9, max_refine=10,
                    prec=sc.SCABEM_C64)
    med = operator.Media(*case.media)
    yield op, g, med, src, x
    sc.scabem_op_destroy(op)
    sc.scabem_mesh_destroy(mh)


def _inc(med):
    ki, zi = med.k[1], med.z[1]
    return lambda q: excitation.beam(q, ki, zi, BEAM["pos"], BEAM["dir"], BEAM["b"], BEAM["pol"])


def test_fields_eh_match_oracle(solved):
    op, g, med, src, x = solved
    xh = x.cpu().numpy()
    (ke, ki), (ze, zi) = med.k, med.z
    inside = np.stack([np.linspace(0.4, 1.6, 9), np.full(9, 0.05), np.full(9, -0.03)], 1)
    outside = np.stack([np.linspace(0.4, 1.6, 9), np.full(9, 0.45), np.full(9, 0.2)], 1)
    E, H = sc.scabem_fields_eh(op, x, inside, side=0, inc=src)
    Eo, Ho = post.radiated_fields(g, xh, inside, ki, zi, "i")
    Ei, Hi = _inc(med)(inside)
    Eo, Ho = Eo + Ei, Ho + Hi
    assert np.linalg.norm(E[0] - Eo) <= 1e-10 * np.linalg.norm(Eo)
    assert np.linalg.norm(H[0] - Ho) <= 1e-10 * np.linalg.norm(Ho)
    E, H = sc.scabem_fields_eh(op, xh, outside, side=1)  # host x is staged
    Eo, Ho = post.radiated_fields(g, xh, outside, ke, ze, "e")
    assert np.linalg.norm(E[0] - Eo) <= 1e-10 * np.linalg.norm(Eo)
    assert np.linalg.norm(H[0] - Ho) <= 1e-10 * np.linalg.norm(Ho)


def test_poynting_rate_matches_oracle(solved):
    op, g, med, src, x = solved
    xh = x.cpu().numpy()
    xc, core, box, slab, n = 0.325, (0.25, 0.11), (0.6, 0.5), 0.025, 6  # x = 0.325 um: inside the left absorber
    out = sc.scabem_poynting_rate(op, x, xc, core, box, slab, n=n, inc=src)[0]
    ref = post.poynting_decay_rate(g, xh, med, SIGMA_S, xc, core, box, slab, inc=_inc(med), n=n)
    for got, want in zip(out, ref):
        assert abs(got - want) <= 1e-9 * max(abs(want), abs(ref[3]) * 1e-3), (out, ref)
    assert out[1] > 0  # the sheet absorbs
