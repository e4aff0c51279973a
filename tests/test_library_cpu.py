"""Host-side checks of the CUDA library that need no GPU: it builds, loads,
exports every symbol the header declares, and its host topology (RWG edge
table, unknown layout, mesh validation) agrees with the oracle's."""

import os
import re
import subprocess

import numpy as np
import pytest

import synth
import paper_1004_5076_gb300 as sc
from oracle import mesh as omesh

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "scabem.h")


@pytest.fixture(scope="module")
def lib():
    from paper_1004_5076_gb300 import build

    build.build()
    return sc.lib()


def _declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"\b(scabem_[a-z_]+)\s*\(", txt)))


def test_library_exports_every_declared_symbol(lib):
    names = _declared()
    assert "scabem_apply" in names and "scabem_solve" in names
    out = subprocess.run(["nm", "-D", "--defined-only", sc.LIBPATH], capture_output=True, text=True).stdout
    exported = set(re.findall(r" T (scabem_[a-z_]+)", out))
    missing = [n for n in names if n not in exported]
    assert not missing, missing
    for n in names:
        assert hasattr(lib, n)


def test_binding_wraps_every_declared_symbol():
    for n in _declared():
        assert callable(getattr(sc, n)), n


@pytest.mark.parametrize("make", [lambda: synth.icosphere(2), lambda: synth.waveguide(2.0, 0.5, 0.22, 20, 4, 2, 0.5, 0.5)])
def test_edge_table_and_layout_match_oracle(lib, make):
    m = make()
    if m.region.sum() == 0:
        m.region[m.V[m.T].mean(1)[:, 0] > 0.1] = 1
    h = sc.scabem_mesh_create(m.V, m.T, m.region)
    nL, nR, N = sc.scabem_mesh_info(h)
    ev, et, ec = sc.scabem_mesh_edges(h)
    g = omesh.build(m.V, m.T, m.region, q=1)
    assert (nL, nR, N) == (g.nL, g.nR, g.N)
    assert np.array_equal(ev, g.edge_v) and np.array_equal(et, g.edge_t) and np.array_equal(ec, g.edge_class)
    sc.scabem_mesh_destroy(h)


def test_mesh_validation_errors(lib):
    m = synth.icosphere(1)
    # open mesh: drop a triangle
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_mesh_create(m.V, m.T[1:], m.region[1:])
    assert e.value.code == -2
    # inconsistent orientation: flip one triangle
    T = m.T.copy()
    T[0, 1], T[0, 2] = T[0, 2], T[0, 1]
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_mesh_create(m.V, T, m.region)
    assert e.value.code == -2
    # bad region flag
    r = m.region.copy()
    r[0] = 2
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_mesh_create(m.V, m.T, r)
    assert e.value.code == -1
    # non-finite vertex
    V = m.V.copy()
    V[0, 0] = np.nan
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_mesh_create(V, m.T, m.region)
    assert e.value.code == -7


def test_operator_needs_a_gb300(lib):
    """Without an sm_103 device op creation fails loudly; there is no CPU fallback."""
    import torch

    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    m = synth.icosphere(1)
    h = sc.scabem_mesh_create(m.V, m.T, m.region)
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_op_create(h, (2.25, 1, 1, 1, 1.55), (16, 16, 16), 0.2, (-1.5, -1.5, -1.5), 3, 6, 0.3, 3)
    assert e.value.code == -3
    sc.scabem_mesh_destroy(h)


def test_decay_fit_argument_checks_without_a_gpu(lib):
    """scabem_decay_fit rejects a bad grid or sample count (SCABEM_E_ARG) and non-finite samples
    (SCABEM_E_NONFINITE) before looking for a device; valid arguments then need a GB300
    (SCABEM_E_DEVICE here): there is no host fallback."""
    t, E = synth.two_wave_samples(16, 0.0, 1.0, 0.2, 6.0, 1.0, 0.1)
    cases = [((t, E, 0.0, 1.0, 0, 4.0, 8.0, 11), -1), ((t[:3], E[:3], 0.0, 1.0, 5, 4.0, 8.0, 11), -1),
             ((t, E, 0.0, 1.0, 4097, 4.0, 8.0, 4097), -1), ((t, E, 0.0, float("inf"), 5, 4.0, 8.0, 11), -1)]
    for args, code in cases:
        with pytest.raises(sc.ScabemError) as e:
            sc.scabem_decay_fit(*args)
        assert e.value.code == code, args
    bad = E.copy()
    bad[5] = complex(float("nan"), 0.0)
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_decay_fit(t, bad, 0.0, 1.0, 5, 4.0, 8.0, 11)
    assert e.value.code == -7
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_decay_fit(t, E, 0.0, 1.0, 5, 4.0, 8.0, 11)
    assert e.value.code == -3


@pytest.mark.parametrize("make,h_max,p", [(lambda: synth.waveguide(), 0.05, 3), (lambda: synth.icosphere(2), 0.1, 4),
                                          (lambda: synth.waveguide(2.0, 0.5, 0.22, 20, 4, 2, 0.5, 0.5), 0.03, 2)])
def test_grid_plan_keeps_every_stencil_inside(lib, make, h_max, p):
    """scabem_grid_plan: power-of-two transform sizes within the limits, h <= h_max, and every
    stencil base the set-up computes (floor(u - (p-2)/2) with u = (r - origin)/h) inside
    [0, n - p] for the mesh's extreme points, so for every quadrature point."""
    m = make()
    h = sc.scabem_mesh_create(m.V, m.T, m.region)
    plan = sc.scabem_grid_plan(h, h_max, p=p, near_h=3.05)
    n, hh, org = np.array(plan["n"]), plan["h"], np.array(plan["origin"])
    for a, tmax in enumerate((1024, 128, 128)):
        t = 2 * n[a]
        assert 8 <= t <= tmax and t & (t - 1) == 0
    assert 4 * n[1] * n[2] <= 4096 and 0 < hh <= h_max
    assert plan["p"] == p and abs(plan["r_near"] - 3.05 * hh) < 1e-15 and plan["q"] == 6
    u = (m.V - org) / hh
    b = np.floor(u - 0.5 * (p - 2))
    assert b.min() >= 0 and np.all(b.max(axis=0) + p - 1 <= n - 1)
    sc.scabem_mesh_destroy(h)


def test_grid_plan_matches_the_guide_workload_and_rejects_bad_requests(lib):
    m = synth.waveguide()
    h = sc.scabem_mesh_create(m.V, m.T, m.region)
    plan = sc.scabem_grid_plan(h, 0.05)
    assert plan["n"] == (256, 16, 16) and abs(plan["h"] - 12.0 / (256 - 4.5)) < 1e-12
    for args in ((0.005,), (0.05, 5), (-1.0,), (0.05, 3, -1.0)):
        with pytest.raises(sc.ScabemError) as e:
            sc.scabem_grid_plan(h, *args)
        assert e.value.code == -1, args
    sc.scabem_mesh_destroy(h)
