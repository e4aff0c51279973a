"""Bounded device waits on the GPU, exercised without any fault.

The near-field record rings wait on their own bulk copies with a time limit
and report an expiry through a host-read flag (SCABEM_E_TIMEOUT on the next
call) instead of trapping.  The self-test entry point makes one such wait run
out on an mbarrier that nothing completes; the test checks the status, that
the wait took about its limit, and that the operator still applies correctly
afterwards (the flag was cleared and the context is intact).
"""

import time

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import paper_1004_5076_gb300 as sc
from test_gpu_parity import build

pytestmark = pytest.mark.gpu

E_TIMEOUT = -8


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def test_expired_wait_reports_timeout_and_operator_stays_usable():
    case = cases.plate_thin()
    mh, op, g, med, sig = build(case)
    x = torch.as_tensor(cases.synth.complex_normal(g.N, seed=5)).cuda()
    y0 = torch.empty_like(x)
    sc.scabem_apply(op, x, y0, prec=sc.SCABEM_C128)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    rc = sc.scabem_selftest_wait_limit(op)
    dt = time.perf_counter() - t0
    assert rc == E_TIMEOUT, rc
    assert 0.5 < dt < 30.0, dt
    # the flag was read and cleared: the next apply succeeds and agrees
    y1 = torch.empty_like(x)
    sc.scabem_apply(op, x, y1, prec=sc.SCABEM_C128)
    torch.cuda.synchronize()
    y0n, y1n = y0.cpu().numpy(), y1.cpu().numpy()
    assert np.linalg.norm(y1n - y0n) <= 1e-13 * np.linalg.norm(y0n)
