"""Decay-rate fit on the GPU (Sec. III).

Parity: the GPU fit (scabem_decay_fit) against the oracle's fit (post.fit_decay) on seeded
synthetic two-wave samples, without and with noise: the same (alpha, beta) candidate, and the
residual and amplitudes to 1e-9.  Consistency: the decay rate on a probe line (scabem_decay_rate)
is the fit of that line's field (scabem_fields at the same points).
"""

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import cases
import synth
import paper_1004_5076_gb300 as sc
from oracle import post
from test_gpu_parity import build

pytestmark = pytest.mark.gpu

ALPHAS = (0.0, 1.0, 41)
BETAS = (10.0, 12.5, 101)


@pytest.fixture(scope="module", autouse=True)
def _require_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


@pytest.mark.parametrize("noise,seed", [(0.0, 0), (1e-3, 3), (3e-2, 4)])
def test_decay_fit_matches_oracle(noise, seed):
    t, E = synth.two_wave_samples(48, 1.0, 4.0, 0.35, 11.3, 0.8 - 0.3j, 0.02 * np.exp(0.7j), noise=noise, seed=seed)
    out = sc.scabem_decay_fit(t, E, *ALPHAS, *BETAS)
    al, bt, res, a, c = post.fit_decay(t, E, np.linspace(*ALPHAS), np.linspace(*BETAS))
    assert abs(out[0] - al) < 1e-12 and abs(out[1] - bt) < 1e-12, (out, al, bt)
    assert abs(out[2] - res) <= 1e-9 * max(res, 1e-6)
    assert abs(complex(out[3], out[4]) - c / a) < 1e-9
    assert abs(out[5] - abs(a)) < 1e-9 * abs(a)


def test_decay_rate_is_the_fit_of_the_probe_field():
    case = cases.guide_small()
    mh, op, g, med, sig = build(case)
    x = torch.as_tensor(cases.synth.complex_normal(g.N, seed=77) * 1e-2).cuda()
    src = sc.make_source("beam", "i", pos=(0.8, 0, 0), dir=(1, 0, 0), pol=(0, 1, 0), b=0.07)
    p0, t0, t1, n = (0.0, 0.01, -0.005), 0.9, 1.3, 16
    out = sc.scabem_decay_rate(op, x, 0, 1, p0, t0, t1, n, 0.0, 2.0, 21, 10.0, 16.0, 61, inc=src)[0]
    tt = np.array([t0 + (t1 - t0) * i / (n - 1) for i in range(n)])
    pts = np.stack([tt, np.full(n, p0[1]), np.full(n, p0[2])], 1)
    E = sc.scabem_fields(op, x, pts, inc=src)[0][:, 1]
    ref = sc.scabem_decay_fit(tt, E, 0.0, 2.0, 21, 10.0, 16.0, 61)
    assert out[0] == ref[0] and out[1] == ref[1]
    assert np.allclose(out, ref, rtol=1e-12, atol=0.0)


def test_decay_fit_rejects_bad_arguments():
    t, E = synth.two_wave_samples(8, 0.0, 1.0, 0.1, 5.0, 1.0, 0.0)
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_decay_fit(t, E, 0.0, 1.0, 0, 4.0, 6.0, 11)
    assert e.value.code == -1
    E[3] = np.nan
    with pytest.raises(sc.ScabemError) as e:
        sc.scabem_decay_fit(t, E, 0.0, 1.0, 11, 4.0, 6.0, 11)
    assert e.value.code == -7
