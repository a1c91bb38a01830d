"""GPU: the scale form, N = 4,194,304 (the spiral of 209,715.2 wavelengths, leaf 128, eps
1e-5, complex-FP32 factors), checked on sampled rows that the oracle computes one at a time
with its own Hankel function: the estimate of ||A^_F x - A^ x|| / ||A^_F x|| from 8 sampled
rows must stay below 2 x 10 eps (factor 2: sampling noise), as for the other workloads.

Construction takes minutes on the host at this size, so the test runs only when
HB_SCALE_TEST=1 is set (`HB_SCALE_TEST=1 pytest tests/test_gpu_scale.py -m gpu`).
"""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import efie

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(os.environ.get("HB_SCALE_TEST") != "1", reason="scale test: set HB_SCALE_TEST=1")]


def test_scale_apply_sampled_rows():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    wl = W.SPIRAL_N4194304
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64)
    p = efie.Problem.from_workload(wl)
    x = W.complex_gaussian(wl.n, 70).astype(np.complex64)
    y = hb.hb_apply(f, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    rows = W.sample_rows(wl.n, 8, W.SEED_ROWS)
    cols = np.arange(wl.n)
    exact = np.array([(p.entries(np.array([i]), cols)[0] * p.scale) @ x.astype(np.complex128) for i in rows])
    est = math.sqrt(wl.n / len(rows) * np.sum(np.abs(y[rows] - exact) ** 2)) / np.linalg.norm(y)
    print("sampled relative error estimate", est)
    assert est <= 2 * 10 * wl.eps, est
