"""GPU parity for the variants, through the C ABI: the exact-leaf-LU preconditioner
(HB_OPT_LEAF_LU), explicitly given curves (HB_POLYLINE) and the TFQMR solver of Sec. 4.

Tolerances (stated per test):
* device sweeps vs the host interpreter of the same packed factor, FP64 on both
  sides: 1e-12 (summation order only);
* FP64 compressed apply vs the oracle's dense Z: 10 eps relative (eps = 1e-6);
* GMRES and TFQMR solutions vs the oracle's dense LU solve: 1e-5 relative.
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense, efie

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hb():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    return hb


def _t(a):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def _sweeps_match_host(hb, f, fh, n, seed):
    b = W.complex_gaussian(n, seed)
    for which, fn, op in ((0, hb.hb_lower_solve, hb.HB_OP_N), (1, hb.hb_upper_solve, hb.HB_OP_N),
                          (2, hb.hb_lower_solve, hb.HB_OP_H), (3, hb.hb_upper_solve, hb.HB_OP_H)):
        x = fn(f, _t(b), op).cpu().numpy()
        assert _rel(x, hb.hb_host_sweep(fh, b, which)) <= 1e-12, which


def test_leaf_lu_factor_on_the_device(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128, options=hb.HB_OPT_LEAF_LU)
    fh = hb.hb_factor_host(g, wl.leaf, wl.eps, options=hb.HB_OPT_LEAF_LU)
    _sweeps_match_host(hb, f, fh, wl.n, 41)
    p = efie.Problem.from_workload(wl)
    b = hb.hb_rhs_plane_wave(f, [30.0])
    x, info = hb.hb_gmres(f, b, rtol=1e-6, restart=30, maxit=500)
    x_lu = dense.solve(p.dense(), p.plane_wave(30.0)[:, 0] * p.scale)
    assert info["true_rel_res"] <= 1e-6
    assert _rel(x.cpu().numpy()[0], x_lu) <= 1e-5


def test_polyline_factor_on_the_device(hb):
    # two sine-modulated open curves of 512 segments each
    n_per = 512
    t = np.arange(n_per + 1) / n_per
    c0 = np.stack([25.6 * t, 1.5 * np.sin(2 * math.pi * 3 * t)], axis=1)
    c1 = np.stack([25.6 * t, 6.0 + 0.8 * np.cos(2 * math.pi * 2 * t)], axis=1)
    nodes, starts = np.concatenate([c0, c1]), [0, n_per + 1]
    n, eps = 2 * n_per, 1e-6
    g = hb.hb_geometry_polyline(nodes, starts)
    f = hb.hb_factor(g, 32, eps, form=hb.HB_C128)
    fh = hb.hb_factor_host(g, 32, eps)
    p = efie.Problem(W.POLYLINE, (nodes, starts), n)
    a = p.dense()
    x = W.complex_gaussian(n, 42)
    assert _rel(hb.hb_apply(f, _t(x)).cpu().numpy(), a @ x) <= 10 * eps
    _sweeps_match_host(hb, f, fh, n, 43)
    b = hb.hb_rhs_plane_wave(f, [30.0])
    np.testing.assert_allclose(b.cpu().numpy()[0], p.plane_wave(30.0)[:, 0], atol=1e-12)
    xs, info = hb.hb_gmres(f, b, rtol=1e-6, restart=30, maxit=500)
    x_lu = dense.solve(a, p.plane_wave(30.0)[:, 0] * p.scale)
    assert info["true_rel_res"] <= 1e-6
    assert _rel(xs.cpu().numpy()[0], x_lu) <= 1e-5


@pytest.fixture(scope="module")
def strip_tfqmr(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    p = efie.Problem.from_workload(wl)
    return dict(wl=wl, p=p, a=p.dense(), f=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128),
                f32=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64))


def test_tfqmr_matches_dense_lu(hb, strip_tfqmr):
    # Sec. 4's solver on the device, three plane waves in lockstep, random shadow vectors
    p, a, f = strip_tfqmr["p"], strip_tfqmr["a"], strip_tfqmr["f"]
    angles = [0.0, 30.0, 75.0]
    b = hb.hb_rhs_plane_wave(f, angles)
    rs = _t(W.complex_gaussian(1024, W.SEED_SHADOW, 3).T)
    x, info = hb.hb_tfqmr(f, b, rstar=rs, rtol=1e-6, maxit=400)
    assert info["converged"] == 3 and info["true_rel_res"] <= 1e-6
    xs = x.cpu().numpy()
    for c, phi in enumerate(angles):
        x_lu = dense.solve(a, p.plane_wave(phi)[:, 0] * p.scale)
        assert _rel(xs[c], x_lu) <= 1e-5, phi
        assert info["res_per_rhs"][c] <= 1e-6
    assert max(info["iters_per_rhs"]) < 80          # half steps (one operator product each)


def test_tfqmr_fp32_factors_matches_dense_lu(hb, strip_tfqmr):
    # the same solve with complex-FP32 factors: FP64 vectors and scalars, FP64
    # arithmetic on the FP32-stored operators; the storage rounding (~1e-7 per
    # entry) stays well inside the 1e-5 solution bound of the FP64 form
    p, a, f = strip_tfqmr["p"], strip_tfqmr["a"], strip_tfqmr["f32"]
    angles = [0.0, 30.0, 75.0]
    b = hb.hb_rhs_plane_wave(f, angles)
    rs = _t(W.complex_gaussian(1024, W.SEED_SHADOW, 3).T)
    x, info = hb.hb_tfqmr(f, b, rstar=rs, rtol=1e-6, maxit=400)
    assert info["converged"] == 3 and info["true_rel_res"] <= 1e-6
    xs = x.cpu().numpy()
    for c, phi in enumerate(angles):
        x_lu = dense.solve(a, p.plane_wave(phi)[:, 0] * p.scale)
        assert _rel(xs[c], x_lu) <= 1e-5, phi


def test_tfqmr_adjoint_and_errors(hb, strip_tfqmr):
    p, a, f = strip_tfqmr["p"], strip_tfqmr["a"], strip_tfqmr["f"]
    b = W.complex_gaussian(1024, 44)
    rs = _t(W.complex_gaussian(1024, W.SEED_SHADOW)[None, :])
    x, info = hb.hb_tfqmr(f, _t(b[None, :]), rstar=rs, op=hb.HB_OP_H, rtol=1e-8, maxit=600)
    assert info["true_rel_res"] <= 1e-8
    assert _rel(x.cpu().numpy()[0], dense.solve(a.conj().T, b * p.scale)) <= 1e-5
    bad = b.copy()
    bad[7] = np.nan
    with pytest.raises(hb.HBError):
        hb.hb_tfqmr(f, _t(bad[None, :]), rstar=rs)


def test_residual_double_float_matches_fp64_arithmetic(hb, strip_tfqmr):
    # The refinement residual r = b - A^_F x of the complex-FP32 forms is computed with
    # FP64-accurate arithmetic on the FP32 factors: for 32 or more columns in double-float
    # (pairs of FP32 values, ~48 bits), below that in FP64.  The same 40 columns in one
    # call (double-float) and in two calls of 20 (FP64) must agree to rounding of that
    # accuracy, far below the FP32 apply's 1e-7.
    f = strip_tfqmr["f32"]
    x = W.complex_gaussian(1024, 80, 40).T.copy()
    b = W.complex_gaussian(1024, 81, 40).T.copy()
    r40 = hb.hb_residual(f, _t(b), _t(x)).cpu().numpy()
    r20 = np.concatenate([hb.hb_residual(f, _t(b[:20]), _t(x[:20])).cpu().numpy(),
                          hb.hb_residual(f, _t(b[20:]), _t(x[20:])).cpu().numpy()])
    err = np.linalg.norm(r40 - r20, axis=1) / np.linalg.norm(r20, axis=1)
    assert err.max() <= 1e-12, err.max()
