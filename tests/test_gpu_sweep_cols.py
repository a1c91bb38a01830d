"""GPU: the column-partitioned sweep kernel (k_sweep_cols) through the C ABI.

Every CTA runs a whole sweep (Algs. 3 / 4) for its own one or two right-hand
sides from host-built schedules.  Checked here:
* all four sweeps against the FP64 host sweep of the same factor (the packed
  program's own interpreter), for 1 .. 300 right-hand sides (one column per CTA up
  to the SM count, two beyond), with the full resident window and with the
  smallest one (every butterfly above two leaves then runs as global phases,
  reading the vectors and a CTA-private state in global memory): complex-FP32
  rounding, bound 1e-5 relative per column as for the cooperative kernel;
* 256 right-hand sides on the N = 4096 semicircle against the oracle's exact
  entry-wise triangles (Eqs. (Lt), (Ut)), bound 1e-6 as for the cooperative kernel;
* the same columns from both kernels agree;
* a wait limit of one poll ends the sweep with HB_ETIMEOUT, and the next sweep is right;
* the complex128 form has no schedules (HB_EUNSUPPORTED).
"""
import ctypes as C
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


def _t(a, dtype=None):
    import torch
    t = torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t if dtype is None else t.to(dtype)


@pytest.fixture(scope="module")
def strip(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    return dict(wl=wl, g=g, fh=hb.hb_factor_host(g, wl.leaf, wl.eps),
                full=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64),
                small=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64, options=hb.HB_OPT_SWEEP_WINDOW_MIN))


def _calls(hb):
    return [(hb.hb_lower_solve, hb.HB_OP_N), (hb.hb_upper_solve, hb.HB_OP_N),
            (hb.hb_lower_solve, hb.HB_OP_H), (hb.hb_upper_solve, hb.HB_OP_H)]


@pytest.mark.parametrize("R", [1, 2, 3, 40, 160, 300])
@pytest.mark.parametrize("window", ["full", "small"])
def test_sweeps_vs_host_interpreter(hb, strip, R, window):
    import torch
    f = strip[window]
    hb.hb_set_sweep_kernel(f, 1)
    b = W.complex_gaussian(1024, 50 + R, R).T.copy()      # [R, n]
    rows = sorted(set([0, R // 2, R - 1]))                  # first, middle and last CTA's columns
    for w, (fn, op) in enumerate(_calls(hb)):
        ref = np.stack([hb.hb_host_sweep(strip["fh"], b[r], w) for r in rows])
        bb = _t(b[0] if R == 1 else b, torch.complex64)
        x = fn(f, bb, op).cpu().numpy().astype(np.complex128).reshape(R, -1)[rows]
        err = np.linalg.norm(x - ref, axis=1) / np.linalg.norm(ref, axis=1)
        assert err.max() <= 1e-5, (window, R, w, err.max())


def test_kernels_agree(hb, strip):
    import torch
    f = strip["full"]
    R = 200
    b = _t(W.complex_gaussian(1024, 60, R).T.copy(), torch.complex64)
    for fn, op in _calls(hb):
        hb.hb_set_sweep_kernel(f, 0)
        x0 = fn(f, b, op).cpu().numpy().astype(np.complex128)
        hb.hb_set_sweep_kernel(f, 1)
        x1 = fn(f, b, op).cpu().numpy().astype(np.complex128)
        err = np.linalg.norm(x1 - x0, axis=1) / np.linalg.norm(x0, axis=1)
        assert err.max() <= 1e-5


def test_256_columns_vs_oracle_triangles(hb):
    # semicircle N = 4096 (20 segments per wavelength), all four sweeps, 256 columns,
    # against the oracle's exact entry-wise triangles solved by its own substitution
    import torch
    wl = W.arc(4096, 64, 1e-6, radius=4096 / 20.0 / math.pi)
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    a = efie.Problem.from_workload(wl).dense()
    R = 256
    b = W.complex_gaussian(4096, 36, R)
    lt, ut = dense.l_tilde(a), dense.u_tilde(a)
    refs = [dense.forward_subst(lt, b, unit=True), dense.back_subst(ut, b),
            dense.back_subst(lt.conj().T, b, unit=True), dense.forward_subst(ut.conj().T, b)]
    for opts in (0, hb.HB_OPT_SWEEP_WINDOW_MIN):
        f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64, options=opts)
        hb.hb_set_sweep_kernel(f, 1)
        bt = _t(b.T.copy(), torch.complex64)
        for w, (fn, op) in enumerate(_calls(hb)):
            x = fn(f, bt, op).cpu().numpy().astype(np.complex128).T
            e = np.linalg.norm(x - refs[w], axis=0) / np.linalg.norm(refs[w], axis=0)
            assert e.max() <= 1e-6, (opts, w, e.max())


def test_autotune_may_choose_it(hb, strip):
    import torch
    f = strip["full"]
    hb.hb_set_sweep_kernel(f, -1)
    chosen = hb.hb_autotune(f, 256)
    times = hb.hb_autotune_times(f, 256)
    assert 0 in times and len(times) == 7
    assert (chosen == 0) == (times[0] < min(v for k, v in times.items() if k != 0))
    b = W.complex_gaussian(1024, 61, 256).T.copy()
    x = hb.hb_lower_solve(f, _t(b, torch.complex64)).cpu().numpy().astype(np.complex128)
    ref = hb.hb_host_sweep(strip["fh"], b[7], 0)
    assert np.linalg.norm(x[7] - ref) / np.linalg.norm(ref) <= 1e-5


def test_bounded_wait_reports_timeout(hb, strip):
    # host-side fault injection: a wait limit of one poll makes the first wait for a
    # staged batch give up; the sweep returns, hb_status reports HB_ETIMEOUT (and clears
    # it), and the next sweep with the normal limit is right
    import torch
    wl, g = strip["wl"], strip["g"]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64)
    hb.hb_set_sweep_kernel(f, 1)
    lib = hb.lib()
    b = W.complex_gaussian(1024, 62, 40).T.copy()
    bb = _t(b, torch.complex64)
    assert lib.hb_set_wait_limit(f._h, 1) == 0
    hb.hb_lower_solve(f, bb, check_status=False)
    rc = lib.hb_status(f._h, C.c_void_p(torch.cuda.current_stream().cuda_stream))
    assert rc == hb._lib.HB_ETIMEOUT
    assert lib.hb_set_wait_limit(f._h, 1 << 24) == 0
    x = hb.hb_lower_solve(f, bb).cpu().numpy().astype(np.complex128)
    ref = hb.hb_host_sweep(strip["fh"], b[5], 0)
    assert np.linalg.norm(x[5] - ref) / np.linalg.norm(ref) <= 1e-5


def test_complex128_has_no_schedules(hb, strip):
    wl, g = strip["wl"], strip["g"]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128)
    with pytest.raises(hb.HBError) as ei:
        hb.hb_set_sweep_kernel(f, 1)
    assert ei.value.code == hb._lib.HB_EUNSUPPORTED
    hb.hb_set_sweep_kernel(f, 0)
    hb.hb_set_sweep_kernel(f, -1)
