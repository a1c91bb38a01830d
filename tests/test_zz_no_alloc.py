"""hb_apply_noalloc: the allocation-free apply agrees with hb_apply.

The entry point exists for callers that must not let the library allocate
device memory (a framework whose allocator owns the device budget, a service
that may not allocate after start-up).  It runs the same kernels as hb_apply
with scratch taken from a fixed 16 MiB device array, so its output must match
hb_apply's to the consistency tolerance used for kernel-vs-kernel checks
(1e-12 relative for complex128 factors, 1e-6 for complex64 ones), on
consecutive calls that reuse the shared array.  The cases cover one, three and
forty right-hand sides (forty runs the column-parallel kernels used from 32
columns on), both storage forms, and requests the array cannot hold.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest

import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128)
    f32 = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64)
    return torch, hb, f, wl, f32


def _noalloc(hb, torch, f, x, y, nrhs, ld, op=0):
    return hb.lib().hb_apply_noalloc(f._h, op, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), nrhs, ld,
                                     C.c_void_p(torch.cuda.current_stream().cuda_stream))


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_apply_two_calls(setup):
    torch, hb, f, wl, _ = setup
    n = wl.n
    for call, seed in enumerate((41, 42)):                       # two calls in a row share the array
        x = torch.from_numpy(W.complex_gaussian(n, seed)).cuda()
        ref = hb.hb_apply(f, x).cpu().numpy()
        y = torch.full_like(x, 3.0)
        assert _noalloc(hb, torch, f, x, y, 1, n) == 0, hb.lib().hb_last_error()
        torch.cuda.synchronize()
        assert _rel(y.cpu().numpy(), ref) <= 1e-12, call


def test_noalloc_multi_rhs_and_adjoint(setup):
    torch, hb, f, wl, _ = setup
    n, R, ld = wl.n, 3, wl.n + 8
    xs = W.complex_gaussian(n, 43, R).T.copy()
    xb = torch.zeros((R, ld), dtype=torch.complex128, device="cuda")
    xb[:, :n] = torch.from_numpy(xs).cuda()
    for op in (0, 1):
        ref = hb.hb_apply(f, torch.from_numpy(xs).cuda(), op).cpu().numpy()
        for _ in range(2):
            yb = torch.zeros_like(xb)
            assert _noalloc(hb, torch, f, xb, yb, R, ld, op) == 0, hb.lib().hb_last_error()
            torch.cuda.synchronize()
            y = yb.cpu().numpy()
            for r in range(R):
                assert _rel(y[r, :n], ref[r]) <= 1e-12


def test_noalloc_rejects_oversize_request(setup):
    torch, hb, f, wl, _ = setup
    n, R = wl.n, 4096                                             # scratch far above 16 MiB
    x = torch.zeros((R, n), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(hb, torch, f, x, y, R, n) == hb._lib.HB_EINVAL
    assert b"fixed limit" in hb.lib().hb_last_error()


@pytest.mark.parametrize("form,R", [("c128", 40), ("c64", 1), ("c64", 3), ("c64", 40)])
def test_noalloc_forms_and_column_parallel(setup, form, R):
    # R = 40 takes the column-parallel kernels (one thread per right-hand side)
    torch, hb, f64, wl, f32 = setup
    f = f64 if form == "c128" else f32
    dt = torch.complex128 if form == "c128" else torch.complex64
    tol = 1e-12 if form == "c128" else 1e-6
    n, ld = wl.n, wl.n + 4
    xs = W.complex_gaussian(n, 44 + R, R).T.copy()
    xb = torch.zeros((R, ld), dtype=dt, device="cuda")
    xb[:, :n] = torch.from_numpy(xs).to(dt).cuda()
    for op in (0, 1):
        ref = hb.hb_apply(f, torch.from_numpy(xs).to(dt).cuda(), op).cpu().numpy().reshape(R, n)
        for _ in range(2):                                        # two calls in a row share the array
            yb = torch.full_like(xb, 5.0)
            assert _noalloc(hb, torch, f, xb, yb, R, ld, op) == 0, hb.lib().hb_last_error()
            torch.cuda.synchronize()
            y = yb.cpu().numpy()
            for r in range(R):
                assert _rel(y[r, :n], ref[r]) <= tol
            assert np.all(y[:, n:] == 5.0)                       # padding rows untouched


def test_noalloc_rejects_huge_column_count(setup):
    # a column count whose scratch size would overflow 64-bit arithmetic is
    # rejected before anything is launched
    torch, hb, f, wl, _ = setup
    x = torch.zeros((1, wl.n), dtype=torch.complex128, device="cuda")
    y = torch.zeros_like(x)
    assert _noalloc(hb, torch, f, x, y, 1 << 60, wl.n) == hb._lib.HB_EINVAL
    assert b"fixed limit" in hb.lib().hb_last_error()
