"""GB300-native H-IDBF-LU (arXiv:1901.11371): Python binding of libhb.

Functions carry the names of the C ABI (include/hb.h) and only marshal
arguments: PyTorch CUDA tensors provide device memory and the current stream;
every step of apply / sweeps / GMRES runs in the library's CUDA kernels.

Tensor convention: a block of R right-hand sides is a contiguous tensor of
shape (R, N) (row r = column r of the ABI's column-major block, ld = N); a
single vector may be given with shape (N,).
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (HB_ARC, HB_C64, HB_C128, HB_OP_H, HB_OP_N, HB_OPT_LEAF_LU, HB_OPT_SWEEP_WINDOW_MIN, HB_PARALLEL_STRIPS, HB_POLYLINE,
                   HB_SPIRAL, HB_SPLIT_BF16, HB_STRIP, HBError)

__all__ = ["HB_STRIP", "HB_SPIRAL", "HB_ARC", "HB_PARALLEL_STRIPS", "HB_POLYLINE", "HB_C128", "HB_C64",
           "HB_SPLIT_BF16", "HB_OP_N", "HB_OP_H", "HB_OPT_LEAF_LU", "HB_OPT_SWEEP_WINDOW_MIN", "HBError", "Geometry", "Factor", "hb_geometry",
           "hb_geometry_polyline", "hb_factor", "hb_factor_host",
           "hb_factor_info", "hb_tree", "hb_apply", "hb_apply_adjoint", "hb_precond_solve", "hb_lower_solve",
           "hb_upper_solve", "hb_residual", "hb_gmres", "hb_tfqmr", "hb_rhs_plane_wave", "hb_far_field", "hb_monostatic",
           "hb_host_apply", "hb_host_apply_plan", "hb_host_tc_apply", "hb_host_sweep", "hb_host_sweep_sched", "hb_far_field_adjoint", "hb_profile", "hb_profile_read", "hb_autotune", "hb_autotune_times", "hb_set_sweep_kernel", "hb_set_gmres_graph", "lib"]


def lib():
    return _lib.load()


def _stream(stream=None):
    import torch
    if stream is None:
        return C.c_void_p(torch.cuda.current_stream().cuda_stream)
    return C.c_void_p(int(stream))


class Geometry:
    def __init__(self, handle, n):
        self._h = C.c_void_p(handle)
        self.n = int(n)

    def segments(self):
        cen = np.empty(2 * self.n)
        w = np.empty(self.n)
        _lib.check(lib().hb_geometry_segments(self._h, cen.ctypes.data_as(C.POINTER(C.c_double)),
                                              w.ctypes.data_as(C.POINTER(C.c_double))))
        return cen.reshape(self.n, 2), w

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.hb_geometry_destroy(h)
            self._h = None


class Factor:
    def __init__(self, handle, form, host_only=False):
        self._h = C.c_void_p(handle)
        self.form = form
        self.host_only = host_only
        st = hb_factor_info(self)
        self.n = int(st["n"])
        self.leaf = int(st["leaf"])

    @property
    def vec_dtype(self):
        import torch
        return torch.complex128 if self.form == HB_C128 else torch.complex64

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value and _lib._lib is not None:
            _lib._lib.hb_factor_destroy(h)
            self._h = None


def hb_geometry(kind, params, n_segments):
    p = (C.c_double * len(params))(*[float(v) for v in params])
    out = C.c_void_p()
    _lib.check(lib().hb_geometry(int(kind), p, len(params), int(n_segments), C.byref(out)))
    return Geometry(out.value, n_segments)


def hb_geometry_polyline(nodes, curve_starts=(0,)):
    """Scatterer from explicit nodes (array (nnodes, 2), wavelengths); curve c uses nodes
    curve_starts[c] .. curve_starts[c+1]-1, one segment per pair of consecutive nodes."""
    xy = np.ascontiguousarray(np.asarray(nodes, dtype=np.float64).reshape(-1, 2))
    st = np.ascontiguousarray(np.asarray(curve_starts, dtype=np.int64))
    out = C.c_void_p()
    _lib.check(lib().hb_geometry_polyline(xy.ctypes.data_as(C.POINTER(C.c_double)),
                                          st.ctypes.data_as(C.POINTER(C.c_int64)), int(len(st)), int(len(xy)),
                                          C.byref(out)))
    return Geometry(out.value, len(xy) - len(st))


def hb_factor(geom, leaf, eps, form=HB_C128, wavelength=1.0, eta0=376.73, gamma=1.781072, seed=0, stream=None,
              options=0):
    """Build and upload the H-IDBF factor; options: HB_OPT_* bits (HB_OPT_LEAF_LU: exact leaf LU)."""
    out = C.c_void_p()
    _lib.check(lib().hb_factor_ex(geom._h, wavelength, eta0, gamma, int(leaf), float(eps), int(form), int(seed),
                                  int(options), _stream(stream), C.byref(out)))
    return Factor(out.value, form)


def hb_factor_host(geom, leaf, eps, wavelength=1.0, eta0=376.73, gamma=1.781072, seed=0, options=0):
    out = C.c_void_p()
    _lib.check(lib().hb_factor_host_ex(geom._h, wavelength, eta0, gamma, int(leaf), float(eps), int(seed),
                                       int(options), C.byref(out)))
    return Factor(out.value, HB_C128, host_only=True)


def hb_factor_info(f):
    st = _lib.FactorStats()
    _lib.check(lib().hb_factor_info(f._h, C.byref(st)))
    d = {name: getattr(st, name) for name, _ in st._fields_ if not name.startswith("pad")}
    d["kmax_depth"] = list(st.kmax_depth)[: st.depth]
    d["kavg_depth"] = list(st.kavg_depth)[: st.depth]
    return d


def hb_tree(f):
    st = hb_factor_info(f)
    nodes = 2 * (st["n"] // st["leaf"]) - 1
    b = np.empty(nodes, dtype=np.int64)
    e = np.empty(nodes, dtype=np.int64)
    _lib.check(lib().hb_tree(f._h, b.ctypes.data_as(C.POINTER(C.c_int64)), e.ctypes.data_as(C.POINTER(C.c_int64))))
    return b, e


def _block(t, n, dtype):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise HBError(_lib.HB_EINVAL, "expected a CUDA tensor")
    if t.dtype != dtype:
        raise HBError(_lib.HB_EINVAL, f"expected dtype {dtype}, got {t.dtype}")
    if t.dim() == 1:
        if t.shape[0] != n:
            raise HBError(_lib.HB_EINVAL, "length mismatch")
        return t.contiguous(), 1
    if t.dim() != 2 or t.shape[1] != n:
        raise HBError(_lib.HB_EINVAL, "expected shape (R, N)")
    return t.contiguous(), t.shape[0]


def hb_apply(f, x, op=HB_OP_N, out=None, stream=None):
    import torch
    x, R = _block(x, f.n, f.vec_dtype)
    y = torch.empty_like(x) if out is None else out
    _lib.check(lib().hb_apply(f._h, int(op), C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), R, f.n,
                              _stream(stream)))
    return y


def hb_apply_adjoint(f, x, out=None, stream=None):
    return hb_apply(f, x, HB_OP_H, out, stream)


def _sweep_call(fn, f, b, op, out, stream, check_status):
    import torch
    b, R = _block(b, f.n, f.vec_dtype)
    x = torch.empty_like(b) if out is None else out
    _lib.check(fn(f._h, int(op), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), R, f.n, _stream(stream)))
    if check_status:
        # synchronises the stream; raises HB_ETIMEOUT if a bounded wait of the sweep expired
        _lib.check(lib().hb_status(f._h, _stream(stream)))
    return x


def hb_precond_solve(f, b, op=HB_OP_N, out=None, stream=None, check_status=True):
    return _sweep_call(lib().hb_precond_solve, f, b, op, out, stream, check_status)


def hb_lower_solve(f, b, op=HB_OP_N, out=None, stream=None, check_status=True):
    return _sweep_call(lib().hb_lower_solve, f, b, op, out, stream, check_status)


def hb_upper_solve(f, b, op=HB_OP_N, out=None, stream=None, check_status=True):
    return _sweep_call(lib().hb_upper_solve, f, b, op, out, stream, check_status)


def hb_residual(f, b, x, op=HB_OP_N, stream=None):
    import torch
    b, R = _block(b, f.n, torch.complex128)
    x, R2 = _block(x, f.n, torch.complex128)
    r = torch.empty_like(b)
    _lib.check(lib().hb_residual(f._h, int(op), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()),
                                 C.c_void_p(r.data_ptr()), R, f.n, _stream(stream)))
    return r


def hb_gmres(f, b_phys, op=HB_OP_N, restart=30, rtol=1e-6, maxit=1000, out=None, stream=None, check=True):
    """Solve A x = b_phys (complex128 physical excitation).  Returns (x, info dict)."""
    import torch
    b, R = _block(b_phys, f.n, torch.complex128)
    x = torch.empty_like(b) if out is None else out
    info = _lib.GmresInfo()
    it = (C.c_int32 * R)()
    rr = (C.c_double * R)()
    info.iters_per_rhs = C.cast(it, C.POINTER(C.c_int32))
    info.res_per_rhs = C.cast(rr, C.POINTER(C.c_double))
    rc = lib().hb_gmres(f._h, int(op), C.c_void_p(b.data_ptr()), C.c_void_p(x.data_ptr()), R, f.n, int(restart),
                        float(rtol), int(maxit), C.byref(info), _stream(stream))
    d = dict(iters=info.iters, restarts=info.restarts, ir_steps=info.ir_steps, converged=info.converged,
             true_rel_res=info.true_rel_res, precond_rel_res=info.precond_rel_res, seconds=info.seconds,
             iters_per_rhs=list(it), res_per_rhs=list(rr), graph_launches=info.graph_launches, status=rc)
    if check and rc not in (_lib.HB_OK,):
        _lib.check(rc)
    return x, d


def hb_tfqmr(f, b_phys, rstar=None, op=HB_OP_N, rtol=1e-6, maxit=2000, out=None, stream=None, check=True):
    """TFQMR (Sec. 4) on the split system; rstar: shadow vectors shaped like b (None: L~^{-1} b).
    Returns (x, info dict); info["iters"] counts half steps."""
    import torch
    b, R = _block(b_phys, f.n, torch.complex128)
    rs = None
    if rstar is not None:
        rs, R2 = _block(rstar, f.n, torch.complex128)
        if R2 != R:
            raise HBError(_lib.HB_EINVAL, "rstar must have the shape of b")
    x = torch.empty_like(b) if out is None else out
    info = _lib.GmresInfo()
    it = (C.c_int32 * R)()
    rr = (C.c_double * R)()
    info.iters_per_rhs = C.cast(it, C.POINTER(C.c_int32))
    info.res_per_rhs = C.cast(rr, C.POINTER(C.c_double))
    rc = lib().hb_tfqmr(f._h, int(op), C.c_void_p(b.data_ptr()), C.c_void_p(rs.data_ptr() if rs is not None else None),
                        C.c_void_p(x.data_ptr()), R, f.n, float(rtol), int(maxit), C.byref(info), _stream(stream))
    d = dict(iters=info.iters, checks=info.restarts, converged=info.converged, true_rel_res=info.true_rel_res,
             bound=info.precond_rel_res, seconds=info.seconds, iters_per_rhs=list(it), res_per_rhs=list(rr), status=rc)
    if check and rc not in (_lib.HB_OK,):
        _lib.check(rc)
    return x, d


def hb_rhs_plane_wave(f, phi_deg, stream=None):
    import torch
    phi = np.ascontiguousarray(np.atleast_1d(np.asarray(phi_deg, dtype=np.float64)))
    R = phi.shape[0]
    b = torch.empty((R, f.n), dtype=torch.complex128, device="cuda")
    _lib.check(lib().hb_rhs_plane_wave(f._h, phi.ctypes.data_as(C.POINTER(C.c_double)), R,
                                       C.c_void_p(b.data_ptr()), f.n, _stream(stream)))
    return b


def hb_far_field(f, x, phi_obs_deg, stream=None):
    import torch
    x, R = _block(x, f.n, torch.complex128)
    phi = np.ascontiguousarray(np.atleast_1d(np.asarray(phi_obs_deg, dtype=np.float64)))
    out = torch.empty((R, phi.shape[0]), dtype=torch.complex128, device="cuda")
    _lib.check(lib().hb_far_field(f._h, C.c_void_p(x.data_ptr()), R, f.n, phi.ctypes.data_as(C.POINTER(C.c_double)),
                                  phi.shape[0], C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def hb_far_field_adjoint(f, g, phi_obs_deg, stream=None):
    """out = F^H g for g of shape (R, nobs) (complex128); returns (R, N)."""
    import torch
    if not (isinstance(g, torch.Tensor) and g.is_cuda and g.dtype == torch.complex128 and g.dim() == 2):
        raise HBError(_lib.HB_EINVAL, "expected a complex128 CUDA tensor of shape (R, nobs)")
    g = g.contiguous()
    phi = np.ascontiguousarray(np.atleast_1d(np.asarray(phi_obs_deg, dtype=np.float64)))
    out = torch.empty((g.shape[0], f.n), dtype=torch.complex128, device="cuda")
    _lib.check(lib().hb_far_field_adjoint(f._h, C.c_void_p(g.data_ptr()), g.shape[0],
                                          phi.ctypes.data_as(C.POINTER(C.c_double)), phi.shape[0],
                                          C.c_void_p(out.data_ptr()), f.n, _stream(stream)))
    return out


def hb_monostatic(f, x, phi_deg, stream=None):
    import torch
    x, R = _block(x, f.n, torch.complex128)
    phi = np.ascontiguousarray(np.atleast_1d(np.asarray(phi_deg, dtype=np.float64)))
    out = torch.empty((R,), dtype=torch.complex128, device="cuda")
    _lib.check(lib().hb_monostatic(f._h, C.c_void_p(x.data_ptr()), R, f.n, phi.ctypes.data_as(C.POINTER(C.c_double)),
                                   C.c_void_p(out.data_ptr()), _stream(stream)))
    return out


def hb_autotune(f, nrhs, stream=None):
    """Pick the fastest sweep kernel / segmentation for `nrhs` right-hand sides; returns the chosen
    threshold (0: the column-partitioned kernel)."""
    ch = C.c_int()
    _lib.check(lib().hb_autotune(f._h, int(nrhs), _stream(stream), C.byref(ch)))
    return ch.value


def hb_autotune_times(f, nrhs):
    """{threshold: ms per sweep} of the last hb_autotune for the class of `nrhs` ({} if untuned;
    threshold 0: the column-partitioned kernel)."""
    ms = (C.c_float * 7)()
    gm = (C.c_int * 7)()
    n = lib().hb_autotune_times(f._h, int(nrhs), ms, gm, 7)
    if n < 0:
        _lib.check(n)
    return {int(gm[i]): float(ms[i]) for i in range(n)}


def hb_set_gmres_graph(f, on):
    """1: hb_gmres runs each restart cycle as one CUDA graph launch (nrhs >= 2); 0: host-driven loop."""
    _lib.check(lib().hb_set_gmres_graph(f._h, int(bool(on))))


def hb_set_sweep_kernel(f, kind):
    """Sweep kernel: -1 the autotuner's choice, 0 cooperative, 1 column-partitioned."""
    _lib.check(lib().hb_set_sweep_kernel(f._h, int(kind)))


def hb_profile(f, enable=True):
    _lib.check(lib().hb_profile(f._h, 1 if enable else 0))


def hb_profile_read(f, kind):
    cnt = C.c_int64()
    ms = C.c_double()
    _lib.check(lib().hb_profile_read(f._h, int(kind), C.byref(cnt), C.byref(ms)))
    return int(cnt.value), float(ms.value)


def hb_host_apply(f, x, op=HB_OP_N):
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    y = np.empty_like(x)
    _lib.check(lib().hb_host_apply(f._h, int(op), x.ctypes.data_as(C.POINTER(C.c_double)),
                                   y.ctypes.data_as(C.POINTER(C.c_double))))
    return y


def hb_host_apply_plan(f, x, op=HB_OP_N, grid=152, factor_bytes=8):
    """Host execution of the persistent single-column apply's schedule (verification without a
    GPU).  Returns (y, number of staging batches)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    y = np.empty_like(x)
    rc = lib().hb_host_apply_plan(f._h, int(op), int(grid), int(factor_bytes),
                                  x.ctypes.data_as(C.POINTER(C.c_double)), y.ctypes.data_as(C.POINTER(C.c_double)))
    if rc < 0:
        _lib.check(rc)
    return y, rc


def hb_host_tc_apply(f, x):
    """Host emulation of the split-BF16 tensor-core forward apply of one column (verification
    without a GPU).  Returns (y, number of operand chunks)."""
    x = np.ascontiguousarray(np.asarray(x, dtype=np.complex128))
    y = np.empty_like(x)
    rc = lib().hb_host_tc_apply(f._h, x.ctypes.data_as(C.POINTER(C.c_double)), y.ctypes.data_as(C.POINTER(C.c_double)))
    if rc < 0:
        _lib.check(rc)
    return y, rc


def hb_host_sweep(f, b, which):
    v = np.array(b, dtype=np.complex128, copy=True)
    _lib.check(lib().hb_host_sweep(f._h, int(which), v.ctypes.data_as(C.POINTER(C.c_double))))
    return v


def hb_host_sweep_sched(f, b, which, coef_bytes=16, win_slots=0):
    """Host execution of the column-partitioned sweep kernel's schedule for one column
    (verification without a GPU).  Returns (x, number of batches)."""
    v = np.array(b, dtype=np.complex128, copy=True)
    rc = lib().hb_host_sweep_sched(f._h, int(which), int(coef_bytes), int(win_slots),
                                   v.ctypes.data_as(C.POINTER(C.c_double)))
    if rc < 0:
        _lib.check(rc)
    return v, rc
