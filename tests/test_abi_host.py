"""CPU tests of the C-ABI library: load + exports, host construction and packing.

No compute call reaches the GPU here: hb_factor_host builds the same H-IDBF and
packed program as hb_factor without a device image, and hb_host_apply /
hb_host_sweep execute that packed program in FP64 on the host.
"""
import math
import os
import re

import numpy as np
import pytest

import workloads as W
from oracle import dense, efie, geometry

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def hb():
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    hb.lib()
    return hb


def _declared_symbols():
    src = open(os.path.join(ROOT, "include", "hb.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hb_[a-z0-9_]+)\s*\(", src)))


def test_library_exports_every_declared_symbol(hb):
    lib = hb.lib()
    names = _declared_symbols()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    assert b"sm_103a" in lib.hb_version()


def test_error_paths_without_gpu(hb):
    import ctypes as C
    lib = hb.lib()
    out = C.c_void_p()
    p = (C.c_double * 4)(0, 0, 1, 0)
    assert lib.hb_geometry(99, p, 4, 64, C.byref(out)) == hb._lib.HB_EINVAL
    assert b"unknown kind" in lib.hb_last_error()
    assert lib.hb_geometry(hb.HB_STRIP, p, 4, 0, C.byref(out)) == hb._lib.HB_EINVAL
    g = hb.hb_geometry(hb.HB_STRIP, (0, 0, 1, 0), 96)           # 96 = 32 * 3: not leaf * 2^D
    with pytest.raises(hb.HBError) as e:
        hb.hb_factor_host(g, 32, 1e-6)
    assert e.value.code == hb._lib.HB_EUNSUPPORTED
    g = hb.hb_geometry(hb.HB_STRIP, (0, 0, 3.2, 0), 64)
    with pytest.raises(hb.HBError):
        hb.hb_factor_host(g, 4, 1e-6)                          # leaf below the supported range
    f = hb.hb_factor_host(g, 32, 1e-6)
    # device entry points refuse a host-only factor (no silent CPU path)
    assert lib.hb_apply(f._h, 0, C.c_void_p(8), C.c_void_p(16), 1, 64, None) == hb._lib.HB_EINVAL
    assert b"no device image" in lib.hb_last_error()
    assert lib.hb_tfqmr(f._h, 0, C.c_void_p(8), None, C.c_void_p(16), 1, 64, 1e-6, 10, None, None) == hb._lib.HB_EINVAL
    assert b"no device image" in lib.hb_last_error()
    # execution settings of the device path: refused on a host-only factor and out of range
    assert lib.hb_set_gmres_graph(f._h, 1) == hb._lib.HB_EINVAL
    assert lib.hb_set_gmres_graph(None, 1) == hb._lib.HB_EINVAL
    assert lib.hb_set_sweep_kernel(f._h, 1) == hb._lib.HB_EINVAL
    assert lib.hb_set_wait_limit(f._h, 10) == hb._lib.HB_EINVAL


@pytest.mark.parametrize("name", ["strip_N1024", "spiral_N65536", "semicircle_N262144", "strips8_N131072"])
def test_geometry_matches_oracle(hb, name):
    wl = W.WORKLOADS[name]
    n = min(wl.n, 8192) if wl.kind != W.PARALLEL_STRIPS else 8192
    params = wl.params
    if wl.kind == W.SPIRAL or wl.kind == W.ARC:
        params = wl.params                                      # same curve, coarser sampling
    g = hb.hb_geometry(wl.kind, params, n)
    cen, w = g.segments()
    c2, w2 = geometry.segments(wl.kind, params, n)
    scale = max(1.0, np.abs(c2).max())
    np.testing.assert_allclose(cen, c2, atol=1e-12 * scale, rtol=0)
    np.testing.assert_allclose(w, w2, rtol=1e-9)


def test_tree_bit_exact(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps)
    b, e = hb.hb_tree(f)
    # Alg. 1 recursion: node (v, p) at BFS index 2^v - 1 + p spans [p N/2^v, (p+1) N/2^v)
    exp_b, exp_e = [], []
    for v in range(wl.depth + 1):
        sz = wl.n >> v
        for p in range(1 << v):
            exp_b.append(p * sz)
            exp_e.append((p + 1) * sz)
    assert b.tolist() == exp_b and e.tolist() == exp_e


@pytest.fixture(scope="module")
def strip_host(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps)
    p = efie.Problem.from_workload(wl)
    return wl, f, p, p.dense()


def test_host_factor_stats(hb, strip_host):
    wl, f, p, a = strip_host
    st = hb.hb_factor_info(f)
    assert st["n"] == 1024 and st["leaf"] == 32 and st["depth"] == 5
    assert st["n_butterflies"] == 62
    assert abs(st["scale"] - p.scale) <= 1e-15 * p.scale
    assert 1 <= st["kmax"] < 32
    assert st["nnz_leaf"] == 1024 * 32


def test_host_apply_within_10eps(hb, strip_host):
    wl, f, p, a = strip_host
    for seed in (1, 2):
        x = W.complex_gaussian(wl.n, seed)
        y = hb.hb_host_apply(f, x)
        assert np.linalg.norm(y - a @ x) / np.linalg.norm(a @ x) <= 10 * wl.eps
        yh = hb.hb_host_apply(f, x, hb.HB_OP_H)
        ah = a.conj().T
        assert np.linalg.norm(yh - ah @ x) / np.linalg.norm(ah @ x) <= 10 * wl.eps


def test_host_sweeps_are_triangular_solves(hb, strip_host):
    wl, f, p, a = strip_host
    af = np.stack([hb.hb_host_apply(f, e) for e in np.eye(wl.n, dtype=np.complex128)], axis=1)
    b = W.complex_gaussian(wl.n, 3)
    refs = {0: dense.forward_subst(dense.l_tilde(af), b, unit=True),
            1: dense.back_subst(dense.u_tilde(af), b),
            2: dense.back_subst(dense.l_tilde(af).conj().T, b, unit=True),
            3: dense.forward_subst(dense.u_tilde(af).conj().T, b)}
    for which, ref in refs.items():
        v = hb.hb_host_sweep(f, b, which)
        assert np.linalg.norm(v - ref) / np.linalg.norm(ref) < 1e-12, which


@pytest.mark.parametrize("n,leaf", [(64, 32), (256, 8), (512, 256), (2048, 64)])
def test_host_apply_edge_shapes(hb, n, leaf):
    # D = 1, smallest and largest leaf, odd and even butterfly depths
    g = hb.hb_geometry(W.SPIRAL, (0.25, 2 * math.pi, 6 * math.pi), n)
    f = hb.hb_factor_host(g, leaf, 1e-8)
    p = efie.Problem(W.SPIRAL, (0.25, 2 * math.pi, 6 * math.pi), n)
    a = p.dense()
    x = W.complex_gaussian(n, 4)
    assert np.linalg.norm(hb.hb_host_apply(f, x) - a @ x) / np.linalg.norm(a @ x) <= 1e-7


def test_memory_scaling_of_library_factor(hb):
    # Secs. 1 and 4: O(N log^2 N) storage of the library's (sampled) construction.
    ratios = []
    for n in (4096, 16384, 65536):
        g = hb.hb_geometry(W.STRIP, (0.0, 0.0, n / 20.0, 0.0), n)
        st = hb.hb_factor_info(hb.hb_factor_host(g, 64, 1e-6))
        ratios.append((st["nnz_butterfly"] + st["nnz_leaf"]) / (n * math.log2(n) ** 2))
    assert max(ratios) / min(ratios) < 2.0, ratios
