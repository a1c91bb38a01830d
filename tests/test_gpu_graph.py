"""GPU: hb_gmres with every restart cycle run as one CUDA graph launch (the
Arnoldi steps, CGS2, the Givens rotations, the convergence test and the
least-squares solve on the device), against the oracle's dense LU solve and
against the host-driven loop.

Bounds: solutions within 1e-5 of the dense LU solve (N <= 4096), the bound of
every solve; the two loops compute the same iteration (FP64 Givens on both
sides, rounded in a different order in the last bits), so their solutions
agree to 1e-5 as well and their iteration counts to within one step per cycle.
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


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


@pytest.fixture(scope="module")
def semi(hb):
    # semicircle at N = 4096, 20 segments per wavelength (the batching workload's family)
    wl = W.arc(4096, 64, 1e-6, radius=4096 / 20.0 / math.pi)
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    p = efie.Problem.from_workload(wl)
    return dict(wl=wl, g=g, p=p, a=p.dense(), f64=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128),
                f32=hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C64))


def _both_loops(hb, f, b, **kw):
    out = {}
    for on in (1, 0):
        hb.hb_set_gmres_graph(f, on)
        x, info = hb.hb_gmres(f, b, **kw)
        out[on] = (x.cpu().numpy(), info)
    hb.hb_set_gmres_graph(f, 1)
    return out


@pytest.mark.parametrize("form", ["f64", "f32"])
def test_graph_cycle_matches_dense_lu_and_host_loop(hb, semi, form):
    p, a, f = semi["p"], semi["a"], semi[form]
    phis = [5.0, 61.0, 118.0, 170.0]
    x_lu = dense.solve(a, p.plane_wave(phis) * p.scale)
    res = _both_loops(hb, f, hb.hb_rhs_plane_wave(f, phis), rtol=1e-6, restart=30, maxit=600)
    xg, ig = res[1]
    xh, ih = res[0]
    assert ig["converged"] == 4 and ig["true_rel_res"] <= 1e-6
    assert ig["graph_launches"] == ig["restarts"] >= 1 and ih["graph_launches"] == 0
    for r in range(4):
        assert _rel(xg[r], x_lu[:, r]) <= 1e-5, r
        assert _rel(xg[r], xh[r]) <= 1e-5, r
    assert abs(ig["iters"] - ih["iters"]) <= ig["restarts"]


def test_graph_cycle_split_form_tensor_cores_and_column_sweeps(hb, semi):
    # 40 columns: the tensor-core leaf contractions and, once tuned, the
    # column-partitioned sweep kernel inside the captured cycle
    p, a, g, wl = semi["p"], semi["a"], semi["g"], semi["wl"]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_SPLIT_BF16)
    phis = list(np.linspace(0.0, 175.0, 40))
    x_lu = dense.solve(a, p.plane_wave(phis) * p.scale)
    b = hb.hb_rhs_plane_wave(f, phis)
    for kernel in (1, 0):
        hb.hb_set_sweep_kernel(f, kernel)
        res = _both_loops(hb, f, b, rtol=1e-6, restart=30, maxit=600)
        xg, ig = res[1]
        assert ig["converged"] == 40 and ig["graph_launches"] == ig["restarts"] >= 1
        err = max(_rel(xg[r], x_lu[:, r]) for r in range(40))
        assert err <= 1e-5, (kernel, err)
        assert max(_rel(xg[r], res[0][0][r]) for r in range(40)) <= 1e-5
    hb.hb_set_sweep_kernel(f, -1)


def test_graph_cycle_adjoint(hb, semi):
    import torch
    p, a, f = semi["p"], semi["a"], semi["f64"]
    bt = W.complex_gaussian(4096, 41, 3)                 # (N, 3)
    x, info = hb.hb_gmres(f, torch.from_numpy(np.ascontiguousarray(bt.T)).cuda(), op=hb.HB_OP_H, rtol=1e-8,
                          maxit=600)
    assert info["graph_launches"] >= 1
    x_ref = dense.solve(a.conj().T, bt * p.scale)
    xs = x.cpu().numpy()
    for r in range(3):
        assert _rel(xs[r], x_ref[:, r]) <= 1e-5


def test_graph_cycle_step_limit_and_single_column(hb, semi):
    f = semi["f32"]
    b = hb.hb_rhs_plane_wave(f, [20.0, 40.0])
    _, info = hb.hb_gmres(f, b, rtol=1e-12, restart=30, maxit=7, check=False)
    assert info["status"] == hb._lib.HB_ENOCONV and info["iters"] == 7 and info["graph_launches"] == 1
    _, info = hb.hb_gmres(f, hb.hb_rhs_plane_wave(f, [20.0]), rtol=1e-6)
    assert info["graph_launches"] == 0 and info["true_rel_res"] <= 1e-6   # one column: host-driven loop


def test_graph_cycle_profile_counts(hb, semi):
    # the timing events inside the graph are read for the steps that ran only
    f = semi["f32"]
    b = hb.hb_rhs_plane_wave(f, [30.0, 90.0, 150.0])
    hb.hb_gmres(f, b)                                    # capture without events
    hb.hb_profile(f, True)                               # recapture with events on the next call
    _, info = hb.hb_gmres(f, b)
    n_sweep, ms_sweep = hb.hb_profile_read(f, 1)
    n_launch, _ = hb.hb_profile_read(f, 2)
    hb.hb_profile(f, False)
    assert info["graph_launches"] >= 1
    assert n_sweep == 2 * info["iters"] and ms_sweep > 0
    assert n_launch > 20 * info["graph_launches"]


def test_graph_cycle_reports_timeout(hb, semi):
    # a one-poll wait limit makes the cooperative sweep's grid barrier give up
    # inside the graph: the solve returns HB_ETIMEOUT after the launch, the flag
    # is cleared, and with the normal limit the next solve (recaptured) converges
    wl, g = semi["wl"], semi["g"]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_C128)
    lib = hb.lib()
    assert lib.hb_set_sweep_grid_min(f._h, 1) >= 1
    assert lib.hb_set_wait_limit(f._h, 1) == 0
    b = hb.hb_rhs_plane_wave(f, [30.0, 60.0])
    _, info = hb.hb_gmres(f, b, check=False)
    assert info["status"] == hb._lib.HB_ETIMEOUT
    assert lib.hb_set_wait_limit(f._h, 1 << 24) == 0
    _, info = hb.hb_gmres(f, b)
    assert info["status"] == 0 and info["true_rel_res"] <= 1e-6 and info["graph_launches"] >= 1


def test_graph_cycle_256_columns_vs_dense_lu(hb, semi):
    # The bench's column count: 256 right-hand sides take the fused first CGS2
    # update with the second pass's dot products (k_sub_dots), the tensor-core
    # leaf contractions and the tuned sweep kernel inside the captured cycle;
    # sampled columns against the dense LU solve, and the host-driven loop.
    p, a, g, wl = semi["p"], semi["a"], semi["g"], semi["wl"]
    f = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_SPLIT_BF16)
    hb.hb_autotune(f, 256)
    phis = 180.0 * np.arange(256) / 256
    cols = [0, 37, 101, 128, 190, 255]
    x_lu = dense.solve(a, p.plane_wave(phis[cols]) * p.scale)
    res = _both_loops(hb, f, hb.hb_rhs_plane_wave(f, phis), rtol=1e-6, restart=30, maxit=600)
    for on in (1, 0):
        xs, info = res[on]
        assert info["converged"] == 256 and info["true_rel_res"] <= 1e-6
        assert (info["graph_launches"] >= 1) == (on == 1)
        for j, c in enumerate(cols):
            assert _rel(xs[c], x_lu[:, j]) <= 1e-5, (on, c)
