"""Column-partitioned sweep schedules (kernel k_sweep_cols), checked on the host.

The schedule writes every butterfly phase of Algs. 3 / 4 as a sparse product in
row form and every sweep-leaf phase as its packed triangle; its host executor
reads rows, coefficients and slots from the batch images exactly as the kernel
does.  With complex128 coefficients it must reproduce the packed program's own
host sweep to rounding (1e-13), for all four sweeps, with the full resident
window and with the smallest one (every butterfly above two leaves then runs
as global phases); with complex64 coefficients (the device form) to the
storage rounding of the coefficients.
"""
import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def hb():
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as m
    return m


@pytest.fixture(scope="module")
def strip_host(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    return wl, hb.hb_factor_host(g, wl.leaf, wl.eps)


def _rel(a, b):
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("which", [0, 1, 2, 3])
def test_schedule_matches_host_sweep(hb, strip_host, which):
    wl, f = strip_host
    b = W.complex_gaussian(wl.n, 40)
    ref = hb.hb_host_sweep(f, b, which)
    x_full, nb_full = hb.hb_host_sweep_sched(f, b, which, 16)
    x_min, nb_min = hb.hb_host_sweep_sched(f, b, which, 16, win_slots=512)
    assert _rel(x_full, ref) <= 1e-13
    assert _rel(x_min, ref) <= 1e-13
    assert nb_min != nb_full          # the small window cuts the program differently
    x32, _ = hb.hb_host_sweep_sched(f, b, which, 8, win_slots=512)
    assert 1e-10 < _rel(x32, ref) <= 1e-6


def test_schedule_leaf_lu(hb):
    # the exact leaf-LU variant (other sweep-leaf triangles, same butterflies)
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps, options=hb.HB_OPT_LEAF_LU)
    b = W.complex_gaussian(wl.n, 41)
    for which in range(4):
        x, _ = hb.hb_host_sweep_sched(f, b, which, 16, win_slots=512)
        assert _rel(x, hb.hb_host_sweep(f, b, which)) <= 1e-13


def test_schedule_rejects_bad_arguments(hb, strip_host):
    wl, f = strip_host
    b = np.zeros(wl.n, dtype=np.complex128)
    for which, cb, ws in ((4, 16, 0), (0, 4, 0), (0, 16, -1), (0, 16, 1 << 20)):
        with pytest.raises(hb.HBError):
            hb.hb_host_sweep_sched(f, b, which, cb, win_slots=ws)


def test_schedule_check_names_planted_defects():
    # tests/schedcheck.cpp, built here against the library's host code: the schedules as
    # built pass the structural check; each planted defect (a window slot written twice
    # or written and read within one resident phase, an input outside the window, a
    # misaligned group, a missing ENDRUN, a global row that adds in place) is named
    import os
    import shutil
    import subprocess
    import tempfile
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    csrc = os.path.join(root, "paper_1901_11371_gb300", "csrc")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "schedcheck")
        cmd = [gxx, "-O2", "-std=c++17", "-fopenmp", "-I", csrc, os.path.join(root, "tests", "schedcheck.cpp"),
               os.path.join(csrc, "hb_host.cpp"), os.path.join(csrc, "hb_swsched.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]
