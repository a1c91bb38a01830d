"""Host logic of the sweep programs (no GPU): flattening, staging offsets, the
segmentation into grid-wide phases and single-CTA runs (coverage, thresholds,
residency budgets, butterfly state produced and consumed inside resident runs), and
the flattened records executed the way the sweep kernel reads them against the host
interpreter (strip, arc, leaf-LU and polyline factors).  The checks live in
tests/segcheck.cpp, built here against the library's host code."""
import os
import shutil
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1901_11371_gb300", "csrc")


def test_sweep_program_segmentation_invariants():
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "segcheck")
        cmd = [gxx, "-O2", "-std=c++17", "-fopenmp", "-I", CSRC, os.path.join(ROOT, "tests", "segcheck.cpp"),
               os.path.join(CSRC, "hb_host.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]


def test_tree_sampling_equals_full_scan():
    # the k-d tree path of the ID sampling picks exactly the full scan's samples
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("g++ not available")
    with tempfile.TemporaryDirectory() as d:
        exe = os.path.join(d, "samplecheck")
        cmd = [gxx, "-O2", "-std=c++17", "-fopenmp", "-I", CSRC, os.path.join(ROOT, "tests", "samplecheck.cpp"), "-o", exe]
        r = subprocess.run(cmd, capture_output=True, text=True)
        assert r.returncode == 0, r.stderr[-2000:]
        r = subprocess.run([exe], capture_output=True, text=True, timeout=600)
        assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout[-3000:]
