"""CPU checks of the persistent single-column apply's schedule.

The kernel (one cooperative launch per apply, Alg. 2 as phases) runs a plan
built on the host: per CTA, staging batches of task and op records, factor
blocks and vector gather lists.  hb_host_apply_plan builds that plan, checks
its structure (areas, offsets, alignment, gather-list ranges) and executes it
on the host in FP64 exactly as the kernel stages it: per phase, per CTA, per
batch, every record, block and gather list read from the batch images the
kernel copies, vectors read through the gather lists, the chained dense-leaf
and exit chunks in their phases.  It must equal the packed program's own host
execution (hb_host_apply) to rounding (1e-13 relative with complex128
images, 2e-6 with complex64 ones), for both directions,
several grid sizes (one CTA, a ragged 7, the GB300's 152) and both factor
element sizes (the 8-byte entries give other chunkings); a wrong offset,
list entry or phase order breaks the equality by O(1).
"""
import math

import numpy as np
import pytest

import workloads as W


@pytest.fixture(scope="module")
def hb():
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    hb.lib()
    return hb


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


CASES = [
    W.strip(1024, 32, 1e-6),
    W.arc(4096, 64, 1e-6, radius=4096 / 20.0 / math.pi),
    W.spiral(2048, 64, 1e-6, a=W.SPIRAL_A_3276_8 / 32.0),
    W.parallel_strips(2048, 64, 1e-6, n_strips=2),
    W.strip(2048, 128, 1e-6),
]


@pytest.mark.parametrize("wl", CASES, ids=[w.name + f"_leaf{w.leaf}" for w in CASES])
def test_plan_execution_equals_host_apply(hb, wl):
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps)
    x = W.complex_gaussian(wl.n, 81)
    for op in (hb.HB_OP_N, hb.HB_OP_H):
        ref = hb.hb_host_apply(f, x, op)
        for grid in (1, 7, 152):
            for fb in (8, 16):
                y, nb = hb.hb_host_apply_plan(f, x, op, grid, fb)
                assert nb >= 1
                assert np.all(np.isfinite(y)), (op, grid, fb)
                # 16-byte entries: the images hold the FP64 factors; 8-byte entries: complex64
                # factors (rounding 2^-24 per entry)
                tol = 1e-13 if fb == 16 else 2e-6
                assert _rel(y, ref) <= tol, (op, grid, fb, _rel(y, ref))


def test_plan_rejects_bad_arguments(hb):
    wl = W.strip(256, 32, 1e-6)
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps)
    x = W.complex_gaussian(wl.n, 82)
    with pytest.raises(hb.HBError):
        hb.hb_host_apply_plan(f, x, 0, 0, 8)
    with pytest.raises(hb.HBError):
        hb.hb_host_apply_plan(f, x, 0, 4, 12)
