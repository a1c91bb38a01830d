"""CPU checks of the split-BF16 tensor-core operands (form HB_SPLIT_BF16).

The entry and exit contractions of every leaf are expanded on the host into
real-form chunks of bf16 hi/lo parts in the tensor cores' K-major layout,
with input / output tables.  hb_host_tc_apply emulates the device's forward
apply from exactly those operands (the same bf16 splitting of the vector
operand and the same three partial products hi*hi + hi*lo + lo*hi; FP64
accumulation) with the inner butterfly items in FP64.  Against the packed
program's FP64 apply the difference is the splitting error: each operand is
kept to about 2^-17 relative (hi + lo) and the dropped lo*lo product is of the
same order, so the apply agrees to about 5e-6 (measured 4.9e-6 .. 5.9e-6);
the bound 1e-5 fails on any misplaced entry, table or chunk (O(1) errors).
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


CASES = [
    W.strip(1024, 32, 1e-6),
    W.arc(4096, 64, 1e-6, radius=4096 / 20.0 / math.pi),
    W.strip(2048, 128, 1e-6),
    W.spiral(2048, 64, 1e-6, a=W.SPIRAL_A_3276_8 / 32.0),
]


@pytest.mark.parametrize("wl", CASES, ids=[w.name + f"_leaf{w.leaf}" for w in CASES])
def test_tc_emulation_matches_packed_apply(hb, wl):
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps)
    x = W.complex_gaussian(wl.n, 90)
    ref = hb.hb_host_apply(f, x)
    y, nchunks = hb.hb_host_tc_apply(f, x)
    assert nchunks >= 2 * (wl.n // wl.leaf)
    err = np.linalg.norm(y - ref) / np.linalg.norm(ref)
    assert 1e-7 < err <= 1e-5, err          # (> 1e-7: the bf16 splitting is really in effect)


def test_bf16_split_keeps_sixteen_bits(hb):
    # the splitting itself: x = hi + lo with |x - hi - lo| <= 2^-17 |x| for normal floats
    g = hb.hb_geometry(W.STRIP, (0.0, 0.0, 12.8, 0.0), 256)
    f = hb.hb_factor_host(g, 32, 1e-6)
    x = np.zeros(256, dtype=np.complex128)
    x[5] = 1.0 + 1e-3j
    ref = hb.hb_host_apply(f, x)
    y, _ = hb.hb_host_tc_apply(f, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 2e-5
