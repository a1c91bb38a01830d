"""CPU checks of the split-BF16 tensor-core operands (form HB_SPLIT_BF16).

The entry and exit contractions of every leaf are expanded on the host into
real-form chunks of three bf16 parts in the tensor cores' K-major layout,
with input / output tables.  hb_host_tc_apply emulates the device's forward
apply from exactly those operands (the same three-part bf16 splitting of the
vector operand and the same six partial products; FP64 accumulation) with the
inner butterfly items in FP64.  Three bf16 parts carry the FP32 value's 24
significant bits and the dropped products are below 2^-24, so against the
packed program's FP64 apply the difference is the FP32 rounding of the
operands: measured 4.6e-8 .. 4.9e-8, bound 2e-7; any misplaced entry, table
or chunk gives O(1) errors, and a missing part or product about 1e-5.
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
    assert 1e-9 < err <= 2e-7, err          # (> 1e-9: the operands really went through FP32 / bf16)


def test_bf16_split_keeps_fp32_accuracy(hb):
    # the splitting itself on a single column of the operator
    g = hb.hb_geometry(W.STRIP, (0.0, 0.0, 12.8, 0.0), 256)
    f = hb.hb_factor_host(g, 32, 1e-6)
    x = np.zeros(256, dtype=np.complex128)
    x[5] = 1.0 + 1e-3j
    ref = hb.hb_host_apply(f, x)
    y, _ = hb.hb_host_tc_apply(f, x)
    assert np.linalg.norm(y - ref) / np.linalg.norm(ref) <= 2e-7
