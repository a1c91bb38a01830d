"""GPU checks of the split-BF16 tensor-core form (HB_SPLIT_BF16).

The forward apply of 32 or more columns runs every leaf's entry and exit
contraction on the tensor cores (tcgen05.mma kind::f16, three bf16 parts of
both operands, six products accumulated in FP32 in tensor memory) and the
inner butterfly steps in complex FP32.  Checks (tolerances stated per test):
* against the library's host emulation of the same operands and splitting
  (FP64 accumulation and FP64 inner items there; FP32 in tensor memory, FP32
  butterfly state and FP32 inner items here): measured 3.3e-7 .. 3.4e-7
  relative per column (FP32 rounding of the state between stages), bound
  1e-6 -- a wrong descriptor, layout, table entry or chunk order is O(1), a
  missing part or product ~1e-5, one accumulator for all six products ~2e-6;
* against the oracle's dense A^: 10 eps + 2e-6, as for the complex-FP32 form;
* the FP64 FGMRES + iterative-refinement solve with this form against the
  oracle's dense LU: 1e-5, the same bound as the other forms (the FP64
  residual on the stored factors sets the solution accuracy).
"""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense, efie

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    wl = W.arc(4096, 64, 1e-6, radius=4096 / 20.0 / math.pi)
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    fs = hb.hb_factor(g, wl.leaf, wl.eps, form=hb.HB_SPLIT_BF16)
    fh = hb.hb_factor_host(g, wl.leaf, wl.eps)
    p = efie.Problem.from_workload(wl)
    return torch, hb, wl, g, fs, fh, p


def _rel_cols(y, ref):
    return np.linalg.norm(y - ref, axis=1) / np.linalg.norm(ref, axis=1)


@pytest.mark.parametrize("R", [32, 200, 256, 300])
def test_tc_apply_matches_host_emulation(setup, R):
    torch, hb, wl, g, fs, fh, p = setup
    x = W.complex_gaussian(wl.n, 91, R).T.copy().astype(np.complex64)       # (R, N)
    y = hb.hb_apply(fs, torch.from_numpy(x).cuda()).cpu().numpy().astype(np.complex128)
    cols = [0, 1, R // 2, R - 1]
    ref = np.stack([hb.hb_host_tc_apply(fh, x[c].astype(np.complex128))[0] for c in cols])
    e = _rel_cols(y[cols], ref)
    assert e.max() <= 1e-6, e


def test_tc_apply_vs_dense_and_adjoint(setup):
    torch, hb, wl, g, fs, fh, p = setup
    a = p.dense()
    R = 64
    x = W.complex_gaussian(wl.n, 92, R).T.copy().astype(np.complex64)
    xt = torch.from_numpy(x).cuda()
    y = hb.hb_apply(fs, xt).cpu().numpy().astype(np.complex128)
    ref = (a @ x.T.astype(np.complex128)).T
    assert _rel_cols(y, ref).max() <= 10 * wl.eps + 2e-6
    # the adjoint of this form runs in complex FP32 (10 eps + 2e-6 as for HB_C64)
    yh = hb.hb_apply(fs, xt, hb.HB_OP_H).cpu().numpy().astype(np.complex128)
    refh = (a.conj().T @ x.T.astype(np.complex128)).T
    assert _rel_cols(yh, refh).max() <= 10 * wl.eps + 2e-6


def test_tc_form_solve_vs_dense_lu(setup):
    torch, hb, wl, g, fs, fh, p = setup
    a = p.dense()
    phis = 180.0 * np.arange(40) / 40.0                   # 40 plane waves: the tensor-core path
    b = hb.hb_rhs_plane_wave(fs, phis)
    x, info = hb.hb_gmres(fs, b, rtol=1e-6, restart=30, maxit=600)
    assert info["converged"] == 40 and info["true_rel_res"] <= 1e-6
    xs = x.cpu().numpy()
    cols = [0, 13, 27, 39]
    x_lu = dense.solve(a, p.plane_wave(phis[cols]) * p.scale)
    for j, c in enumerate(cols):
        assert np.linalg.norm(xs[c] - x_lu[:, j]) / np.linalg.norm(x_lu[:, j]) <= 1e-5
