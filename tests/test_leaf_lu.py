"""Exact-leaf-LU variant of the preconditioner (HB_OPT_LEAF_LU): the leaf blocks of L~
and U~ are the LU factors of the dense leaf block instead of its entry-wise triangles.

Oracle pins: the LU factors rebuild the block and equal scipy's LU where no row exchange
happens; the library's host sweeps with the option equal dense triangular solves with
the oracle's variant triangles of the densified compressed operator (1e-12), as the
default sweeps do with the entry-wise triangles."""
import numpy as np
import pytest

import workloads as W
from oracle import dense


@pytest.fixture(scope="module")
def hb():
    from paper_1901_11371_gb300 import build
    build.build()
    import paper_1901_11371_gb300 as hb
    hb.lib()
    return hb


def test_oracle_leaf_lu_rebuilds_the_block():
    rng = np.random.default_rng(11)
    blk = rng.standard_normal((40, 40)) + 1j * rng.standard_normal((40, 40)) + 60 * np.eye(40)
    lo, up = dense.leaf_lu(blk)
    assert np.allclose(np.triu(lo, 1), 0) and np.allclose(np.diag(lo), 1) and np.allclose(np.tril(up, -1), 0)
    assert np.linalg.norm(lo @ up - blk) / np.linalg.norm(blk) < 1e-14
    linalg = pytest.importorskip("scipy.linalg")
    p, l2, u2 = linalg.lu(blk)
    assert np.array_equal(p, np.eye(40))                # diagonally dominant: no row exchange
    assert np.linalg.norm(l2 - lo) < 1e-12 and np.linalg.norm(u2 - up) / np.linalg.norm(up) < 1e-13


def test_oracle_variant_triangles_keep_the_off_diagonal_split():
    rng = np.random.default_rng(12)
    a = rng.standard_normal((64, 64)) + 1j * rng.standard_normal((64, 64)) + 40 * np.eye(64)
    lt, ut = dense.l_tilde_leaf_lu(a, 16), dense.u_tilde_leaf_lu(a, 16)
    for s in range(0, 64, 16):
        blk = slice(s, s + 16)
        assert np.linalg.norm(lt[blk, blk] @ ut[blk, blk] - a[blk, blk]) < 1e-12 * np.linalg.norm(a[blk, blk])
    mask = np.kron(np.eye(4), np.ones((16, 16))) == 0     # outside the diagonal blocks
    np.testing.assert_array_equal(lt[mask], dense.l_tilde(a)[mask])
    np.testing.assert_array_equal(ut[mask], dense.u_tilde(a)[mask])


def test_host_sweeps_with_leaf_lu_are_variant_triangular_solves(hb):
    wl = W.STRIP_N1024
    g = hb.hb_geometry(wl.kind, wl.params, wl.n)
    f = hb.hb_factor_host(g, wl.leaf, wl.eps, options=hb.HB_OPT_LEAF_LU)
    af = np.stack([hb.hb_host_apply(f, e) for e in np.eye(wl.n, dtype=np.complex128)], axis=1)
    lt, ut = dense.l_tilde_leaf_lu(af, wl.leaf), dense.u_tilde_leaf_lu(af, wl.leaf)
    b = W.complex_gaussian(wl.n, 13)
    refs = {0: dense.forward_subst(lt, b, unit=True),
            1: dense.back_subst(ut, b),
            2: dense.back_subst(lt.conj().T, b, unit=True),
            3: dense.forward_subst(ut.conj().T, b)}
    for which, ref in refs.items():
        v = hb.hb_host_sweep(f, b, which)
        assert np.linalg.norm(v - ref) / np.linalg.norm(ref) < 1e-12, which
    # the default factor's sweeps differ (the leaf triangles differ)
    f0 = hb.hb_factor_host(g, wl.leaf, wl.eps)
    assert np.linalg.norm(hb.hb_host_sweep(f0, b, 0) - refs[0]) > 1e-6 * np.linalg.norm(refs[0])


def test_unknown_option_bits_are_rejected(hb):
    g = hb.hb_geometry(hb.HB_STRIP, (0.0, 0.0, 3.2, 0.0), 64)
    with pytest.raises(hb.HBError):
        hb.hb_factor_host(g, 32, 1e-6, options=4)   # bits 1 and 2 are HB_OPT_LEAF_LU and HB_OPT_SWEEP_WINDOW_MIN
