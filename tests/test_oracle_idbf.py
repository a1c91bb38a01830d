"""Pins for the oracle's IDs, butterflies, H-IDBF apply/sweeps, GMRES and TFQMR (Secs. 2-4, Appendix)."""
import math
import os

import numpy as np
import pytest

import workloads as W
from oracle import dense, efie, idbf, krylov


# ---------------------------------------------------------------- IDs

def test_column_id_exact_on_low_rank():
    rng = np.random.default_rng(0)
    r = 7
    m = (rng.standard_normal((60, r)) + 1j * rng.standard_normal((60, r))) @ \
        (rng.standard_normal((r, 40)) + 1j * rng.standard_normal((r, 40)))
    q, p, t = idbf.column_id(m, 1e-10)
    assert len(q) == r and len(q) + len(p) == 40
    np.testing.assert_allclose(m[:, q] @ t, m[:, p], atol=1e-10 * np.abs(m).max())
    # row ID: m[p,:] ~ e m[q,:]
    q, p, e = idbf.row_id(m, 1e-10)
    assert len(q) == r
    np.testing.assert_allclose(e @ m[q, :], m[p, :], atol=1e-10 * np.abs(m).max())


def test_pivoted_qr_matches_library():
    sl = pytest.importorskip("scipy.linalg")
    rng = np.random.default_rng(1)
    m = rng.standard_normal((30, 20)) + 1j * rng.standard_normal((30, 20))
    perm, r = idbf.pivoted_qr(m)
    q, r2, p2 = sl.qr(m, pivoting=True, mode="economic")
    np.testing.assert_allclose(np.abs(np.diag(r)), np.abs(np.diag(r2)), rtol=1e-12)
    # reconstruct m[:, perm] = Q r with Q orthonormal
    qq, _ = np.linalg.qr(m[:, perm])
    np.testing.assert_allclose(np.abs(np.diag(r)), np.abs(np.diag(np.linalg.qr(m[:, perm])[1])), rtol=1e-12)


def test_column_id_error_tracks_tolerance():
    p = efie.Problem(W.STRIP, (0, 0, 25.6, 0), 512)
    blk = p.scaled_entries(np.arange(0, 256), np.arange(256, 320))
    for tol in (1e-4, 1e-6, 1e-8):
        q, pp, t = idbf.column_id(blk, tol)
        err = np.linalg.norm(blk[:, q] @ t - blk[:, pp]) / np.linalg.norm(blk)
        assert err < 10 * tol


# ---------------------------------------------------------------- butterflies

def _strip(n):
    return efie.Problem(W.STRIP, (0.0, 0.0, n / 20.0, 0.0), n)


@pytest.mark.parametrize("n,n0", [(256, 32), (512, 32), (512, 64), (1024, 32)])
def test_butterfly_block_error(n, n0):
    p = _strip(2 * n)
    blk = p.scaled_entries(np.arange(n, 2 * n), np.arange(0, n))     # an F21 block
    eps = 1e-6
    bf = idbf.Butterfly(blk, n0, eps)
    assert bf.hc + bf.hr == bf.levels + 2
    err = np.linalg.norm(bf.dense() - blk) / np.linalg.norm(blk)
    assert err <= 3 * eps, err                       # plain ID tolerance eps: O(eps) block error
    bf = idbf.butterfly_within_tolerance(blk, n0, eps)
    err = np.linalg.norm(bf.dense() - blk) / np.linalg.norm(blk)
    assert err <= eps, err
    x = W.complex_gaussian(n, 9, 2)
    np.testing.assert_allclose(bf.apply(x), bf.dense() @ x, rtol=1e-12, atol=1e-14)


def test_butterfly_adjoint_identity():
    p = _strip(1024)
    blk = p.scaled_entries(np.arange(0, 512), np.arange(512, 1024))
    bf = idbf.Butterfly(blk, 32, 1e-6)
    x = W.complex_gaussian(512, 10)
    y = W.complex_gaussian(512, 11)
    lhs = np.vdot(y, bf.apply(x))
    rhs = np.vdot(bf.apply_adjoint(y), x)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    np.testing.assert_allclose(bf.apply_adjoint(np.eye(512)), bf.dense().conj().T, atol=1e-13)


def test_butterfly_odd_and_zero_levels():
    p = _strip(256)
    for n in (32, 64):   # L = 0 and L = 1 with n0 = 32
        blk = p.scaled_entries(np.arange(n, 2 * n), np.arange(0, n))
        bf = idbf.Butterfly(blk, 32, 1e-8)
        assert bf.levels == int(math.log2(n // 32))
        assert np.linalg.norm(bf.dense() - blk) / np.linalg.norm(blk) < 1e-8


def test_ranks_flat_in_n():
    # Sec. 4: the maximum butterfly rank is almost independent of N at fixed sampling.
    ranks = []
    for n in (512, 1024, 2048):
        p = _strip(2 * n)
        blk = p.scaled_entries(np.arange(n, 2 * n), np.arange(0, n))
        ranks.append(idbf.Butterfly(blk, 32, 1e-6).max_rank())
    assert max(ranks) - min(ranks) <= 3, ranks
    assert max(ranks) < 32


# ---------------------------------------------------------------- H-IDBF

@pytest.fixture(scope="module")
def strip1024():
    p = efie.Problem.from_workload(W.STRIP_N1024)
    a = p.dense()
    h = idbf.HIDBF(a, 32, 1e-6)
    return p, a, h


def test_hidbf_apply_within_10eps(strip1024):
    p, a, h = strip1024
    x = W.complex_gaussian(1024, 12)
    assert np.linalg.norm(h.apply(x) - a @ x) / np.linalg.norm(a @ x) <= 10 * 1e-6
    y = W.complex_gaussian(1024, 13)
    ah = a.conj().T
    assert np.linalg.norm(h.apply(y, adjoint=True) - ah @ y) / np.linalg.norm(ah @ y) <= 10 * 1e-6


def test_hidbf_structure_counts(strip1024):
    p, a, h = strip1024
    bfs = h.butterflies()
    assert len(bfs) == 2 * (1024 // 32 - 1)     # two off-diagonal blocks per internal node
    levels = sorted({bf.levels for bf in bfs})
    assert levels == [0, 1, 2, 3, 4]


def test_sweeps_equal_dense_triangular_solves(strip1024):
    p, a, h = strip1024
    af = h.dense()                                 # the compressed operator A_F, densified
    b = W.complex_gaussian(1024, 14)
    xl = h.solve_lower(b)
    np.testing.assert_allclose(xl, dense.forward_subst(dense.l_tilde(af), b, unit=True), rtol=1e-11, atol=1e-12)
    xu = h.solve_upper(b)
    np.testing.assert_allclose(xu, dense.back_subst(dense.u_tilde(af), b), rtol=1e-11, atol=1e-12)
    # adjoint sweeps against dense conjugate-transposed triangles
    xlh = h.solve_lower_adjoint(b)
    np.testing.assert_allclose(xlh, dense.back_subst(dense.l_tilde(af).conj().T, b, unit=True), rtol=1e-11, atol=1e-12)
    xuh = h.solve_upper_adjoint(b)
    np.testing.assert_allclose(xuh, dense.forward_subst(dense.u_tilde(af).conj().T, b), rtol=1e-11, atol=1e-12)
    # and close to the exact entry-wise triangles of the uncompressed A
    x_exact = dense.precond_solve(a, b)
    assert np.linalg.norm(h.precond(b) - x_exact) / np.linalg.norm(x_exact) < 1e-4


def test_memory_scaling_n_log2_n():
    # Secs. 1 and 4: memory grows as O(N log^2 N).
    ratios = []
    for n in (512, 1024, 2048, 4096):
        a = _strip(n).dense()
        h = idbf.HIDBF(a, 32, 1e-6)
        ratios.append(h.nnz() / (n * math.log2(n) ** 2))
    assert max(ratios) / min(ratios) < 2.0, ratios
    # and far below dense N^2 at the largest size
    assert h.nnz() < 0.5 * 4096 ** 2


def test_gmres_matches_dense_lu(strip1024):
    p, a, h = strip1024
    b = p.plane_wave(30.0)[:, 0] * p.scale
    x_lu = dense.solve(a, b)
    x, info = krylov.gmres_split(h.apply, h.solve_lower, h.solve_upper, b, rtol=1e-6, restart=30)
    assert info["true_rel_res"] <= 1e-6
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-5
    assert info["iters"] < 60


def test_gmres_paper_protocol_b_equals_a_xt():
    # Sec. 4: b = A x^t for random x^t; the solution error is small.
    p = efie.Problem(W.SPIRAL, (0.35, 2 * math.pi, 8 * math.pi), 512)
    a = p.dense()
    h = idbf.HIDBF(a, 32, 1e-6)
    xt = W.complex_gaussian(512, W.SEED_XTRUE)
    b = a @ xt
    x, info = krylov.gmres_split(h.apply, h.solve_lower, h.solve_upper, b, rtol=1e-8)
    assert np.linalg.norm(x - xt) / np.linalg.norm(xt) < 1e-3


def test_tfqmr_dense_system_matches_solve():
    # Unpreconditioned TFQMR on a small well-conditioned nonsymmetric complex system reaches
    # the direct solution; a wrong coefficient in the half-step recurrences stalls it.
    n = 60
    a = np.eye(n) * 4.0 + W.complex_gaussian(n * n, 21).reshape(n, n) * 0.4
    b = W.complex_gaussian(n, 22)
    ident = lambda v: v
    x, info = krylov.tfqmr_split(lambda z: a @ z, ident, ident, b,
                                 rstar=W.complex_gaussian(n, W.SEED_SHADOW), rtol=1e-10, maxit=400)
    x_ref = np.linalg.solve(a, b)
    assert info["true_rel_res"] <= 1e-10
    assert np.linalg.norm(x - x_ref) / np.linalg.norm(x_ref) <= 1e-9
    # one product per half step (plus the start, less one when it stops after an even step)
    assert info["iters"] <= info["matvecs"] <= info["iters"] + 1


def test_tfqmr_split_preconditioned_strip(strip1024):
    # Sec. 4's solver on the split system: same solution as the dense LU, in about as many
    # products with L~^{-1} A U~^{-1} as GMRES takes iterations.
    p, a, h = strip1024
    b = p.plane_wave(30.0)[:, 0] * p.scale
    x_lu = dense.solve(a, b)
    x, info = krylov.tfqmr_split(h.apply, h.solve_lower, h.solve_upper, b,
                                 rstar=W.complex_gaussian(a.shape[0], W.SEED_SHADOW), rtol=1e-6)
    assert info["true_rel_res"] <= 1e-6
    assert np.linalg.norm(x - x_lu) / np.linalg.norm(x_lu) <= 1e-5
    assert info["matvecs"] < 80


def _paper_errors(golden_dir):
    vals = {}
    with open(os.path.join(golden_dir, "paper_solution_error_n5e3.txt")) as f:
        for line in f:
            parts = line.split("#")[0].split()
            if parts:
                vals[parts[0]] = float(parts[1])
    return vals


@pytest.mark.parametrize("shape", ["semicircle", "spiral"])
def test_solution_error_has_the_papers_order(golden_dir, shape):
    # Sec. 4's accuracy protocol on the oracle: random x^t, b = F x^t with the compressed F
    # (eps = 1e-4), TFQMR to 1e-5 on the split system.  The solution error lands within a
    # factor 5 of the paper's N = 5E3 value (here N = 2048, leaf 128; the spiral makes one
    # turn from theta = 2 pi; the paper states neither size).  A wrong sign or term in the
    # apply or the sweeps would leave it far larger.
    n = 2048
    if shape == "semicircle":
        params, kind = (n / 20 / math.pi, 0.0, math.pi), W.ARC
    else:
        s = lambda t: 0.5 * (t * math.sqrt(1 + t * t) + math.asinh(t))
        t0, t1 = 2 * math.pi, 4 * math.pi
        params, kind = ((n / 20.0) / (s(t1) - s(t0)), t0, t1), W.SPIRAL
    a = efie.Problem(kind, params, n).dense()
    h = idbf.HIDBF(a, 128, 1e-4)
    xt = W.complex_gaussian(n, W.SEED_XTRUE)
    x, info = krylov.tfqmr_split(h.apply, h.solve_lower, h.solve_upper, h.apply(xt),
                                 rstar=W.complex_gaussian(n, W.SEED_SHADOW), rtol=1e-5)
    err = np.linalg.norm(x - xt) / np.linalg.norm(xt)
    paper = _paper_errors(golden_dir)[shape]
    assert paper / 5 <= err <= 5 * paper, (err, paper)
    assert info["matvecs"] < 60
