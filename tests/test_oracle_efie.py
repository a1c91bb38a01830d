"""Pins for the oracle's geometry, impedance matrix, dense solves and far field."""
import math

import numpy as np
import pytest

import workloads as W
from oracle import dense, efie, farfield, geometry, hankel


def test_strip_segments_exact():
    c, w = geometry.segments(W.STRIP, (0.0, 0.0, 51.2, 0.0), 1024)
    np.testing.assert_allclose(w, 0.05, rtol=1e-12)
    np.testing.assert_allclose(c[:, 0], 0.05 * (np.arange(1024) + 0.5), atol=1e-12)
    assert np.all(c[:, 1] == 0.0)


def test_arc_chords_closed_form():
    R, n = 100.0, 2000
    c, w = geometry.segments(W.ARC, (R, 0.0, math.pi), n)
    np.testing.assert_allclose(w, 2 * R * math.sin(math.pi / n / 2), rtol=1e-11)
    np.testing.assert_allclose(np.hypot(c[:, 0], c[:, 1]), R * math.cos(math.pi / n / 2), rtol=1e-13)


def test_spiral_equal_arclength_nodes():
    # Node arc lengths checked against an independent quadrature of a sqrt(1+theta^2).
    integrate = pytest.importorskip("scipy.integrate")
    a, th0, th1, n = W.SPIRAL_A_3276_8, 2 * math.pi, 8 * math.pi, 4096
    th = geometry.spiral_nodes(a, th0, th1, n)
    total = integrate.quad(lambda t: a * math.sqrt(1 + t * t), th0, th1, epsabs=0, epsrel=1e-13)[0]
    assert abs(total - 3276.8) < 1e-8
    for i in (1, 777, 2048, 4095):
        s = integrate.quad(lambda t: a * math.sqrt(1 + t * t), th0, th[i], epsabs=0, epsrel=1e-13)[0]
        assert abs(s - total * i / n) < 1e-8
    c, w = geometry.segments(W.SPIRAL, (a, th0, th1), n)
    # chords are slightly shorter than arcs (deficit ~ sum w^3 curvature^2 / 24, here a few 1e-3)
    assert 0 < 3276.8 - w.sum() < 1e-2


def test_parallel_strips_layout():
    c, w = geometry.segments(W.PARALLEL_STRIPS, (8.0, 12.8, 2.0), 2048)
    np.testing.assert_allclose(w, 12.8 / 256, rtol=1e-12)
    np.testing.assert_allclose(c[::256, 1], 2.0 * np.arange(8))
    assert np.all(np.diff(c[:256, 0]) > 0)


def _small_problem(n=256):
    return efie.Problem(W.SPIRAL, (0.35, 2 * math.pi, 6 * math.pi), n)


def test_reciprocity():
    p = _small_problem()
    a = p.dense(scaled=False)
    w = p.lengths
    # Z_ij / w_j = Z_ji / w_i: the off-diagonal kernel depends on |rho_i - rho_j| only.
    lhs = a / w[None, :]
    np.testing.assert_allclose(lhs, lhs.T, rtol=1e-14, atol=0)


def test_diagonal_closed_form_and_scale():
    p = efie.Problem(W.STRIP, (0.0, 0.0, 51.2, 0.0), 1024)
    k, eta, g, d = 2 * math.pi, 376.73, 1.781072, 0.05
    # BASELINE form ln(gamma k d / 4) - 1 equals the paper's ln(gamma k w / (4e)).
    expect = (k * eta * d / 4) * (1 - 1j * (2 / math.pi) * (math.log(g * k * d / 4) - 1))
    np.testing.assert_allclose(p.diagonal(), expect, rtol=1e-12)
    a = p.dense()
    assert abs(np.max(np.abs(np.diag(a))) - 1.0) < 1e-15
    off = p.entries(np.array([3]), np.array([10]))[0, 0]
    expect_off = (k * eta * d / 4) * hankel.hankel2_0(np.array([k * 7 * d]))[0]
    np.testing.assert_allclose(off, expect_off, rtol=1e-14)


def test_self_term_is_segment_average():
    # The diagonal formula is the small-segment limit of (kappa eta/4) int_{-w/2}^{w/2} H0^(2)(kappa|s|) ds.
    integrate = pytest.importorskip("scipy.integrate")
    k, eta, g = 2 * math.pi, 376.73, 1.781072
    for w in (2e-3, 5e-3):
        f_re = lambda s: hankel.hankel2_0(np.array([k * s]))[0].real
        f_im = lambda s: hankel.hankel2_0(np.array([k * s]))[0].imag
        re = 2 * integrate.quad(f_re, 0, w / 2, epsrel=1e-12, limit=200)[0]
        im = 2 * integrate.quad(f_im, 0, w / 2, epsrel=1e-12, limit=200)[0]
        quad = (k * eta / 4) * (re + 1j * im)
        formula = (k * eta * w / 4) * (1 - 1j * (2 / math.pi) * math.log(g * k * w / (4 * math.e)))
        assert abs(quad - formula) / abs(formula) < 1e-4


@pytest.mark.parametrize("n", [16, 64, 200])
def test_lu_solve_bruteforce(n):
    rng = np.random.default_rng(n)
    a = rng.standard_normal((n, n)) + 1j * rng.standard_normal((n, n))
    b = rng.standard_normal(n) + 1j * rng.standard_normal(n)
    x = dense.solve(a, b)
    assert np.linalg.norm(a @ x - b) / np.linalg.norm(b) < 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-10, atol=1e-12)


def test_lu_on_efie_matrix():
    p = _small_problem(256)
    a = p.dense()
    b = p.plane_wave(45.0)[:, 0]
    x = dense.solve(a, b)
    assert np.linalg.norm(a @ x - b) / np.linalg.norm(b) < 1e-12
    np.testing.assert_allclose(x, np.linalg.solve(a, b), rtol=1e-9)


def test_triangles_and_split_operator():
    p = _small_problem(128)
    a = p.dense()
    lt, ut = dense.l_tilde(a), dense.u_tilde(a)
    # Eqs. (Lt), (Ut): L~ + U~ - I = A, unit diagonal of L~, zero upper part.
    np.testing.assert_allclose(lt + ut - np.eye(128), a, atol=0)
    assert np.all(np.diag(lt) == 1) and np.all(np.triu(lt, 1) == 0) and np.all(np.tril(ut, -1) == 0)
    s = dense.split_operator(a)
    np.testing.assert_allclose(lt @ s @ ut, a, rtol=0, atol=1e-10)
    b = p.plane_wave(10.0)[:, 0]
    np.testing.assert_allclose(lt @ (ut @ dense.precond_solve(a, b)), b, atol=1e-11)


def test_precond_spectrum_clusters_near_one():
    # Qualitative claim of Sec. 3.1 on a smooth non-resonant open curve (semicircle,
    # 20 segments per wavelength): L~^{-1} A U~^{-1} has no eigenvalues near 0 and a
    # much smaller condition number than A.
    p = efie.Problem(W.ARC, (25.6 / math.pi, 0.0, math.pi), 512)
    a = p.dense()
    s = dense.split_operator(a)
    ev_s = np.linalg.eigvals(s)
    assert np.min(np.abs(ev_s)) > 0.4
    assert np.linalg.cond(s) < np.linalg.cond(a) / 5


def test_far_field_matches_large_distance_field():
    # Far-field formula vs. the exact scattered field -(k eta/4) sum w x H0^(2) at R = 1e7.
    p = _small_problem(256)
    x = W.complex_gaussian(256, 5)
    phi = np.array([0.0, 33.0, 190.0])
    ff = farfield.far_field(p, x, phi)
    R = 1e7
    for i, ph in enumerate(phi * math.pi / 180):
        obs = np.array([R * math.cos(ph), R * math.sin(ph)])
        dist = np.hypot(obs[0] - p.centres[:, 0], obs[1] - p.centres[:, 1])
        es = -(p.kappa * p.eta0 / 4) * np.sum(p.lengths * x * hankel.hankel2_0(p.kappa * dist))
        norm = es * math.sqrt(R) * np.exp(1j * p.kappa * R)
        assert abs(norm - ff[i]) / abs(ff[i]) < 1e-4


def test_monostatic_is_backscatter():
    p = _small_problem(128)
    x = W.complex_gaussian(128, 6, 3)
    phi = np.array([10.0, 50.0, 170.0])
    mono = farfield.monostatic(p, x, phi)
    for i in range(3):
        np.testing.assert_allclose(mono[i], farfield.far_field(p, x[:, i], [phi[i] + 180.0])[0], rtol=1e-12)
