"""Pins for the oracle's own H0^(2) (Sec. 3.1 kernel) against textbook facts."""
import math
import os

import numpy as np
import pytest

from oracle import hankel


def _table(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "bessel_table.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            name, x, v = line.split()
            rows.append((name, float(x), float(v)))
    return rows


def test_tabulated_values(golden_dir):
    # A&S Table 9.1 / 9.5 values, through every evaluation route of the oracle.
    for name, x, v in _table(golden_dir):
        xs = np.array([x])
        j0, y0 = hankel.j0_y0(xs)
        got = {"J0": j0[0], "Y0": y0[0]}
        if x <= 2.5:
            sj0, sy0, sj1, sy1 = hankel.series_j0_y0_j1_y1(xs)
            got_series = {"J0": sj0[0], "Y0": sy0[0], "J1": sj1[0], "Y1": sy1[0]}
            assert abs(got_series[name] - v) <= 2e-15 + 1e-15 * abs(v), (name, x)
        if name in got:
            assert abs(got[name] - v) <= 2e-15 + 2e-15 * abs(v), (name, x, got[name], v)


def test_series_wronskian():
    # A&S 9.1.16: J1(x) Y0(x) - J0(x) Y1(x) = 2 / (pi x); all four from the ascending series.
    x = np.linspace(0.02, 2.0, 100)
    j0, y0, j1, y1 = hankel.series_j0_y0_j1_y1(x)
    w = j1 * y0 - j0 * y1
    np.testing.assert_allclose(w, 2.0 / (math.pi * x), rtol=1e-13)


def test_miller_matches_series_small_x():
    # Two independent routes (ascending series vs. backward recurrence + Neumann series).
    x = np.linspace(0.01, 2.0, 200)
    sj0, sy0, _, _ = hankel.series_j0_y0_j1_y1(x)
    mj0, my0 = hankel.miller_j0_y0(x)
    np.testing.assert_allclose(mj0, sj0, atol=2e-15, rtol=1e-14)
    np.testing.assert_allclose(my0, sy0, atol=2e-15, rtol=1e-14)


def test_asymptotic_matches_miller_in_overlap():
    x = np.linspace(22.0, 30.0, 200)
    mj0, my0 = hankel.miller_j0_y0(x)
    aj0, ay0 = hankel.asym_j0_y0(x)
    np.testing.assert_allclose(aj0, mj0, atol=3e-15)
    np.testing.assert_allclose(ay0, my0, atol=3e-15)


def test_large_x_modulus():
    # |H0^(2)(x)|^2 = (2/(pi x)) (P^2 + Q^2) has the non-oscillatory expansion
    # (2/(pi x)) (1 - 1/(8 x^2) + 27/(128 x^4) - ...)  (DLMF 10.18.17 at nu = 0).
    x = np.logspace(np.log10(50.0), np.log10(3e5), 50)
    h = hankel.hankel2_0(x)
    expect = (2.0 / (math.pi * x)) * (1.0 - 1.0 / (8.0 * x ** 2) + 27.0 / (128.0 * x ** 4))
    np.testing.assert_allclose(np.abs(h) ** 2, expect, rtol=1e-9)


def test_library_cross_check():
    # Independent library implementation (test only); large-x phase differs by ~ulp(x).
    sp = pytest.importorskip("scipy.special")
    x = np.logspace(-6, np.log10(3e5), 3000)
    h = hankel.hankel2_0(x)
    ref = sp.hankel2(0, x)
    tol = 1e-12 * np.abs(ref) + 4e-16 * x * np.abs(ref) + 1e-15
    assert np.all(np.abs(h - ref) <= tol)


def test_h2_is_j_minus_i_y():
    x = np.array([0.5, 3.0, 40.0])
    j0, y0 = hankel.j0_y0(x)
    h = hankel.hankel2_0(x)
    np.testing.assert_array_equal(h.real, j0)
    np.testing.assert_array_equal(h.imag, -y0)
