"""Oracle: zeroth-order Hankel function of the second kind, H0^(2)(x) = J0(x) - i Y0(x).

TEST INFRASTRUCTURE ONLY.  The product path never imports this package.

The EFIE kernel of Sec. 3.1 needs H0^(2) at real x > 0.  This module computes it
from textbook definitions, independently of any library Bessel routine:

* small x (pins only): ascending power series, Abramowitz & Stegun 9.1.10
  (J0, J1) and 9.1.11 / 9.1.13 (Y0, Y1);
* 0 < x < X_ASYM: Miller's backward recurrence for J_n normalised by
  J0 + 2 sum_k J_2k = 1 (A&S 9.1.46), and Neumann's series for Y0
  (A&S 9.1.88): (pi/2) Y0 = (ln(x/2) + gamma_E) J0 - 2 sum_k (-1)^k J_2k / k;
* x >= X_ASYM: Hankel's asymptotic expansion (DLMF 10.17.3):
  H0^(2)(x) ~ sqrt(2/(pi x)) e^{-i(x - pi/4)} (P(x) - i Q(x)).

Everything is fp64 and vectorised over numpy arrays.
"""
from __future__ import annotations

import math

import numpy as np

EULER_GAMMA = 0.57721566490153286060651209
X_ASYM = 25.0


# ----------------------------------------------------------------------------
# Ascending series (A&S 9.1.10, 9.1.11, 9.1.13).  Used by the pins for x <= 2.
# ----------------------------------------------------------------------------

def series_j0_y0_j1_y1(x):
    x = np.asarray(x, dtype=np.float64)
    t = x * x / 4.0
    j0 = np.zeros_like(x)
    j1 = np.zeros_like(x)
    s0 = np.zeros_like(x)   # sum_{k>=1} (-1)^{k+1} H_k t^k / (k!)^2
    s1 = np.zeros_like(x)   # sum_k {psi(k+1)+psi(k+2)} (-t)^k / (k!(k+1)!)
    term0 = np.ones_like(x)            # (-t)^k / (k!)^2
    term1 = np.ones_like(x)            # (-t)^k / (k!(k+1)!)
    harmonic = 0.0
    for k in range(0, 60):
        if k > 0:
            term0 = term0 * (-t) / (k * k)
            term1 = term1 * (-t) / (k * (k + 1))
            harmonic += 1.0 / k
        j0 = j0 + term0
        j1 = j1 + term1
        if k > 0:
            s0 = s0 - harmonic * term0          # (-1)^{k+1} H_k t^k/(k!)^2 = -H_k * term0
        psi_k1 = -EULER_GAMMA + harmonic                 # psi(k+1)
        psi_k2 = -EULER_GAMMA + harmonic + 1.0 / (k + 1)  # psi(k+2)
        s1 = s1 + (psi_k1 + psi_k2) * term1
    j1 = j1 * (x / 2.0)
    y0 = (2.0 / math.pi) * (np.log(x / 2.0) + EULER_GAMMA) * j0 + (2.0 / math.pi) * s0
    y1 = -2.0 / (math.pi * x) + (2.0 / math.pi) * np.log(x / 2.0) * j1 - (x / (2.0 * math.pi)) * s1
    return j0, y0, j1, y1


# ----------------------------------------------------------------------------
# Miller backward recurrence + Neumann series, 0 < x < X_ASYM.
# ----------------------------------------------------------------------------

def miller_j0_y0(x):
    """J0 and Y0 for 0 < x < ~30 by Miller's algorithm and Neumann's series."""
    x = np.asarray(x, dtype=np.float64)
    xmax = float(np.max(x)) if x.size else 1.0
    nstart = int(2 * ((int(xmax) + 40) // 2))           # even start index, well above x
    jp1 = np.zeros_like(x)                              # J_{n+1}
    jn = np.full_like(x, 1e-30)                         # J_n (unnormalised)
    norm = np.zeros_like(x)                             # J0 + 2 sum_k J_2k
    neumann = np.zeros_like(x)                          # sum_k (-1)^k J_2k / k
    j0 = None
    n = nstart
    while n > 0:
        if n % 2 == 0:
            k = n // 2
            norm += 2.0 * jn
            neumann += ((-1.0) ** k) * jn / k
        jm1 = (2.0 * n / x) * jn - jp1
        jp1, jn = jn, jm1
        n -= 1
        # rescale to avoid overflow in the upward-growing recurrence
        big = np.abs(jn) > 1e250
        if np.any(big):
            scale = np.where(big, 1e-250, 1.0)
            jn, jp1, norm, neumann = jn * scale, jp1 * scale, norm * scale, neumann * scale
    j0_unnorm = jn
    norm = norm + j0_unnorm
    j0 = j0_unnorm / norm
    neumann = neumann / norm
    y0 = (2.0 / math.pi) * ((np.log(x / 2.0) + EULER_GAMMA) * j0 - 2.0 * neumann)
    return j0, y0


# ----------------------------------------------------------------------------
# Hankel asymptotic expansion (DLMF 10.17.1-10.17.3), x >= X_ASYM.
# ----------------------------------------------------------------------------

def _ak0(kmax):
    """a_k(0) = (-1)^k (1^2 3^2 ... (2k-1)^2) / (k! 8^k)  (DLMF 10.17.1 at nu = 0)."""
    a = [1.0]
    for k in range(1, kmax + 1):
        a.append(a[-1] * (-(2 * k - 1) ** 2) / (k * 8.0))
    return a


_AK = _ak0(60)


def asym_p_q(x):
    """P(x) = sum_k (-1)^k a_2k / x^2k,  Q(x) = sum_k (-1)^k a_{2k+1} / x^{2k+1}."""
    x = np.asarray(x, dtype=np.float64)
    p = np.zeros_like(x)
    q = np.zeros_like(x)
    for k in range(0, 30):
        tp = ((-1.0) ** k) * _AK[2 * k] / x ** (2 * k)
        tq = ((-1.0) ** k) * _AK[2 * k + 1] / x ** (2 * k + 1)
        p += tp
        q += tq
        if np.all(np.abs(tq) < 1e-18 * np.abs(p)):
            break
    return p, q


def asym_j0_y0(x):
    x = np.asarray(x, dtype=np.float64)
    p, q = asym_p_q(x)
    w = x - math.pi / 4.0
    amp = np.sqrt(2.0 / (math.pi * x))
    j0 = amp * (p * np.cos(w) - q * np.sin(w))
    y0 = amp * (p * np.sin(w) + q * np.cos(w))
    return j0, y0


def j0_y0(x):
    """J0(x), Y0(x) for x > 0 (Miller + Neumann below X_ASYM, asymptotic above)."""
    x = np.asarray(x, dtype=np.float64)
    j0 = np.empty_like(x)
    y0 = np.empty_like(x)
    lo = x < X_ASYM
    if np.any(lo):
        j0[lo], y0[lo] = miller_j0_y0(x[lo])
    if np.any(~lo):
        j0[~lo], y0[~lo] = asym_j0_y0(x[~lo])
    return j0, y0


def hankel2_0(x):
    """H0^(2)(x) = J0(x) - i Y0(x) for real x > 0."""
    j0, y0 = j0_y0(x)
    return j0 - 1j * y0
