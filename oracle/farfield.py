"""Oracle: 2D TM far field of the induced current (no counterpart in the paper).

TEST INFRASTRUCTURE ONLY.

The scattered field E^s(rho) = -(kappa eta0 / 4) int J(rho') H0^(2)(kappa|rho - rho'|) ds'
(the sign convention of the EFIE in Sec. 3.1) has, with the large-argument form
H0^(2)(z) ~ sqrt(2j/(pi z)) e^{-jz} and |rho - rho'| ~ rho - r^ . rho', the far zone
    E_far(phi) = C sum_n w_n x_n exp(+j kappa (x_n cos phi + y_n sin phi)),
    C = -(kappa eta0 / 4) sqrt(2j / (pi kappa))
(the common factor e^{-j kappa rho}/sqrt(rho) is dropped).  The monostatic
value at incidence phi_i is the backscatter at phi_i + pi:  C sum_n w_n b_n x_n.
"""
from __future__ import annotations

import math

import numpy as np


def far_field(problem, x, phi_obs_deg):
    """Bistatic far field for the current(s) x ([N] or [N, R]) at the observation angles."""
    phi = np.asarray(phi_obs_deg, dtype=np.float64) * math.pi / 180.0
    k = problem.kappa
    c = -(k * problem.eta0 / 4.0) * np.sqrt(2j / (math.pi * k))
    cx = problem.centres[:, 0]
    cy = problem.centres[:, 1]
    steer = np.exp(1j * k * (cx[None, :] * np.cos(phi)[:, None] + cy[None, :] * np.sin(phi)[:, None]))
    xw = np.asarray(x) * (problem.lengths if np.ndim(x) == 1 else problem.lengths[:, None])
    return c * (steer @ xw)


def monostatic(problem, x, phi_inc_deg):
    """Backscatter at each incidence angle for the matching column of x ([N, R])."""
    b = problem.plane_wave(phi_inc_deg)
    k = problem.kappa
    c = -(k * problem.eta0 / 4.0) * np.sqrt(2j / (math.pi * k))
    return c * np.sum(problem.lengths[:, None] * b * np.asarray(x).reshape(b.shape), axis=0)


def far_field_matrix(problem, phi_obs_deg):
    """Dense F with E_far = F x: F[q, n] = C w_n exp(+i kappa (x_n cos phi_q + y_n sin phi_q))."""
    phi = np.asarray(phi_obs_deg, dtype=np.float64) * math.pi / 180.0
    k = problem.kappa
    c = -(k * problem.eta0 / 4.0) * np.sqrt(2j / (math.pi * k))
    cx = problem.centres[:, 0]
    cy = problem.centres[:, 1]
    return c * problem.lengths[None, :] * np.exp(
        1j * k * (cx[None, :] * np.cos(phi)[:, None] + cy[None, :] * np.sin(phi)[:, None]))


def loss_gradient(a_unscaled, problem, b, target, phi_obs_deg):
    """Far-field loss L(b) = sum_q |(F A^{-1} b)_q - t_q|^2 and its gradient
    dL/dRe b + i dL/dIm b = A^{-H} 2 F^H (F x - t) (dense solves written out)."""
    from . import dense
    f = far_field_matrix(problem, phi_obs_deg)
    x = dense.solve(a_unscaled, b)
    e = f @ x
    loss = float(np.sum(np.abs(e - target) ** 2))
    g = 2.0 * f.conj().T @ (e - target)
    lam = dense.solve(a_unscaled.conj().T, g)
    return loss, lam
