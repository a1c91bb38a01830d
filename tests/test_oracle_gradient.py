"""Pins for the oracle's far-field loss gradient (adjoint form; no counterpart in the paper)."""
import numpy as np

import workloads as W
from oracle import efie, farfield


def test_far_field_matrix_matches_direct_sum():
    p = efie.Problem(W.PARALLEL_STRIPS, (2.0, 3.2, 2.0), 128)
    x = W.complex_gaussian(128, 50)
    phi = W.observation_angles_deg(16)
    np.testing.assert_allclose(farfield.far_field_matrix(p, phi) @ x, farfield.far_field(p, x, phi), rtol=1e-12)


def test_loss_gradient_central_difference():
    # L is quadratic in b, so the central difference has no truncation error:
    # [L(b+hd) - L(b-hd)] / (2h) = Re(lambda^H d) up to rounding.
    p = efie.Problem(W.PARALLEL_STRIPS, (2.0, 3.2, 2.0), 128)
    a = p.dense(scaled=False)
    phi = W.observation_angles_deg(16)
    t = W.complex_gaussian(16, W.SEED_TARGET)
    b = p.plane_wave(30.0)[:, 0]
    loss, lam = farfield.loss_gradient(a, p, b, t, phi)
    d = W.complex_gaussian(128, W.SEED_FD, 4)
    for j in range(4):
        h = 1e-4
        lp, _ = farfield.loss_gradient(a, p, b + h * d[:, j], t, phi)
        lm, _ = farfield.loss_gradient(a, p, b - h * d[:, j], t, phi)
        fd = (lp - lm) / (2 * h)
        assert abs(fd - np.real(np.vdot(lam, d[:, j]))) <= 1e-7 * max(1.0, abs(fd))
