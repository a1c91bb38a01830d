"""Oracle: TM_z EFIE impedance matrix by pulse basis and point matching (Sec. 3.1).

TEST INFRASTRUCTURE ONLY.

Definitions (Sec. 3.1, the entries under Eq. (Axb)):
    A_ij = (kappa eta0 w_j / 4) H0^(2)(kappa |rho_i - rho_j|),                 i != j
    A_ii = (kappa eta0 w_i / 4) [1 - i (2/pi) ln(gamma kappa w_i / (4 e))]
    b_i  = E^inc_z(rho_i)
The system is rescaled by a = 1 / max_i |A_ii| so that the largest diagonal
entry has unit magnitude (Sec. 4, first paragraph).
"""
from __future__ import annotations

import math

import numpy as np

from . import geometry
from .hankel import hankel2_0


class Problem:
    """Discretised scatterer: segment centres/lengths plus the EFIE constants."""

    def __init__(self, kind, params, n, wavelength=1.0, eta0=376.73, gamma=1.781072):
        self.kind = int(kind)
        self.params = tuple(params) if self.kind == geometry.POLYLINE else tuple(float(p) for p in params)
        self.n = int(n)
        self.centres, self.lengths = geometry.segments(kind, params, n)
        self.kappa = 2.0 * math.pi / wavelength
        self.eta0 = float(eta0)
        self.gamma = float(gamma)
        self.scale = 1.0 / float(np.max(np.abs(self.diagonal())))

    @classmethod
    def from_workload(cls, wl):
        return cls(wl.kind, wl.params, wl.n)

    def diagonal(self):
        k, w = self.kappa, self.lengths
        return (k * self.eta0 * w / 4.0) * (1.0 - 1j * (2.0 / math.pi) * np.log(self.gamma * k * w / (4.0 * math.e)))

    def entries(self, rows, cols):
        """Unscaled A(rows, cols) as a dense block."""
        rows = np.asarray(rows, dtype=np.int64)
        cols = np.asarray(cols, dtype=np.int64)
        dx = self.centres[rows, 0][:, None] - self.centres[cols, 0][None, :]
        dy = self.centres[rows, 1][:, None] - self.centres[cols, 1][None, :]
        dist = np.hypot(dx, dy)
        same = rows[:, None] == cols[None, :]
        dist_safe = np.where(same, 1.0, dist)
        blk = (self.kappa * self.eta0 * self.lengths[cols][None, :] / 4.0) * hankel2_0(self.kappa * dist_safe)
        if np.any(same):
            d = self.diagonal()
            ii, jj = np.nonzero(same)
            blk[ii, jj] = d[rows[ii]]
        return blk

    def scaled_entries(self, rows, cols):
        return self.scale * self.entries(rows, cols)

    def dense(self, scaled=True):
        idx = np.arange(self.n)
        out = np.empty((self.n, self.n), dtype=np.complex128)
        step = 512
        for r0 in range(0, self.n, step):
            r = idx[r0:r0 + step]
            out[r0:r0 + step] = self.entries(r, idx)
        return self.scale * out if scaled else out

    def plane_wave(self, phi_deg):
        """b_i = exp(-i kappa (x_i cos phi + y_i sin phi)) for each angle (columns)."""
        phi = np.atleast_1d(np.asarray(phi_deg, dtype=np.float64)) * math.pi / 180.0
        x = self.centres[:, 0][:, None]
        y = self.centres[:, 1][:, None]
        return np.exp(-1j * self.kappa * (x * np.cos(phi)[None, :] + y * np.sin(phi)[None, :]))

    def exact_rows_residual(self, rows, x, b, scaled=True):
        """r_i = b_i - sum_j A_ij x_j for the sampled rows, one O(N) row at a time."""
        rows = np.asarray(rows, dtype=np.int64)
        x = np.asarray(x)
        cols = np.arange(self.n)
        out = []
        for i in rows:
            a_row = self.entries(np.array([i]), cols)[0]
            if scaled:
                a_row = a_row * self.scale
            out.append(b[i] - a_row @ x)
        return np.array(out)
