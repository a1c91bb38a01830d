"""Seeded synthetic workloads shared by the oracle, the tests and the benchmark.

This module holds only problem *definitions* (geometry parameters, sizes,
tolerances) and seeded random draws (incidence angles, random vectors).  It
contains none of the method's arithmetic: no discretisation, no kernel
entries, no compression, no solves.  Both the CPU oracle and the CUDA path
take their inputs from here, and neither imports the other.

Geometries are the paper's kind of scatterer (open PEC curves discretised at a
fixed number of pulse segments per wavelength, Sec. 4); wavelength = 1.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# Geometry kinds (same numbering as the C ABI's hb_geometry kinds).
STRIP = 0            # params (x0, y0, x1, y1)
SPIRAL = 1           # params (a, theta0, theta1): r = a*theta
ARC = 2              # params (R, phi0, phi1): circle arc centred at the origin
PARALLEL_STRIPS = 3  # params (n_strips, length, spacing): y = s*spacing, x in [0, length]
POLYLINE = 4         # explicit nodes (hb_geometry_polyline): params (nodes [n+c, 2], curve_starts [c])

# Physical constants fixed by the problem statement (wavelength lambda = 1).
WAVELENGTH = 1.0
ETA0 = 376.73
GAMMA = 1.781072

# Archimedean spiral r = a*theta over theta in [2*pi, 8*pi]; `a` chosen so that
# the arc length equals the stated value.  The literals were computed once at
# 30 significant digits from s(theta) = (a/2) [theta sqrt(1+theta^2) + asinh theta].
SPIRAL_A_3276_8 = 11.041182539781965448     # arc length 3276.8 lambda
SPIRAL_A_209715_2 = 706.63568254604578868   # arc length 209,715.2 lambda
# Semicircle of arc length 6553.6 lambda: R = 6553.6/pi.
SEMICIRCLE_R_6553_6 = 2086.075670094090545


@dataclass(frozen=True)
class Workload:
    name: str
    kind: int
    params: tuple
    n: int              # number of unknowns N (= leaf * 2^D)
    leaf: int           # n0
    eps: float          # compression tolerance
    form: str           # "c128" | "c64" | "split_bf16"
    nrhs: int = 1
    note: str = ""
    extra: dict = field(default_factory=dict)

    @property
    def depth(self) -> int:
        m = self.n // self.leaf
        return int(round(math.log2(m)))


def strip(n: int, leaf: int, eps: float, length: float | None = None, form="c128") -> Workload:
    """Straight strip from (0,0) to (length,0) at 20 segments per wavelength by default."""
    if length is None:
        length = n / 20.0
    return Workload(f"strip_N{n}", STRIP, (0.0, 0.0, float(length), 0.0), n, leaf, eps, form)


def spiral(n: int, leaf: int, eps: float, a: float, form="c64", nrhs=1) -> Workload:
    return Workload(f"spiral_N{n}", SPIRAL, (float(a), 2 * math.pi, 8 * math.pi), n, leaf, eps, form, nrhs)


def arc(n: int, leaf: int, eps: float, radius: float, phi0=0.0, phi1=math.pi, form="c64", nrhs=1) -> Workload:
    return Workload(f"arc_N{n}", ARC, (float(radius), float(phi0), float(phi1)), n, leaf, eps, form, nrhs)


def parallel_strips(n: int, leaf: int, eps: float, n_strips=8, length=None, spacing=2.0, form="c64") -> Workload:
    if length is None:
        length = n / n_strips / 20.0
    return Workload(f"strips{n_strips}_N{n}", PARALLEL_STRIPS, (float(n_strips), float(length), float(spacing)),
                    n, leaf, eps, form)


# The five workloads of the measurement plan.
STRIP_N1024 = Workload("strip_N1024", STRIP, (0.0, 0.0, 51.2, 0.0), 1024, 32, 1e-6, "c128",
                   note="plain FP64 form; one plane wave at 30 deg")
SPIRAL_N65536 = Workload("spiral_N65536", SPIRAL, (SPIRAL_A_3276_8, 2 * math.pi, 8 * math.pi), 65536, 64, 1e-6, "c64",
                   note="complex FP32 apply/preconditioner, FP64 outer FGMRES + IR; phi ~ U[0,180) seed 0")
SEMICIRCLE_N262144 = Workload("semicircle_N262144", ARC, (SEMICIRCLE_R_6553_6, 0.0, math.pi), 262144, 64, 1e-6, "split_bf16",
                   nrhs=256, note="256 plane waves, multi-RHS block")
STRIPS8_N131072 = Workload("strips8_N131072", PARALLEL_STRIPS, (8.0, 409.6, 2.0), 131072, 64, 1e-6, "c64",
                   note="adjoint form; far-field loss")
SPIRAL_N4194304 = Workload("spiral_N4194304", SPIRAL, (SPIRAL_A_209715_2, 2 * math.pi, 8 * math.pi), 4194304, 128, 1e-5,
                   "c64", nrhs=16, note="scale form")

WORKLOADS = {wl.name: wl for wl in (STRIP_N1024, SPIRAL_N65536, SEMICIRCLE_N262144, STRIPS8_N131072, SPIRAL_N4194304)}


# ----------------------------------------------------------------------------
# Seeded draws
# ----------------------------------------------------------------------------

def incidence_angles_deg(wl: Workload) -> np.ndarray:
    """Incidence angles (degrees) of the plane waves of a workload."""
    if wl.name in ("strip_N1024", "strips8_N131072"):
        return np.array([30.0])
    if wl.name == "spiral_N65536":
        return np.random.default_rng(0).uniform(0.0, 180.0, size=1)
    if wl.name == "semicircle_N262144":
        return 180.0 * np.arange(256) / 256.0
    if wl.name == "spiral_N4194304":
        return 180.0 * np.arange(16) / 16.0
    raise ValueError(wl.name)


def observation_angles_deg(n_obs: int = 64) -> np.ndarray:
    """Observation angles uniform in [0, 360) degrees."""
    return 360.0 * np.arange(n_obs) / n_obs


def complex_gaussian(n: int, seed: int, ncols: int | None = None) -> np.ndarray:
    """CN(0, 1) samples: real and imaginary parts N(0, 1/2)."""
    rng = np.random.default_rng(seed)
    shape = (n,) if ncols is None else (n, ncols)
    return (rng.standard_normal(shape) + 1j * rng.standard_normal(shape)) / math.sqrt(2.0)


def sample_rows(n: int, count: int, seed: int) -> np.ndarray:
    """Seeded distinct row indices for sampled exact-row checks at large N."""
    rng = np.random.default_rng(seed)
    return np.sort(rng.choice(n, size=min(count, n), replace=False)).astype(np.int64)


# Seeds used across tests and the benchmark.
SEED_XTRUE = 3      # x^t ~ CN(0, I) for the b = A x^t protocol (Sec. 4)
SEED_TARGET = 1     # far-field target t ~ CN(0,1)
SEED_FD = 2         # finite-difference directions d ~ CN(0, I)
SEED_ROWS = 7       # sampled rows for exact residual checks
SEED_SHADOW = 11    # TFQMR shadow vector r* ~ CN(0, I)
