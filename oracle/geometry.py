"""Oracle: discretisation of open PEC curves into pulse segments (Sec. 3.1).

TEST INFRASTRUCTURE ONLY.

Each pulse basis function lives on a straight segment; w_i is its length and
rho_i its centre (Sec. 3.1, the definitions under Eq. (Axb)).  Curved
scatterers are split into N pieces of equal arc length along the exact curve;
each segment is the chord between consecutive nodes (centre = chord
midpoint, w = chord length).  Unknowns follow the curve parameter (the
geometric order of Sec. 3.3.1); several strips are ordered strip after strip.
"""
from __future__ import annotations

import math

import numpy as np

STRIP, SPIRAL, ARC, PARALLEL_STRIPS, POLYLINE = 0, 1, 2, 3, 4


def _chords(nodes_x, nodes_y):
    cx = 0.5 * (nodes_x[1:] + nodes_x[:-1])
    cy = 0.5 * (nodes_y[1:] + nodes_y[:-1])
    w = np.hypot(nodes_x[1:] - nodes_x[:-1], nodes_y[1:] - nodes_y[:-1])
    return np.stack([cx, cy], axis=1), w


def spiral_arclength(a, theta):
    """Arc length of r = a*theta from 0 to theta: (a/2)[theta sqrt(1+theta^2) + asinh(theta)]."""
    return 0.5 * a * (theta * np.sqrt(1.0 + theta * theta) + np.arcsinh(theta))


def spiral_nodes(a, theta0, theta1, n):
    """Nodes theta_0..theta_n at equal arc length (Newton on s(theta) = target)."""
    s0 = spiral_arclength(a, theta0)
    s1 = spiral_arclength(a, theta1)
    target = s0 + (s1 - s0) * np.arange(n + 1, dtype=np.float64) / n
    # initial guess: linear in theta, then Newton with ds/dtheta = a sqrt(1+theta^2)
    th = theta0 + (theta1 - theta0) * np.arange(n + 1, dtype=np.float64) / n
    for _ in range(60):
        f = spiral_arclength(a, th) - target
        th_new = th - f / (a * np.sqrt(1.0 + th * th))
        if np.max(np.abs(th_new - th)) < 1e-15 * max(abs(theta1), 1.0):
            th = th_new
            break
        th = th_new
    th[0], th[-1] = theta0, theta1
    return th


def polyline_segments(nodes, curve_starts=(0,)):
    """Explicit scatterer: curves given by their nodes (rows of `nodes`, x and y); curve c
    uses nodes curve_starts[c] .. curve_starts[c+1] - 1 (the last one up to the end) and
    contributes one segment per pair of consecutive nodes."""
    nodes = np.asarray(nodes, dtype=np.float64)
    starts = [int(c) for c in curve_starts] + [len(nodes)]
    cs, ws = [], []
    for c in range(len(starts) - 1):
        sub = nodes[starts[c]:starts[c + 1]]
        cc, w = _chords(sub[:, 0], sub[:, 1])
        cs.append(cc)
        ws.append(w)
    return np.concatenate(cs), np.concatenate(ws)


def segments(kind, params, n):
    """Return (centres [n,2], lengths [n]) for the curve `kind` with `params`
    (POLYLINE: params = (nodes, curve_starts), see polyline_segments)."""
    kind = int(kind)
    if kind == POLYLINE:
        nodes, starts = params
        c, w = polyline_segments(nodes, starts)
        if len(w) != n:
            raise ValueError("polyline: n does not match the node list")
        return c, w
    if kind == STRIP:
        x0, y0, x1, y1 = params
        t = np.arange(n + 1, dtype=np.float64) / n
        return _chords(x0 + (x1 - x0) * t, y0 + (y1 - y0) * t)
    if kind == SPIRAL:
        a, th0, th1 = params
        th = spiral_nodes(a, th0, th1, n)
        r = a * th
        return _chords(r * np.cos(th), r * np.sin(th))
    if kind == ARC:
        radius, p0, p1 = params
        ph = p0 + (p1 - p0) * np.arange(n + 1, dtype=np.float64) / n
        return _chords(radius * np.cos(ph), radius * np.sin(ph))
    if kind == PARALLEL_STRIPS:
        ns, length, spacing = params
        ns = int(round(ns))
        if n % ns:
            raise ValueError("segments must divide evenly among strips")
        per = n // ns
        cs, ws = [], []
        for s in range(ns):
            t = np.arange(per + 1, dtype=np.float64) / per
            c, w = _chords(length * t, np.full(per + 1, s * spacing))
            cs.append(c)
            ws.append(w)
        return np.concatenate(cs), np.concatenate(ws)
    raise ValueError(f"unknown geometry kind {kind}")
