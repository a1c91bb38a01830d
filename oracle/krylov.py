"""Oracle: restarted GMRES on the split-preconditioned system (Eqs. (Axb2), (Axb3)).

TEST INFRASTRUCTURE ONLY.

Solve  L~^{-1} A U~^{-1} y = L~^{-1} b  with GMRES(restart) (modified Gram-Schmidt
Arnoldi, Givens rotations), then  x = U~^{-1} y.  Stopping rule (reading of
the solver settings in Sec. 4): the TRUE relative residual ||b - A x|| / ||b||
must reach `rtol`; it is checked whenever the Arnoldi estimate of the
preconditioned residual reaches its current target and at every restart.
"""
from __future__ import annotations

import numpy as np


def gmres_split(apply_a, solve_lower, solve_upper, b, rtol=1e-6, restart=30, maxit=2000):
    """Return (x, info) where info = dict(iters, restarts, true_rel_res)."""
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    n = b.shape[0]
    y = np.zeros(n, dtype=np.complex128)
    rhs = solve_lower(b)
    target_scale = 1.0
    iters = 0
    restarts = 0
    x = np.zeros(n, dtype=np.complex128)
    true_res = 1.0
    while iters < maxit:
        r = rhs - solve_lower(apply_a(solve_upper(y)))
        beta = np.linalg.norm(r)
        target = rtol * target_scale * np.linalg.norm(rhs)
        if beta <= target:
            break
        v = np.zeros((restart + 1, n), dtype=np.complex128)
        h = np.zeros((restart + 1, restart), dtype=np.complex128)
        cs = np.zeros(restart, dtype=np.complex128)
        sn = np.zeros(restart, dtype=np.complex128)
        g = np.zeros(restart + 1, dtype=np.complex128)
        g[0] = beta
        v[0] = r / beta
        j_used = 0
        for j in range(restart):
            w = solve_lower(apply_a(solve_upper(v[j])))
            for i in range(j + 1):                      # modified Gram-Schmidt
                h[i, j] = np.vdot(v[i], w)
                w = w - h[i, j] * v[i]
            h[j + 1, j] = np.linalg.norm(w)
            if h[j + 1, j] != 0:
                v[j + 1] = w / h[j + 1, j]
            for i in range(j):                          # previous rotations G_i = [[c*, s*], [-s, c]]
                t = np.conj(cs[i]) * h[i, j] + np.conj(sn[i]) * h[i + 1, j]
                h[i + 1, j] = -sn[i] * h[i, j] + cs[i] * h[i + 1, j]
                h[i, j] = t
            # new rotation zeroing h[j+1, j]
            a_, b_ = h[j, j], h[j + 1, j]
            den = np.sqrt(abs(a_) ** 2 + abs(b_) ** 2)
            cs[j] = a_ / den if den else 1.0
            sn[j] = b_ / den if den else 0.0
            h[j, j] = cs[j].conjugate() * a_ + sn[j].conjugate() * b_
            h[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = np.conj(cs[j]) * g[j]
            iters += 1
            j_used = j + 1
            if abs(g[j + 1]) <= target or iters >= maxit:
                break
        # back substitution for the least-squares coefficients
        k = j_used
        coef = np.zeros(k, dtype=np.complex128)
        for i in range(k - 1, -1, -1):
            coef[i] = (g[i] - h[i, i + 1:k] @ coef[i + 1:k]) / h[i, i]
        y = y + coef @ v[:k]
        restarts += 1
        x = solve_upper(y)
        true_res = np.linalg.norm(b - apply_a(x)) / bnorm
        if true_res <= rtol:
            break
        # tighten the internal target in proportion to the miss
        target_scale *= min(0.5, rtol / true_res)
    return x, dict(iters=iters, restarts=restarts, true_rel_res=true_res)
