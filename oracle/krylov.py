"""Oracle: Krylov solvers on the split-preconditioned system (Eqs. (Axb2), (Axb3)):
restarted GMRES (the solver the GPU path runs) and TFQMR (the solver of Sec. 4).

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


def tfqmr_split(apply_a, solve_lower, solve_upper, b, rstar=None, rtol=1e-6, maxit=5000):
    """Transpose-free QMR (Freund's method, the solver of the paper's Sec. 4) on the same
    split system L~^{-1} A U~^{-1} y = L~^{-1} b, then x = U~^{-1} y.

    The underlying squared-BiCG recurrence has directions u (with A u kept) and p (with
    v = A p kept).  Half steps m = 0, 1, 2, ...: an even step takes a new alpha =
    rho / (r*, v) and the direction u; the odd step that follows uses the second
    direction q = u - alpha v.  Each half step updates the squared residual w, the QMR
    direction d and the iterate (theta, c, tau, eta); after an odd step the new
    rho = (r*, w) gives beta, u = w + beta q and v = A u + beta (A q + beta v).
    tau sqrt(m + 1) bounds the split system's residual; when it reaches
    rtol ||L~^{-1} b|| the true residual ||b - A x|| / ||b|| is checked (and the bound
    tightened if it misses).  Returns (x, info) with info = dict(iters=half steps,
    matvecs=products with the split operator, true_rel_res).

    rstar is the shadow vector r* of the Lanczos biorthogonalisation.  Sec. 4 does not say
    which one was used; the default is the initial residual L~^{-1} b.  On the strip that
    choice meets a near-breakdown (theta grows to ~1e3 and the iteration stalls near a
    1e-5 relative residual), while a random complex Gaussian r*, drawn by the caller,
    converges in about as many products as GMRES.
    """
    op = lambda z: solve_lower(apply_a(solve_upper(z)))
    b = np.asarray(b, dtype=np.complex128)
    bnorm = np.linalg.norm(b)
    rhs = solve_lower(b)
    n = rhs.shape[0]
    y = np.zeros(n, dtype=np.complex128)
    w = rhs.copy()                      # y = 0: r = rhs
    u = rhs.copy()
    rstar = rhs.copy() if rstar is None else np.asarray(rstar, dtype=np.complex128)
    v = op(u)                           # p = u at the start: A p = A u
    au_first = v
    matvecs = 1
    d = np.zeros(n, dtype=np.complex128)
    tau = np.linalg.norm(rhs)
    theta = 0.0
    eta = 0.0
    rho = np.vdot(rstar, rhs)
    alpha = 0.0
    u_second = None
    target = rtol * np.linalg.norm(rhs)
    true_res = 1.0
    m = 0
    while m < maxit:
        if m % 2 == 0:
            alpha = rho / np.vdot(rstar, v)
            u_second = u - alpha * v
            au = au_first               # A u, kept from the previous step
        else:
            au = op(u)                  # u = the second direction q of this step
            matvecs += 1
        w = w - alpha * au
        d = u + (theta ** 2 * eta / alpha) * d
        theta = np.linalg.norm(w) / tau
        c = 1.0 / np.sqrt(1.0 + theta ** 2)
        tau = tau * theta * c
        eta = c ** 2 * alpha
        y = y + eta * d
        if m % 2 == 1:
            rho_new = np.vdot(rstar, w)
            beta = rho_new / rho
            rho = rho_new
            u_new = w + beta * u
            au_new = op(u_new)
            matvecs += 1
            v = au_new + beta * (au + beta * v)
            u = u_new
            au_first = au_new
        else:
            u = u_second
        m += 1
        if tau * np.sqrt(m + 1.0) <= target:
            x = solve_upper(y)
            true_res = np.linalg.norm(b - apply_a(x)) / bnorm
            if true_res <= rtol:
                break
            target *= min(0.5, rtol / true_res)
    x = solve_upper(y)
    true_res = np.linalg.norm(b - apply_a(x)) / bnorm
    return x, dict(iters=m, matvecs=matvecs, true_rel_res=true_res)
