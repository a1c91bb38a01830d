"""Oracle: dense linear algebra written out (LU with partial pivoting, triangular solves).

TEST INFRASTRUCTURE ONLY.

Also builds the entry-wise triangular matrices of Sec. 3.1 (Eqs. (Lt), (Ut)):
    L~(i,j) = 0 (i<j), 1 (i=j), A(i,j) (i>j);   U~(i,j) = 0 (i>j), A(i,j) (i<=j)
and the split-preconditioned operator L~^{-1} A U~^{-1} of Eq. (Axb2).
"""
from __future__ import annotations

import numpy as np


def lu_factor(a):
    """Doolittle LU with partial (row) pivoting: P A = L U.  Returns (lu, perm)."""
    lu = np.array(a, dtype=np.complex128, copy=True)
    n = lu.shape[0]
    perm = np.arange(n)
    for k in range(n):
        p = k + int(np.argmax(np.abs(lu[k:, k])))
        if p != k:
            lu[[k, p]] = lu[[p, k]]
            perm[[k, p]] = perm[[p, k]]
        piv = lu[k, k]
        if piv == 0:
            raise ZeroDivisionError("singular matrix")
        lu[k + 1:, k] /= piv
        lu[k + 1:, k + 1:] -= np.outer(lu[k + 1:, k], lu[k, k + 1:])
    return lu, perm


def forward_subst(lower, b, unit=False):
    """Solve lower x = b by forward substitution (b may have several columns)."""
    b = np.array(b, dtype=np.complex128, copy=True)
    n = lower.shape[0]
    for i in range(n):
        if i:
            b[i] -= lower[i, :i] @ b[:i]
        if not unit:
            b[i] /= lower[i, i]
    return b


def back_subst(upper, b, unit=False):
    """Solve upper x = b by back substitution."""
    b = np.array(b, dtype=np.complex128, copy=True)
    n = upper.shape[0]
    for i in range(n - 1, -1, -1):
        if i < n - 1:
            b[i] -= upper[i, i + 1:] @ b[i + 1:]
        if not unit:
            b[i] /= upper[i, i]
    return b


def lu_solve(lu, perm, b):
    y = forward_subst(lu, np.asarray(b)[perm], unit=True)
    return back_subst(lu, y, unit=False)


def solve(a, b):
    lu, perm = lu_factor(a)
    return lu_solve(lu, perm, b)


def l_tilde(a):
    """Eq. (Lt): strict lower part of A with a unit diagonal."""
    out = np.tril(a, -1)
    np.fill_diagonal(out, 1.0)
    return out


def u_tilde(a):
    """Eq. (Ut): upper part of A including the diagonal."""
    return np.triu(a)


def leaf_lu(block):
    """LU without pivoting (Doolittle): block = L U, L unit lower, U upper (the exact
    leaf LU variant of the leaf solves of Algs. 3/4)."""
    n = block.shape[0]
    lo = np.eye(n, dtype=np.complex128)
    up = np.zeros((n, n), dtype=np.complex128)
    for k in range(n):
        up[k, k:] = block[k, k:] - lo[k, :k] @ up[:k, k:]
        lo[k + 1:, k] = (block[k + 1:, k] - lo[k + 1:, :k] @ up[:k, k]) / up[k, k]
    return lo, up


def l_tilde_leaf_lu(a, n0):
    """L~ with each n0 x n0 diagonal block replaced by the L factor of that block of A."""
    out = l_tilde(a)
    for s in range(0, a.shape[0], n0):
        out[s:s + n0, s:s + n0] = leaf_lu(a[s:s + n0, s:s + n0])[0]
    return out


def u_tilde_leaf_lu(a, n0):
    """U~ with each n0 x n0 diagonal block replaced by the U factor of that block of A."""
    out = u_tilde(a)
    for s in range(0, a.shape[0], n0):
        out[s:s + n0, s:s + n0] = leaf_lu(a[s:s + n0, s:s + n0])[1]
    return out


def precond_solve(a, b):
    """x = U~^{-1} L~^{-1} b with the exact entry-wise triangles of A."""
    y = forward_subst(l_tilde(a), b, unit=True)
    return back_subst(u_tilde(a), y, unit=False)


def split_operator(a):
    """Dense L~^{-1} A U~^{-1} (Eq. (Axb2))."""
    lt, ut = l_tilde(a), u_tilde(a)
    left = forward_subst(lt, a, unit=True)                     # L~^{-1} A
    # (L~^{-1} A) U~^{-1} = (U~^{-T} (L~^{-1} A)^T)^T
    return forward_subst(ut.T, left.T, unit=False).T
