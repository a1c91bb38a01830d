"""Oracle: naive IDBF, H-IDBF (Alg. 1), its apply (Alg. 2) and the L~/U~ sweeps (Algs. 3, 4).

TEST INFRASTRUCTURE ONLY.  Plain and slow on purpose: every interpolative
decomposition is a pivoted QR of the FULL dense sub-block (no sampling), and
every step runs in the order the factorisation states.

Interpolative decomposition (Appendix, Sec. "Linear scaling interpolative
decompositions"): a pivoted QR  M Lambda = Q [R1 R2]  truncated at rank k gives
T = R1^{-1} R2 and the column ID  M ~ M(:, q) [I T] Lambda^*,  i.e.
M(:, p) ~ M(:, q) T.  A row ID is the column ID of M^T:  M(p, :) ~ T^T M(q, :).
Truncation (reading of Eq. (req)): the first k with |R_kk| <= tol |R_00|.

Butterfly structure (reading of Eq. (BFM) and the recursive MSCS, Appendix):
an n x n complementary low-rank block with L = log2(n/n0) levels factorises as
    K ~ U^0 U^1 ... U^{hr-1} S V^{hc-1} ... V^1 V^0
* column stage l (l = 0..hc-1) pairs row node a at level l with column node b
  at level L-l; its column ID selects skeleton columns cskel(a,b) from the
  candidates (the n0 leaf columns at l = 0, else cskel(a>>1, 2b) U cskel(a>>1, 2b+1));
* row stage l (l = 0..hr-1) pairs row node a at level L-l with column node b at
  level l; its row ID selects rskel(a,b) from the n0 leaf rows (l = 0) or from
  rskel(2a, b>>1) U rskel(2a+1, b>>1);
* the middle factor holds S(a,b) = K(rskel(a,b), cskel(a,b)) for the pairs
  where both sides meet (row level hc-1, column level L-hc+1);
* hc + hr = L + 2; hc = L/2 + 1 for even L, hc = (L+1)/2 for odd L.
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------------------
# Interpolative decomposition
# ----------------------------------------------------------------------------

def pivoted_qr(m):
    """Householder QR with column pivoting (largest remaining column norm, ties -> lowest index).

    Returns (perm, r) with m[:, perm] = Q r, r upper trapezoidal (min(rows,cols) x cols).
    """
    a = np.array(m, dtype=np.complex128, copy=True)
    rows, cols = a.shape
    perm = np.arange(cols)
    steps = min(rows, cols)
    for j in range(steps):
        norms = np.sum(np.abs(a[j:, j:]) ** 2, axis=0)
        p = j + int(np.argmax(norms))
        if p != j:
            a[:, [j, p]] = a[:, [p, j]]
            perm[[j, p]] = perm[[p, j]]
        x = a[j:, j].copy()
        alpha = np.linalg.norm(x)
        if alpha == 0.0:
            continue
        phase = x[0] / abs(x[0]) if x[0] != 0 else 1.0
        v = x.copy()
        v[0] += phase * alpha
        v /= np.linalg.norm(v)
        # apply H = I - 2 v v^H to the trailing block
        a[j:, j:] -= 2.0 * np.outer(v, v.conj() @ a[j:, j:])
    r = np.triu(a[:steps, :])
    return perm, r


def column_id(m, tol):
    """Column ID of m: returns (q, p, t) with m[:, p] ~ m[:, q] @ t."""
    rows, cols = m.shape
    perm, r = pivoted_qr(m)
    diag = np.abs(np.diag(r))
    k = len(diag)
    if len(diag) and diag[0] > 0:
        small = np.nonzero(diag <= tol * diag[0])[0]
        if len(small):
            k = int(small[0])
    k = max(k, 1)
    k = min(k, cols)
    q, p = perm[:k], perm[k:]
    if len(p):
        t = np.linalg.solve(np.triu(r[:k, :k]), r[:k, k:])   # T = R1^{-1} R2 (triangular system)
    else:
        t = np.zeros((k, 0), dtype=np.complex128)
    return q, p, t


def row_id(m, tol):
    """Row ID of m: returns (q, p, e) with m[p, :] ~ e @ m[q, :] (e = T^T of the column ID of m^T)."""
    q, p, t = column_id(m.T, tol)
    return q, p, t.T


# ----------------------------------------------------------------------------
# One butterfly (IDBF of one complementary low-rank block)
# ----------------------------------------------------------------------------

def stage_counts(levels):
    hc = levels // 2 + 1 if levels % 2 == 0 else (levels + 1) // 2
    return hc, levels + 2 - hc


class Butterfly:
    """IDBF of a dense n x n block with leaves of n0 rows/columns."""

    def __init__(self, block, n0, tol):
        block = np.asarray(block)
        n = block.shape[0]
        assert block.shape == (n, n) and n % n0 == 0
        levels = int(round(np.log2(n // n0)))
        assert n0 << levels == n
        self.n, self.n0, self.levels = n, n0, levels
        self.hc, self.hr = stage_counts(levels)
        L = levels
        # ---- column stages: col[l][(a, b)] = (skel, q, p, t)
        self.col = []
        for l in range(self.hc):
            stage = {}
            rsz = n >> l
            for a in range(1 << l):
                rows = np.arange(a * rsz, (a + 1) * rsz)
                for b in range(1 << (L - l)):
                    if l == 0:
                        cand = np.arange(b * n0, (b + 1) * n0)
                    else:
                        cand = np.concatenate([self.col[l - 1][(a >> 1, 2 * b)][0],
                                               self.col[l - 1][(a >> 1, 2 * b + 1)][0]])
                    q, p, t = column_id(block[np.ix_(rows, cand)], tol)
                    stage[(a, b)] = (cand[q], q, p, t)
            self.col.append(stage)
        # ---- row stages: row[l][(a, b)] = (skel, q, p, e)
        self.row = []
        for l in range(self.hr):
            stage = {}
            csz = n >> l
            for b in range(1 << l):
                cols = np.arange(b * csz, (b + 1) * csz)
                for a in range(1 << (L - l)):
                    if l == 0:
                        cand = np.arange(a * n0, (a + 1) * n0)
                    else:
                        cand = np.concatenate([self.row[l - 1][(2 * a, b >> 1)][0],
                                               self.row[l - 1][(2 * a + 1, b >> 1)][0]])
                    q, p, e = row_id(block[np.ix_(cand, cols)], tol)
                    stage[(a, b)] = (cand[q], q, p, e)
            self.row.append(stage)
        # ---- middle factor
        self.mid = {}
        for (a, b), (cskel, *_rest) in self.col[self.hc - 1].items():
            rskel = self.row[self.hr - 1][(a, b)][0]
            self.mid[(a, b)] = block[np.ix_(rskel, cskel)]

    # -- storage count (ID form: only T/E and the middle blocks are stored)
    def nnz(self):
        total = 0
        for stage in self.col + self.row:
            for (_s, _q, _p, t) in stage.values():
                total += t.size
        for s in self.mid.values():
            total += s.size
        return total

    def max_rank(self):
        ks = [len(v[0]) for st in self.col + self.row for v in st.values()]
        return max(ks) if ks else 0

    def apply(self, x):
        """K_F x for x of shape (n,) or (n, r): V stages, middle, then U stages."""
        x = np.asarray(x, dtype=np.complex128)
        squeeze = x.ndim == 1
        if squeeze:
            x = x[:, None]
        n0, L = self.n0, self.levels
        # V^0 ... V^{hc-1}
        z = {}
        for l in range(self.hc):
            znew = {}
            for (a, b), (_skel, q, p, t) in self.col[l].items():
                if l == 0:
                    cand_vals = x[b * n0:(b + 1) * n0]
                else:
                    cand_vals = np.concatenate([z[(a >> 1, 2 * b)], z[(a >> 1, 2 * b + 1)]])
                znew[(a, b)] = cand_vals[q] + t @ cand_vals[p]
            z = znew
        # S
        y = {ab: self.mid[ab] @ z[ab] for ab in self.mid}
        # U^{hr-1} ... U^0
        for l in range(self.hr - 1, 0, -1):
            ynew = {}
            for (a, b), (_skel, q, p, e) in self.row[l].items():
                k0 = len(self.row[l - 1][(2 * a, b >> 1)][0])
                full = np.zeros((len(q) + len(p), x.shape[1]), dtype=np.complex128)
                full[q] = y[(a, b)]
                full[p] = e @ y[(a, b)]
                for child, part in ((2 * a, full[:k0]), (2 * a + 1, full[k0:])):
                    key = (child, b >> 1)
                    ynew[key] = ynew[key] + part if key in ynew else part
            y = ynew
        out = np.zeros((self.n, x.shape[1]), dtype=np.complex128)
        for (a, b), (_skel, q, p, e) in self.row[0].items():
            full = np.zeros((n0, x.shape[1]), dtype=np.complex128)
            full[q] = y[(a, b)]
            full[p] = e @ y[(a, b)]
            out[a * n0:(a + 1) * n0] += full
        return out[:, 0] if squeeze else out

    def apply_adjoint(self, x):
        """K_F^H x: the conjugate-transposed factors in reverse order."""
        x = np.asarray(x, dtype=np.complex128)
        squeeze = x.ndim == 1
        if squeeze:
            x = x[:, None]
        n0 = self.n0
        # (U^0)^H: y(a,0) = full[q] + e^H full[p] with full = x(rows of leaf a)
        y = {}
        for (a, b), (_skel, q, p, e) in self.row[0].items():
            full = x[a * n0:(a + 1) * n0]
            y[(a, b)] = full[q] + e.conj().T @ full[p]
        for l in range(1, self.hr):
            ynew = {}
            for (a, b), (_skel, q, p, e) in self.row[l].items():
                full = np.concatenate([y[(2 * a, b >> 1)], y[(2 * a + 1, b >> 1)]])
                ynew[(a, b)] = full[q] + e.conj().T @ full[p]
            y = ynew
        z = {ab: self.mid[ab].conj().T @ y[ab] for ab in self.mid}
        for l in range(self.hc - 1, 0, -1):
            znew = {}
            for (a, b), (_skel, q, p, t) in self.col[l].items():
                k0 = len(self.col[l - 1][(a >> 1, 2 * b)][0])
                full = np.zeros((len(q) + len(p), x.shape[1]), dtype=np.complex128)
                full[q] = z[(a, b)]
                full[p] = t.conj().T @ z[(a, b)]
                for child, part in ((2 * b, full[:k0]), (2 * b + 1, full[k0:])):
                    key = (a >> 1, child)
                    znew[key] = znew[key] + part if key in znew else part
            z = znew
        out = np.zeros((self.n, x.shape[1]), dtype=np.complex128)
        for (a, b), (_skel, q, p, t) in self.col[0].items():
            full = np.zeros((n0, x.shape[1]), dtype=np.complex128)
            full[q] = z[(a, b)]
            full[p] = t.conj().T @ z[(a, b)]
            out[b * n0:(b + 1) * n0] += full
        return out[:, 0] if squeeze else out

    def dense(self):
        return self.apply(np.eye(self.n, dtype=np.complex128))


# ----------------------------------------------------------------------------
# H-IDBF (Algorithm 1) and its apply / sweeps (Algorithms 2-4)
# ----------------------------------------------------------------------------

def butterfly_within_tolerance(block, n0, eps):
    """IDBF of `block` with ID tolerance eps; if the Frobenius block error misses eps,
    rebuild with eps/10 (reading of the tolerance rule of Eq. (req))."""
    bf = Butterfly(block, n0, eps)
    nb = np.linalg.norm(block)
    if np.linalg.norm(bf.dense() - block) > eps * nb:
        bf = Butterfly(block, n0, eps / 10.0)
    return bf


class HIDBF:
    """Recursive H-IDBF of a dense N x N matrix (weak admissibility, Alg. 1)."""

    def __init__(self, a, n0, tol):
        a = np.asarray(a)
        self.n = a.shape[0]
        self.n0 = n0
        if self.n <= n0:
            self.leaf = np.array(a, copy=True)
            return
        self.leaf = None
        h = self.n // 2
        self.f11 = HIDBF(a[:h, :h], n0, tol)
        self.f22 = HIDBF(a[h:, h:], n0, tol)
        self.f12 = butterfly_within_tolerance(a[:h, h:], n0, tol)
        self.f21 = butterfly_within_tolerance(a[h:, :h], n0, tol)

    def butterflies(self):
        if self.leaf is not None:
            return []
        return [self.f12, self.f21] + self.f11.butterflies() + self.f22.butterflies()

    def nnz(self):
        if self.leaf is not None:
            return self.leaf.size
        return self.f11.nnz() + self.f22.nnz() + self.f12.nnz() + self.f21.nnz()

    def apply(self, v, adjoint=False):
        """Alg. 2: u = A v (or A^H v).  The leaf line multiplies v (reading of the typo in Alg. 2)."""
        v = np.asarray(v, dtype=np.complex128)
        if self.leaf is not None:
            m = self.leaf.conj().T if adjoint else self.leaf
            return m @ v
        h = self.n // 2
        u = np.zeros_like(v)
        u[:h] = self.f11.apply(v[:h], adjoint)
        u[h:] = self.f22.apply(v[h:], adjoint)
        if not adjoint:
            u[h:] += self.f21.apply(v[:h])
            u[:h] += self.f12.apply(v[h:])
        else:
            u[h:] += self.f12.apply_adjoint(v[:h])
            u[:h] += self.f21.apply_adjoint(v[h:])
        return u

    def solve_lower(self, b):
        """Alg. 3: x = L~^{-1} b, L~ = unit-diagonal lower part of the H-IDBF."""
        b = np.array(b, dtype=np.complex128, copy=True)
        if self.leaf is not None:
            return _trsv_lower_unit(self.leaf, b)
        h = self.n // 2
        x = np.zeros_like(b)
        x[:h] = self.f11.solve_lower(b[:h])
        b[h:] -= self.f21.apply(x[:h])
        x[h:] = self.f22.solve_lower(b[h:])
        return x

    def solve_upper(self, b):
        """Alg. 4: x = U~^{-1} b, U~ = upper part (with diagonal) of the H-IDBF."""
        b = np.array(b, dtype=np.complex128, copy=True)
        if self.leaf is not None:
            return _trsv_upper(self.leaf, b)
        h = self.n // 2
        x = np.zeros_like(b)
        x[h:] = self.f22.solve_upper(b[h:])
        b[:h] -= self.f12.apply(x[h:])
        x[:h] = self.f11.solve_upper(b[:h])
        return x

    def solve_lower_adjoint(self, b):
        """x = L~^{-H} b: L~^H is unit upper; sweep right to left with F21^H."""
        b = np.array(b, dtype=np.complex128, copy=True)
        if self.leaf is not None:
            return _trsv_upper_unit_conj(self.leaf, b)
        h = self.n // 2
        x = np.zeros_like(b)
        x[h:] = self.f22.solve_lower_adjoint(b[h:])
        b[:h] -= self.f21.apply_adjoint(x[h:])
        x[:h] = self.f11.solve_lower_adjoint(b[:h])
        return x

    def solve_upper_adjoint(self, b):
        """x = U~^{-H} b: U~^H is lower; sweep left to right with F12^H."""
        b = np.array(b, dtype=np.complex128, copy=True)
        if self.leaf is not None:
            return _trsv_lower_conj(self.leaf, b)
        h = self.n // 2
        x = np.zeros_like(b)
        x[:h] = self.f11.solve_upper_adjoint(b[:h])
        b[h:] -= self.f12.apply_adjoint(x[:h])
        x[h:] = self.f22.solve_upper_adjoint(b[h:])
        return x

    def precond(self, b, adjoint=False):
        """M^{-1} b = U~^{-1} L~^{-1} b; adjoint: L~^{-H} U~^{-H} b."""
        if adjoint:
            return self.solve_lower_adjoint(self.solve_upper_adjoint(b))
        return self.solve_upper(self.solve_lower(b))

    def dense(self):
        return self.apply(np.eye(self.n, dtype=np.complex128))


def _trsv_lower_unit(a, b):
    n = a.shape[0]
    x = np.array(b, copy=True)
    for i in range(n):
        x[i] -= a[i, :i] @ x[:i]
    return x


def _trsv_upper(a, b):
    n = a.shape[0]
    x = np.array(b, copy=True)
    for i in range(n - 1, -1, -1):
        x[i] = (x[i] - a[i, i + 1:] @ x[i + 1:]) / a[i, i]
    return x


def _trsv_upper_unit_conj(a, b):
    """Solve (unit lower part of a)^H x = b."""
    n = a.shape[0]
    x = np.array(b, copy=True)
    for i in range(n - 1, -1, -1):
        x[i] -= a[i + 1:, i].conj() @ x[i + 1:]
    return x


def _trsv_lower_conj(a, b):
    """Solve (upper part of a incl. diagonal)^H x = b."""
    n = a.shape[0]
    x = np.array(b, copy=True)
    for i in range(n):
        x[i] = (x[i] - a[:i, i].conj() @ x[:i]) / np.conj(a[i, i])
    return x
