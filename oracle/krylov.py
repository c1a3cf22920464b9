"""FP64 CPU oracle of the iterative solution of the block-Hessenberg system
A alpha = g (Sec. 4): restarted flexible GMRES, the recursive algebraic
block-Hessenberg preconditioner (Sec. 4.2, Algorithm 1) and restarted GMRES
preconditioned by deflation, DGMRES(m, l) (Sec. 4.1).

TEST INFRASTRUCTURE: only the test suite, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` import this module. It never imports the CUDA
package, and the CUDA package never imports it. Plain numpy on dense
matrices; small cases only.

Readings of Sec. 4.2 taken here (the paper leaves them open):
* FGMRES is Saad's flexible variant (the paper's reference for it): the
  preconditioned vectors z_j are kept and the iterate is x0 + Z_j y_j, so the
  preconditioner may change from one step to the next. Modified Gram-Schmidt
  Arnoldi; the small least-squares problem is solved by numpy's lstsq after
  every step, and its residual is the residual estimate.
* Splitting: a diagonal range [lo, hi) of block rows/columns (0-based) is cut
  at h = lo + ceil((hi - lo) / 2); the block (h - 1, h) above the diagonal at
  the cut is dropped (the paper's 1-based block (ceil(N/2), ceil(N/2) + 1)),
  leaving the block lower-triangular 2 x 2 matrix of Sec. 4.2.
* Levels: FGMRES(m, r(i_1, ..., i_r)) of the experiments (Sec. 6) means r
  levels. The outer solve is preconditioned by the level-1 splitting; the
  two half systems of a level-l splitting are solved by i_l steps of FGMRES,
  preconditioned by the level-(l + 1) splitting of the half when l < r and
  the half spans at least two blocks, unpreconditioned otherwise. Each inner
  solve is one cycle from zero with the solver's relative tolerance.
"""
from __future__ import annotations

import numpy as np


def fgmres(apply_A, b, m, tol, max_iter, prec=None):
    """Restarted flexible GMRES(m) for A x = b from x0 = 0.

    apply_A(v) returns A v, prec(v) an approximation of M^-1 v (it may change
    between calls; None is the identity). One iteration is one Arnoldi step:
    z_j = prec(v_j), w = A z_j, w orthogonalised against v_1..v_j in order
    (h_ij = (w, v_i), w -= h_ij v_i), h_{j+1,j} = |w|, v_{j+1} = w / h_{j+1,j}.
    After the step, y_j = argmin |beta e_1 - Hbar_j y| and the estimate of the
    residual norm is that minimum. A cycle ends after m steps, when the
    estimate reaches tol |b|, after max_iter steps in all, or at breakdown
    (h_{j+1,j} = 0); then x += Z_j y_j and the next cycle starts from the
    true residual b - A x, unless that already meets the tolerance.

    Returns (x, iterations, history): history holds |b - A x| / |b| at each
    restart (first entry: the start) and every step's estimate / |b|."""
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.size
    x = np.zeros(n)
    bn = float(np.linalg.norm(b))
    hist = []
    if bn == 0.0:
        return x, 0, [0.0]
    total = 0
    while True:
        r = b - apply_A(x)
        beta = float(np.linalg.norm(r))
        hist.append(beta / bn)
        if beta <= tol * bn or total >= max_iter:
            return x, total, hist
        V = np.zeros((m + 1, n))
        Z = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        V[0] = r / beta
        y = np.zeros(0)
        jdone = 0
        stop = False
        for j in range(m):
            Z[j] = V[j] if prec is None else prec(V[j])
            w = apply_A(Z[j])
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            rhs = np.zeros(j + 2)
            rhs[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], rhs, rcond=None)[0]
            est = float(np.linalg.norm(rhs - H[:j + 2, :j + 1] @ y))
            total += 1
            jdone = j + 1
            hist.append(est / bn)
            if est <= tol * bn or total >= max_iter or H[j + 1, j] == 0.0:
                stop = True
                break
        x = x + Z[:jdone].T @ y
        if stop:
            return x, total, hist


class RecursivePreconditioner:
    """z = M^-1 r for the block-Hessenberg matrix A (Sec. 4.2, Algorithm 1).

    A is dense (nblk bs, nblk bs) with bs x bs blocks. On a range [lo, hi)
    split at h (module docstring), M keeps the blocks of A except block
    (h - 1, h), so M^-1 r = (M11^-1 r1, M22^-1 (r2 - M21 M11^-1 r1)): the two
    diagonal systems are solved approximately by `inner[l - 1]` FGMRES steps
    at level l, recursively preconditioned up to level len(inner)."""

    def __init__(self, A, nblk, bs, inner, tol):
        self.A = np.asarray(A, dtype=np.float64)
        self.nblk, self.bs = int(nblk), int(bs)
        self.inner = tuple(int(i) for i in inner)
        self.tol = float(tol)
        assert self.A.shape == (self.nblk * self.bs, self.nblk * self.bs)
        assert len(self.inner) >= 1 and min(self.inner) >= 1

    def _sub(self, k0, k1, i0, i1):
        s = self.bs
        return self.A[k0 * s:k1 * s, i0 * s:i1 * s]

    def _half_solve(self, lo, hi, rhs, level):
        Ad = self._sub(lo, hi, lo, hi)
        prec = None
        if level < len(self.inner) and hi - lo >= 2:
            prec = lambda v: self.apply(v, lo, hi, level + 1)
        it = self.inner[level - 1]
        return fgmres(lambda v: Ad @ v, rhs, it, self.tol, it, prec)[0]

    def apply(self, r, lo=0, hi=None, level=1):
        """M^-1 r for the level-`level` splitting of block range [lo, hi);
        a range of one block cannot be split and is left as it is."""
        hi = self.nblk if hi is None else hi
        r = np.asarray(r, dtype=np.float64).ravel()
        assert r.size == (hi - lo) * self.bs
        if hi - lo < 2:
            return r.copy()
        h = lo + (hi - lo + 1) // 2
        n1 = (h - lo) * self.bs
        y1 = self._half_solve(lo, h, r[:n1], level)
        t = r[n1:] - self._sub(h, hi, lo, h) @ y1
        y2 = self._half_solve(h, hi, t, level)
        return np.concatenate([y1, y2])


def solve(A, nblk, bs, b, m, tol, max_iter, inner=()):
    """FGMRES(m, r(inner)) on the whole system: the recursive preconditioner
    with len(inner) levels, or none (plain GMRES(m)) for inner = ()."""
    A = np.asarray(A, dtype=np.float64)
    prec = None
    if len(inner) and nblk >= 2:
        P = RecursivePreconditioner(A, nblk, bs, inner, tol)
        prec = P.apply
    return fgmres(lambda v: A @ v, b, m, tol, max_iter, prec)


def deflation_inverse(apply_A, U, lam_max):
    """M^-1 of the deflation preconditioner (Sec. 4.1) for an orthonormal
    basis U (n, r) of an approximately invariant subspace:
    M^-1 = I + U (|lam_max| T^-1 - I_r) U^T with T = U^T A U. Returns a
    function v -> M^-1 v (and T)."""
    U = np.asarray(U, dtype=np.float64)
    if U.shape[1] == 0:
        return (lambda v: np.array(v, dtype=np.float64)), np.zeros((0, 0))
    AU = np.column_stack([apply_A(U[:, j]) for j in range(U.shape[1])])
    T = U.T @ AU
    Tinv = np.linalg.inv(T)
    lam = abs(float(lam_max))

    def apply(v):
        v = np.asarray(v, dtype=np.float64)
        c = U.T @ v
        return v + U @ (lam * (Tinv @ c) - c)
    return apply, T


def dgmres(apply_A, b, m, l, r, tol, max_iter):
    """DGMRES(m, l) of Sec. 4.1 for A x = b from x0 = 0: restarted GMRES(m)
    right-preconditioned by the deflation preconditioner M^-1 of
    `deflation_inverse`, fixed within a cycle. After every cycle the
    Schur decomposition H_m = S R S^T of the cycle's square Hessenberg
    matrix (of A M^-1) is sorted so that its eigenvalues of smallest modulus
    come first; the first l Schur vectors (l + 1 when the l-th closes a
    complex pair) give V_m S_l, which is orthonormalised against U (two
    Gram-Schmidt passes) and appended, until U has r columns. The largest
    modulus among the eigenvalues of H_m estimates |lambda_max|. l = 0 (or
    r = 0) is plain GMRES(m).

    Returns (x, iterations, history, U) with history as in fgmres."""
    import scipy.linalg as sla
    b = np.asarray(b, dtype=np.float64).ravel()
    n = b.size
    x = np.zeros(n)
    bn = float(np.linalg.norm(b))
    if bn == 0.0:
        return x, 0, [0.0], np.zeros((n, 0))
    U = np.zeros((n, 0))
    lam_max = 1.0
    prec = lambda v: np.array(v, dtype=np.float64)
    total, hist = 0, []
    while True:
        res = b - apply_A(x)
        beta = float(np.linalg.norm(res))
        hist.append(beta / bn)
        if beta <= tol * bn or total >= max_iter:
            return x, total, hist, U
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        V[0] = res / beta
        y = np.zeros(0)
        jdone, stop = 0, False
        for j in range(m):
            w = apply_A(prec(V[j]))
            for i in range(j + 1):
                H[i, j] = np.dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0.0:
                V[j + 1] = w / H[j + 1, j]
            rhs = np.zeros(j + 2)
            rhs[0] = beta
            y = np.linalg.lstsq(H[:j + 2, :j + 1], rhs, rcond=None)[0]
            est = float(np.linalg.norm(rhs - H[:j + 2, :j + 1] @ y))
            total += 1
            jdone = j + 1
            hist.append(est / bn)
            if est <= tol * bn or total >= max_iter or H[j + 1, j] == 0.0:
                stop = True
                break
        x = x + prec(V[:jdone].T @ y)
        if stop:
            return x, total, hist, U
        if l > 0 and U.shape[1] < r:
            Hm = H[:m, :m]
            ev = np.linalg.eigvals(Hm)
            lam_max = float(np.abs(ev).max())
            cut = np.sort(np.abs(ev))[min(l, m) - 1]
            R_, S, sdim = sla.schur(Hm, output="real", sort=lambda re, im: np.hypot(re, im) <= cut * (1 + 1e-12))
            W = V[:m].T @ S[:, :sdim]
            for k in range(W.shape[1]):
                if U.shape[1] >= r:
                    break
                u = W[:, k]
                for _ in range(2):
                    u = u - U @ (U.T @ u)
                nu = np.linalg.norm(u)
                if nu > 1e-10 * np.linalg.norm(W[:, k]):
                    U = np.column_stack([U, u / nu])
            prec, _ = deflation_inverse(apply_A, U, lam_max)
