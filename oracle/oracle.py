"""ctypes front end of the FP64 CPU oracle (tdbem_oracle.c).

TEST INFRASTRUCTURE: only the test suite, `__graft_entry__.smoke()` and the
CPU-baseline leg of `bench.py` import this module. It never imports the CUDA
package, and the CUDA package never imports it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "tdbem_oracle.c")
_LIB = os.path.join(_HERE, "_tdbem_oracle.so")
_lib = None

f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")
i64p = np.ctypeslib.ndpointer(np.int64, flags="C_CONTIGUOUS")
i32p = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")


def compile_library(src: str, out: str) -> str:
    """gcc -O2 -fopenmp of one oracle source file into a shared library."""
    subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fopenmp", "-fPIC", "-shared", "-o", out, src, "-lm"])
    return out


def build(force: bool = False) -> str:
    """Compile the oracle next to its source (when the source is newer)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        compile_library(_SRC, tmp)
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    """The oracle library. TDBEM_ORACLE_LIB names a prebuilt copy to load
    instead (the mutation tests point it at a copy with a planted mistake)."""
    global _lib
    if _lib is None:
        path = os.environ.get("TDBEM_ORACLE_LIB")
        if not path:
            path = build()
        L = C.CDLL(path)
        L.or_create.restype = C.c_void_p
        L.or_create.argtypes = [f64p, C.c_int64, i32p, C.c_int64, f64p, C.c_int64,
                                C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]
        L.or_destroy.argtypes = [C.c_void_p]
        L.or_num_blocks.restype = C.c_int64
        L.or_num_blocks.argtypes = [C.c_void_p]
        L.or_block.argtypes = [C.c_void_p, C.c_int64, i32p, f64p]
        L.or_diam.restype = C.c_double
        L.or_diam.argtypes = [C.c_void_p]
        L.or_tri_geom.argtypes = [C.c_void_p, C.c_int64, f64p]
        L.or_set_first_kind.argtypes = [C.c_void_p, C.c_int]
        L.or_step.argtypes = [C.c_int, C.c_double, f64p]
        L.or_basis.argtypes = [C.c_void_p, C.c_int, C.c_int, f64p, C.c_int64, f64p]
        L.or_mu.argtypes = [C.c_void_p, C.c_int, f64p, C.c_int64, f64p]
        L.or_psi.argtypes = [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_int, f64p, C.c_int64, f64p]
        L.or_psi_block.argtypes = [C.c_void_p, C.c_int64, f64p, C.c_int64, f64p]
        L.or_tri_bounds.argtypes = [C.c_void_p, C.c_int64, C.c_int64, f64p]
        L.or_rule7.argtypes = [f64p, f64p]
        L.or_ss_rule.restype = C.c_int64
        L.or_ss_rule.argtypes = [C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]
        L.or_gauss_legendre.argtypes = [C.c_int, f64p, f64p]
        L.or_pair_local.argtypes = [C.c_void_p, C.c_int64, C.c_int64, i64p, C.c_int, C.c_int, C.c_int, f64p]
        L.or_pattern_counts.argtypes = [C.c_void_p, i64p, C.c_int64, i64p, C.c_int64, i64p]
        L.or_pattern_hash.argtypes = [C.c_void_p, i64p, C.c_int64, i64p, C.c_int64,
                                      np.ctypeslib.ndpointer(np.uint64, flags="C_CONTIGUOUS"), i64p]
        L.or_assemble_rows.argtypes = [C.c_void_p, i64p, C.c_int64, i64p, C.c_int64, i64p, i32p, f64p, f64p]
        L.or_num_threads.restype = C.c_int
        L.or_set_threads.restype = C.c_int
        L.or_set_threads.argtypes = [C.c_int]
        _lib = L
    return _lib


def gauss_legendre(n):
    x = np.zeros(n)
    w = np.zeros(n)
    lib().or_gauss_legendre(n, x, w)
    return x, w


def rule7():
    b = np.zeros(21)
    w = np.zeros(7)
    lib().or_rule7(b, w)
    return b.reshape(7, 3), w


def ss_rule(kase, n):
    L = lib()
    cnt = L.or_ss_rule(kase, n, None, None, None)
    xh = np.zeros(2 * cnt)
    yh = np.zeros(2 * cnt)
    w = np.zeros(cnt)
    L.or_ss_rule(kase, n, xh.ctypes.data, yh.ctypes.data, w.ctypes.data)
    return xh.reshape(-1, 2), yh.reshape(-1, 2), w


def num_threads():
    return lib().or_num_threads()


def set_threads(n):
    """OpenMP thread count of later oracle calls; returns the previous one."""
    return lib().or_set_threads(int(n))


# ---------------------------------------------------------------- data g --
# Neumann data g(x, t) of the boundary integral equation W phi = g (Eq. BIE),
# by kind:
#   0  plane wave u_inc = exp(-(t - x.d - c)^2 / (2 w^2)), params (dx, dy, dz,
#      c, w): g = -d/dn u_inc = (d.n) f'(t - x.d), the sound-hard condition
#   1  g(t) Y_0^0 with g(t) = sin(3t) t^2 exp(-t) (Sec. 6.1, first test)
#   2  g(t) Y_1^0(x) with g(t) = sin(2 pi t) t^3 exp(-2t) (Sec. 6.1, second)
Y00 = 1.0 / np.sqrt(4.0 * np.pi)
Y10 = np.sqrt(3.0 / (4.0 * np.pi))


def g_time(kind, t):
    t = np.asarray(t, dtype=np.float64)
    if kind == 1:
        return np.where(t > 0, np.sin(3 * t) * t * t * np.exp(-t), 0.0)
    if kind == 2:
        return np.where(t > 0, np.sin(2 * np.pi * t) * t ** 3 * np.exp(-2 * t), 0.0)
    raise ValueError(kind)


def g_data(kind, params, x, n, t):
    """g at points x (..., 3) with unit normals n (..., 3) and times t (T,):
    array (..., T)."""
    x = np.asarray(x, dtype=np.float64)
    t = np.asarray(t, dtype=np.float64)
    if kind == 0:
        d = np.asarray(params[:3], dtype=np.float64)
        c, w = float(params[3]), float(params[4])
        s = t[None, :] - (x.reshape(-1, 3) @ d)[:, None] - c
        fp = -s / (w * w) * np.exp(-0.5 * (s / w) ** 2)
        dn = n.reshape(-1, 3) @ d
        return (dn[:, None] * fp).reshape(x.shape[:-1] + (t.size,))
    if kind == 1:
        return np.broadcast_to(Y00 * g_time(1, t), x.shape[:-1] + (t.size,)).copy()
    if kind == 2:
        return (Y10 * x[..., 2])[..., None] * g_time(2, t)
    raise ValueError(kind)


class Oracle:
    """FP64 CPU oracle bound to one mesh and time grid.

    psi_mode: "direct" (1-D Gauss quadrature per evaluation) or "interp"
    (the oracle's own barycentric interpolant, sampled from the direct mode).
    """

    def __init__(self, verts, tris, t, p=0, equidistant=True, gl_n=32, gl_sub=4,
                 ss_n=4, psi_mode="interp", interp_S=8, interp_n=32, basis_kind=0):
        self.V = np.ascontiguousarray(verts, dtype=np.float64)
        self.F = np.ascontiguousarray(tris, dtype=np.int32)
        self.t = np.ascontiguousarray(t, dtype=np.float64)
        self.p = p
        self.equidistant = bool(equidistant)
        mode = {"direct": 0, "interp": 1}[psi_mode]
        # basis_kind: smooth step of the time basis, 0 erf(2 artanh x) (Sec. 3),
        # 1 built from exp(-1/s)
        self.h = lib().or_create(self.V, self.V.shape[0], self.F, self.F.shape[0], self.t, self.t.shape[0],
                                 p, int(equidistant), gl_n, gl_sub, ss_n, mode, interp_S, interp_n,
                                 int(basis_kind))

    def __del__(self):
        if getattr(self, "h", None):
            lib().or_destroy(self.h)
            self.h = None

    @property
    def M(self):
        return self.V.shape[0]

    @property
    def E(self):
        return self.F.shape[0]

    @property
    def N(self):
        return self.t.shape[0]

    def num_blocks(self):
        return lib().or_num_blocks(self.h)

    def blocks(self):
        """list of (kb, ib, m2, m1, a, b): 0-based test/trial time index,
        temporal orders and the support [a, b] of psi on r >= 0."""
        out = []
        for b in range(self.num_blocks()):
            q = np.zeros(4, np.int32)
            ab = np.zeros(2)
            lib().or_block(self.h, b, q, ab)
            out.append((int(q[0]), int(q[1]), int(q[2]), int(q[3]), float(ab[0]), float(ab[1])))
        return out

    def diam(self):
        return lib().or_diam(self.h)

    def tri_geom(self, e):
        """(unit normal, area, 3x3 surface curls of the corner hat functions)"""
        out = np.zeros(13)
        lib().or_tri_geom(self.h, e, out)
        return out[:3], out[3], out[4:].reshape(3, 3)

    def set_first_kind(self, kind):
        lib().or_set_first_kind(self.h, kind)

    def basis(self, ib, m, s):
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.zeros((s.size, 3))
        lib().or_basis(self.h, ib, m, s, s.size, out)
        return out

    def mu(self, ib, s):
        s = np.ascontiguousarray(s, dtype=np.float64)
        out = np.zeros((s.size, 3))
        lib().or_mu(self.h, ib, s, s.size, out)
        return out

    def psi(self, kb, ib, r, m2=0, m1=0):
        """direct (psi, psi~) of test basis kb against trial basis ib at r"""
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.zeros((r.size, 2))
        lib().or_psi(self.h, kb, m2, ib, m1, r, r.size, out)
        return out

    def psi_block(self, blk, r):
        r = np.ascontiguousarray(r, dtype=np.float64)
        out = np.zeros((r.size, 2))
        lib().or_psi_block(self.h, blk, r, r.size, out)
        return out

    def tri_bounds(self, s, q):
        out = np.zeros(2)
        lib().or_tri_bounds(self.h, s, q, out)
        return out

    def pair_local(self, s, q, blks, far_n=0, near_n=0):
        blks = np.ascontiguousarray(blks, dtype=np.int64)
        L = np.zeros(9 * blks.size)
        lib().or_pair_local(self.h, s, q, blks, blks.size, far_n, near_n, L)
        return L.reshape(blks.size, 3, 3)

    def pattern_counts(self, rows, blks):
        """Structural entries of rows `rows` in blocks `blks`: (nb, nr) int64."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        blks = np.ascontiguousarray(blks, dtype=np.int64)
        counts = np.zeros(rows.size * blks.size, np.int64)
        lib().or_pattern_counts(self.h, rows, rows.size, blks, blks.size, counts)
        return counts.reshape(blks.size, rows.size)

    def pattern_hash(self, blks, rows=None):
        """Fingerprint of the patterns of blocks `blks` over rows `rows` (all
        rows by default): (hash uint64[nb], nnz int64[nb]), hash the sum mod
        2^64 of splitmix64(l M + j) over the entries (l, j)."""
        rows = np.arange(self.M, dtype=np.int64) if rows is None else np.ascontiguousarray(rows, dtype=np.int64)
        blks = np.ascontiguousarray(blks, dtype=np.int64)
        hs = np.zeros(blks.size, np.uint64)
        nz = np.zeros(blks.size, np.int64)
        lib().or_pattern_hash(self.h, rows, rows.size, blks, blks.size, hs, nz)
        return hs, nz

    def assemble_rows(self, rows, blks):
        """Rows `rows` of blocks `blks`: dict blk -> list over rows of
        (cols int32, far float64, near float64)."""
        rows = np.ascontiguousarray(rows, dtype=np.int64)
        blks = np.ascontiguousarray(blks, dtype=np.int64)
        nr, nb = rows.size, blks.size
        counts = np.zeros(nr * nb, np.int64)
        lib().or_pattern_counts(self.h, rows, nr, blks, nb, counts)
        offs = np.zeros(nr * nb + 1, np.int64)
        offs[1:] = np.cumsum(counts)
        tot = int(offs[-1])
        cols = np.zeros(max(tot, 1), np.int32)
        vf = np.zeros(max(tot, 1))
        vn = np.zeros(max(tot, 1))
        lib().or_assemble_rows(self.h, rows, nr, blks, nb, offs, cols, vf, vn)
        out = {}
        for bi, b in enumerate(blks):
            lst = []
            for ri in range(nr):
                a, e = offs[bi * nr + ri], offs[bi * nr + ri + 1]
                lst.append((cols[a:e].copy(), vf[a:e].copy(), vn[a:e].copy()))
            out[int(b)] = lst
        return out

    def block_source(self, kb, ib, m2=0, m1=0):
        """Listed block that holds block (kb, ib) of the whole matrix
        (0-based time indices, Eq. Apartitioned) for test order m2 and trial
        order m1, or None for a zero block.

        Without the equidistant reduction every nonzero block is listed. On an
        equidistant grid the list holds the first two block columns, the last
        block row and the blocks (1, 2) and (N-2, N-1); every other block with
        both indices in the inner range 1..N-2 is, by Eq. relationAtildeBlock,
        block (k - i + 1, 1) when k >= i and block (1, 2) when k = i - 1, and
        is zero above that (Hessenberg, Eq. Apartitioned). Blocks cut by the
        diam criterion (Sec. 5.1) are absent from the list and zero."""
        if not hasattr(self, "_bidx"):
            self._bidx = {b[:4]: n for n, b in enumerate(self.blocks())}
        N = self.N
        key = (kb, ib)
        if self.equidistant and 1 <= kb <= N - 2 and 1 <= ib <= N - 2:
            d = kb - ib
            if d >= 0:
                key = (d + 1, 1)
            elif d == -1:
                key = (1, 2)
            else:
                return None
        return self._bidx.get(key + (m2, m1))

    @property
    def L(self):
        """Number of time basis functions, N (p + 1) (Sec. 3)."""
        return self.N * (self.p + 1)

    def hessenberg_apply(self, x, rows=None):
        """y = A x for the whole space-time system (Eq. Apartitioned): x and y
        are (L, M) arrays, L = N (p + 1), row kb (p + 1) + m the coefficients
        of time basis function b_{kb, m} (the numbering of Sec. 3 with 0-based
        indices; for p = 0 row k is time function k): x of the trial, y of
        the test functions. With `rows` given, only the columns y[:, rows]
        are computed (the rest stay zero). Every block comes from the listed
        blocks through block_source."""
        x = np.asarray(x, dtype=np.float64)
        N, M, P = self.N, self.M, self.p + 1
        rows = np.arange(M) if rows is None else np.asarray(rows, dtype=np.int64)
        nb = self.num_blocks()
        R = self.assemble_rows(rows, np.arange(nb))
        y = np.zeros((N * P, M))
        for kb in range(N):
            for ib in range(N):
                for m2 in range(P):
                    for m1 in range(P):
                        b = self.block_source(kb, ib, m2, m1)
                        if b is None:
                            continue
                        for r, (c, f, n) in enumerate(R[b]):
                            y[kb * P + m2, rows[r]] += np.dot(f + n, x[ib * P + m1, c])
        return y

    def rhs(self, kind, params=(), nt=16, sub=4):
        """Right-hand side g_k(l) = int_0^T int_Gamma g(x,t) phi_l(x)
        bdot_k(t) dGamma dt of the linear system (Sec. 3, Eq. of the
        partitioned system), as an (N, M) array: the 7-point rule on every
        triangle in space, composite Gauss-Legendre in time on every
        [t_j, t_{j+1}] (the breakpoints of every bdot_k), `sub` panels of
        `nt` points each. Shape (L, M), row k (p + 1) + m for b_{k, m}."""
        bary, w7 = rule7()
        P = self.V[self.F]                                     # (E, 3, 3)
        X = np.einsum("pa,eaj->epj", bary, P)                  # (E, 7, 3)
        cr = np.cross(P[:, 1] - P[:, 0], P[:, 2] - P[:, 0])
        area = 0.5 * np.linalg.norm(cr, axis=1)
        nrm = cr / (2.0 * area[:, None])
        xg, wg = gauss_legendre(nt)
        t = self.t
        s_list, w_list = [], []
        for j in range(t.size - 1):
            h = (t[j + 1] - t[j]) / sub
            for q in range(sub):
                a0 = t[j] + q * h
                s_list.append(a0 + h * xg)
                w_list.append(h * wg)
        s_n = np.concatenate(s_list)
        w_n = np.concatenate(w_list)
        G = g_data(kind, params, X, np.repeat(nrm[:, None, :], 7, axis=1), s_n)  # (E, 7, Ns)
        P = self.p + 1
        out = np.zeros((self.N * P, self.M))
        coef = area[:, None, None] * w7[None, :, None] * bary[None, :, :]     # (E, 7, 3)
        for k in range(self.N):
            for m in range(P):
                bd = self.basis(k, m, s_n)[:, 1]
                H = G @ (w_n * bd)                              # (E, 7)
                contrib = np.einsum("ep,epa->ea", H, coef)      # (E, 3)
                np.add.at(out[k * P + m], self.F.ravel(), contrib.ravel())
        return out

    def full_matrix(self):
        """The whole space-time matrix (L M x L M, L = N (p + 1)) of Eq.
        Apartitioned, block (k, i) of orders (m2, m1) at rows
        (k (p + 1) + m2) M.., columns (i (p + 1) + m1) M.., from the listed
        blocks through block_source (small cases only)."""
        N, M, P = self.N, self.M, self.p + 1
        nb = self.num_blocks()
        R = self.assemble_rows(np.arange(M), np.arange(nb))
        D = []
        for b in range(nb):
            B = np.zeros((M, M))
            for l, (c, f, n) in enumerate(R[b]):
                B[l, c] = f + n
            D.append(B)
        A = np.zeros((N * P * M, N * P * M))
        for kb in range(N):
            for ib in range(N):
                for m2 in range(P):
                    for m1 in range(P):
                        b = self.block_source(kb, ib, m2, m1)
                        if b is not None:
                            r0, c0 = (kb * P + m2) * M, (ib * P + m1) * M
                            A[r0:r0 + M, c0:c0 + M] = D[b]
        return A

    def solve_dense(self, g):
        """alpha with A alpha = g by dense LU (numpy), shapes (L, M)."""
        A = self.full_matrix()
        return np.linalg.solve(A, np.asarray(g, dtype=np.float64).ravel()).reshape(self.L, self.M)

    def dense_block(self, blk):
        """The whole block as a dense M x M array (far + near), row = test vertex."""
        res = self.assemble_rows(np.arange(self.M), [blk])[int(blk)]
        A = np.zeros((self.M, self.M))
        for l, (c, f, n) in enumerate(res):
            A[l, c] = f + n
        return A

    def double_layer(self, alpha, X, times, n=8):
        """Retarded double layer potential u = D phi (Eq. RetardedPotential)
        of the density phi(y, s) = sum_{k,m,j} alpha[k (p + 1) + m, j]
        b_{k,m}(s) phi_j(y) at points X (P, 3) off the surface and times
        `times`:

            u(x, t) = -1/(4 pi) int_Gamma n_y.(x - y)/|x - y|
                      [phi(y, t - |x - y|)/|x - y|^2
                       + d_t phi(y, t - |x - y|)/|x - y|] dGamma_y,

        integrated over every flat triangle by a collapsed Gauss product rule
        with n points per direction ((u, v) -> barycentric (1 - u, u (1 - v),
        u v), weight 2 u w_u w_v |T|). Returns an array (P, len(times))."""
        alpha = np.asarray(alpha, dtype=np.float64)
        P1 = self.p + 1
        assert alpha.shape == (self.N * P1, self.M)
        X = np.atleast_2d(np.asarray(X, dtype=np.float64))
        times = np.atleast_1d(np.asarray(times, dtype=np.float64))
        g, w = gauss_legendre(n)
        uu, vv = np.meshgrid(g, g, indexing="ij")
        lam = np.stack([1.0 - uu, uu * (1.0 - vv), uu * vv], axis=-1).reshape(-1, 3)   # (Q, 3)
        wq = (2.0 * uu * w[:, None] * w[None, :]).ravel()                               # (Q,)
        Pt = self.V[self.F]                                                             # (E, 3, 3)
        cr = np.cross(Pt[:, 1] - Pt[:, 0], Pt[:, 2] - Pt[:, 0])
        area = 0.5 * np.linalg.norm(cr, axis=1)
        nrm = cr / (2.0 * area[:, None])
        Y = np.einsum("qa,ead->eqd", lam, Pt)                                           # (E, Q, 3)
        W = area[:, None] * wq[None, :]                                                 # (E, Q)
        coef = np.einsum("qa,lea->leq", lam, alpha[:, self.F])                          # (L, E, Q)
        out = np.zeros((X.shape[0], times.size))
        for ip, x in enumerate(X):
            d = x[None, None, :] - Y
            r = np.sqrt(np.einsum("eqd,eqd->eq", d, d))
            kern = np.einsum("ed,eqd->eq", nrm, d) / r * W                              # n_y.(x-y)/r dGamma
            for it, t in enumerate(times):
                s = (t - r).ravel()
                phi = np.zeros(s.size)
                dphi = np.zeros(s.size)
                for k in range(self.N):
                    for m in range(P1):
                        b = self.basis(k, m, s)
                        c = coef[k * P1 + m].ravel()
                        phi += c * b[:, 0]
                        dphi += c * b[:, 1]
                integrand = kern.ravel() * (phi / r.ravel() ** 2 + dphi / r.ravel())
                out[ip, it] = -np.sum(integrand) / (4.0 * np.pi)
        return out
