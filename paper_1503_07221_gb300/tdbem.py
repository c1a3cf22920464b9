"""Python binding of libtdbem (argument marshalling only).

Every function forwards to the C ABI declared in include/tdbem.h; all
computation runs in the CUDA library. PyTorch supplies device memory (its
caching allocator is registered as libtdbem's allocator) and the current CUDA
stream. Loading fails loudly when the library has not been built.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libtdbem.so")

OK = 0
RHS_PLANE_WAVE, RHS_SPHERE_N0, RHS_SPHERE_N1 = 0, 1, 2
E_INVALID_ARG, E_MESH, E_TIMEGRID, E_OOM, E_CUDA, E_DEVICE, E_NOT_ASSEMBLED, E_UNSUPPORTED, E_NUMERIC = range(1, 10)
LAST_BLOCK = -1
PREC_FP64 = 0
PREC_MIXED = 1
FAR = 0
NEAR = 1


class TdbemError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__("libtdbem error %d: %s" % (code, msg))
        self.code = code


class Opts(C.Structure):
    _fields_ = [("precision", C.c_int32), ("near_order", C.c_int32), ("cheb_degree", C.c_int32),
                ("staging_mb", C.c_int32), ("reserved", C.c_int32 * 4)]


class Stats(C.Structure):
    _fields_ = [("n_blocks", C.c_int64), ("nnz", C.c_int64), ("nnz_near", C.c_int64),
                ("far_pairs", C.c_int64), ("near_pairs", C.c_int64), ("quad_points", C.c_int64),
                ("ms_total", C.c_double), ("ms_pattern", C.c_double), ("ms_far", C.c_double),
                ("ms_near", C.c_double), ("ms_extract", C.c_double), ("kernel_launches", C.c_int64),
                ("graph_replays", C.c_int64), ("matvec_variant", C.c_int64), ("quad_points_far", C.c_int64),
                ("matvec_launches", C.c_int64)]


_ALLOC = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p, C.c_void_p)
_FREE = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p, C.c_void_p)
_lib = None
_cb = None


def lib():
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libtdbem.so is not built (run __graft_entry__.build())")
    L = C.CDLL(LIB_PATH)
    vp, i64, i32 = C.c_void_p, C.c_int64, C.c_int32
    L.tdbem_last_error.restype = C.c_char_p
    L.tdbem_set_allocator.argtypes = [_ALLOC, _FREE, vp]
    L.tdbem_mesh_create.argtypes = [vp, i64, vp, i64, C.POINTER(vp)]
    L.tdbem_timegrid_create.argtypes = [vp, i64, i32, i32, C.c_double, C.POINTER(vp)]
    L.tdbem_assembler_create.argtypes = [vp, vp, C.POINTER(Opts), vp, C.POINTER(vp)]
    L.tdbem_num_blocks.argtypes = [vp, C.POINTER(i64)]
    L.tdbem_block_info.argtypes = [vp, i64, C.POINTER(i32), C.POINTER(i32), C.POINTER(i32), C.POINTER(i32),
                                   C.POINTER(i64), C.POINTER(i64)]
    L.tdbem_assemble_all.argtypes = [vp, vp]
    L.tdbem_assemble_block.argtypes = [vp, i32, i32, vp]
    L.tdbem_block_csr.argtypes = [vp, i64, i32, C.POINTER(vp), C.POINTER(vp), C.POINTER(vp), C.POINTER(i64)]
    L.tdbem_block_csr_host.argtypes = [vp, i64, i32, vp, vp, vp]
    L.tdbem_hessenberg_apply.argtypes = [vp, vp, vp, vp]
    L.tdbem_hessenberg_apply_noalloc.argtypes = [vp, vp, vp, vp]
    L.tdbem_rhs_assemble.argtypes = [vp, i32, vp, i32, vp, vp]
    L.tdbem_double_layer.argtypes = [vp, vp, vp, i64, vp, i32, i32, vp, vp]
    L.tdbem_psi_table.argtypes = [vp, i64, i32, vp, i64, vp, vp]
    L.tdbem_solve_gmres.argtypes = [vp, vp, vp, i32, C.c_double, i32, C.POINTER(i32), C.POINTER(C.c_double), vp]
    L.tdbem_solve_dgmres.argtypes = [vp, vp, vp, i32, i32, i32, C.c_double, i32, C.POINTER(i32),
                                     C.POINTER(C.c_double), C.POINTER(i32), vp]
    L.tdbem_deflation_basis.argtypes = [vp, i32, i32, i32, vp, C.POINTER(i32), C.POINTER(C.c_double)]
    L.tdbem_solve_fgmres.argtypes = [vp, vp, vp, i32, C.c_double, i32, i32, vp, C.POINTER(i32),
                                     C.POINTER(C.c_double), vp]
    L.tdbem_precond_apply.argtypes = [vp, i32, vp, C.c_double, vp, vp, vp]
    L.tdbem_measure_fma_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double), vp]
    L.tdbem_stats.argtypes = [vp, C.POINTER(Stats)]
    L.tdbem_mesh_destroy.argtypes = [vp]
    L.tdbem_timegrid_destroy.argtypes = [vp]
    L.tdbem_asm_destroy.argtypes = [vp]
    L.tdbem_mesh_destroy.restype = None
    L.tdbem_timegrid_destroy.restype = None
    L.tdbem_asm_destroy.restype = None
    _lib = L
    return L


def exported_symbols():
    """Names of the C entry points this binding expects."""
    return ["tdbem_last_error", "tdbem_set_allocator", "tdbem_mesh_create", "tdbem_timegrid_create",
            "tdbem_assembler_create", "tdbem_num_blocks", "tdbem_block_info", "tdbem_assemble_all",
            "tdbem_block_csr", "tdbem_block_csr_host", "tdbem_stats", "tdbem_mesh_destroy",
            "tdbem_timegrid_destroy", "tdbem_asm_destroy"]


def _check(code):
    if code != OK:
        raise TdbemError(code, lib().tdbem_last_error().decode())


def use_torch_allocator():
    """Route libtdbem's device allocations through torch's caching allocator.

    Idempotent: the callbacks are created once and kept alive for the life of
    the process, because every device buffer remembers the free callback it
    was allocated with."""
    global _cb
    if _cb is not None:
        return
    import torch

    def alloc(n, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(n))
        except Exception:
            return None

    def free(p, stream, ctx):
        torch.cuda.caching_allocator_delete(p)

    _cb = (_ALLOC(alloc), _FREE(free))
    _check(lib().tdbem_set_allocator(_cb[0], _cb[1], None))


def _stream(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return int(stream)


def deflation_basis(H, l):
    """Host-only (no device): (B, lam_max) for the square upper Hessenberg H
    (m x m, m <= 62): B (m, sdim) an orthonormal real basis of the invariant
    subspace of H for its eigenvalues of modulus at most the l-th smallest,
    lam_max the largest eigenvalue modulus (tdbem_deflation_basis)."""
    import numpy as np
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = H.shape[0]
    B = np.zeros((m, m))
    sd, lm = C.c_int32(), C.c_double()
    _check(lib().tdbem_deflation_basis(C.c_void_p(H.ctypes.data), m, m, int(l), C.c_void_p(B.ctypes.data),
                                       C.byref(sd), C.byref(lm)))
    return B[:, :sd.value].copy(), lm.value


def measure_fma_peaks(stream=None):
    """(FP32 packed-FMA, FP64 FMA) throughput of the current device, TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(lib().tdbem_measure_fma_peaks(C.byref(a), C.byref(b), C.c_void_p(_stream(stream))))
    return a.value, b.value


class Mesh:
    def __init__(self, verts, tris):
        V = np.ascontiguousarray(verts, dtype=np.float64)
        F = np.ascontiguousarray(tris, dtype=np.int32)
        h = C.c_void_p()
        _check(lib().tdbem_mesh_create(V.ctypes.data, V.shape[0], F.ctypes.data, F.shape[0], C.byref(h)))
        self.h = h
        self.M, self.E = V.shape[0], F.shape[0]

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tdbem_mesh_destroy(self.h)
            self.h = None


class TimeGrid:
    def __init__(self, t, p=0, basis_kind=0, c=1.0):
        t = np.ascontiguousarray(t, dtype=np.float64)
        h = C.c_void_p()
        _check(lib().tdbem_timegrid_create(t.ctypes.data, t.size, p, basis_kind, c, C.byref(h)))
        self.h = h
        self.N = t.size
        self.p = int(p)
        self.L = self.N * (self.p + 1)  # time functions: rows of x and y

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tdbem_timegrid_destroy(self.h)
            self.h = None


class Assembler:
    """Unique blocks of the block-Hessenberg system of one mesh and time grid."""

    def __init__(self, mesh: Mesh, grid: TimeGrid, precision=PREC_MIXED, near_order=4, stream=None, staging_mb=0):
        o = Opts()
        o.precision = precision
        o.near_order = near_order
        o.staging_mb = staging_mb
        o.cheb_degree = 32
        h = C.c_void_p()
        _check(lib().tdbem_assembler_create(mesh.h, grid.h, C.byref(o), C.c_void_p(_stream(stream)), C.byref(h)))
        self.h = h
        self.mesh, self.grid = mesh, grid
        self.precision = precision

    def __del__(self):
        if getattr(self, "h", None) and _lib is not None:
            _lib.tdbem_asm_destroy(self.h)
            self.h = None

    def assemble(self, stream=None):
        _check(lib().tdbem_assemble_all(self.h, C.c_void_p(_stream(stream))))

    def assemble_block(self, k, i, stream=None):
        """Block (k, i) on its own; read it back with b = LAST_BLOCK."""
        _check(lib().tdbem_assemble_block(self.h, k, i, C.c_void_p(_stream(stream))))

    def num_blocks(self):
        n = C.c_int64()
        _check(lib().tdbem_num_blocks(self.h, C.byref(n)))
        return n.value

    def block_info(self, b):
        k, i, m2, m1 = C.c_int32(), C.c_int32(), C.c_int32(), C.c_int32()
        nf, nn = C.c_int64(), C.c_int64()
        _check(lib().tdbem_block_info(self.h, b, C.byref(k), C.byref(i), C.byref(m2), C.byref(m1),
                                      C.byref(nf), C.byref(nn)))
        return dict(k=k.value, i=i.value, m2=m2.value, m1=m1.value, nnz_far=nf.value, nnz_near=nn.value)

    def blocks(self):
        return [(d["k"], d["i"]) for d in (self.block_info(b) for b in range(self.num_blocks()))]

    def block_csr_device(self, b, which=FAR):
        rp, col, val = C.c_void_p(), C.c_void_p(), C.c_void_p()
        nnz = C.c_int64()
        _check(lib().tdbem_block_csr(self.h, b, which, C.byref(rp), C.byref(col), C.byref(val), C.byref(nnz)))
        return rp.value, col.value, val.value, nnz.value

    def block_csr_torch(self, b, which=FAR):
        """(row_ptr, col, val) as zero-copy torch CUDA tensors over the
        library's borrowed device arrays (valid until the next assemble)."""
        import torch
        rp, col, val, nnz = self.block_csr_device(b, which)
        vt = "<f4" if (which == FAR and self.precision == PREC_MIXED) else "<f8"
        M = self.mesh.M

        def view(ptr, n, typestr):
            class _A:
                __cuda_array_interface__ = {"shape": (n,), "typestr": typestr, "data": (ptr, False), "version": 2}
            return torch.as_tensor(_A(), device="cuda") if n > 0 else torch.empty(0, device="cuda")

        return view(rp, M + 1, "<i8"), view(col, nnz, "<i4"), view(val, nnz, vt)

    def block_csr_host(self, b, which=FAR):
        """(row_ptr int64[M+1], col int32[nnz], val) copied to host."""
        info = self.block_info(b)
        nnz = info["nnz_far"] if which == FAR else info["nnz_near"]
        rp = np.zeros(self.mesh.M + 1, np.int64)
        col = np.zeros(max(nnz, 1), np.int32)
        vdt = np.float32 if (which == FAR and self.precision == PREC_MIXED) else np.float64
        val = np.zeros(max(nnz, 1), vdt)
        _check(lib().tdbem_block_csr_host(self.h, b, which, rp.ctypes.data, col.ctypes.data, val.ctypes.data))
        return rp, col[:nnz], val[:nnz]

    def hessenberg_apply(self, x, y=None, stream=None, noalloc=False):
        """y = A x over the whole block-Hessenberg matrix; x and y are
        contiguous float64 CUDA tensors of shape (N, M) (row = time index).
        noalloc=True calls tdbem_hessenberg_apply_noalloc (fixed scratch,
        N*M <= 2^21); y must then be given."""
        import torch
        shape = (self.grid.L, self.mesh.M)
        for name, v in (("x", x), ("y", y)):
            if v is not None and (tuple(v.shape) != shape or v.dtype != torch.float64 or not v.is_cuda
                                  or not v.is_contiguous()):
                raise ValueError("%s must be a contiguous float64 CUDA tensor of shape %s" % (name, shape))
        if y is None:
            if noalloc:
                raise ValueError("noalloc=True needs a caller-provided y")
            y = torch.empty_like(x)
        fn = lib().tdbem_hessenberg_apply_noalloc if noalloc else lib().tdbem_hessenberg_apply
        _check(fn(self.h, C.c_void_p(x.data_ptr()), C.c_void_p(y.data_ptr()), C.c_void_p(_stream(stream))))
        return y

    def rhs(self, kind, params=(), out=None, stream=None):
        """Right-hand side g_{k,m}(l) as a float64 CUDA tensor of shape (N (p + 1), M),
        row k (p + 1) + m."""
        import torch
        shape = (self.grid.L, self.mesh.M)
        if out is None:
            out = torch.empty(shape, dtype=torch.float64, device="cuda")
        p = np.ascontiguousarray(params, dtype=np.float64)
        _check(lib().tdbem_rhs_assemble(self.h, kind, p.ctypes.data if p.size else None, p.size,
                                        C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream))))
        return out

    def psi_table(self, b, r, which=0, stream=None):
        """The assembler's psi / psi~ table of unique block b at distances r
        (float64 CUDA tensor): (n, 2) float64 CUDA tensor; which 0 = FP64 set,
        1 = FP32 set."""
        import torch
        out = torch.empty((r.shape[0], 2), dtype=torch.float64, device="cuda")
        _check(lib().tdbem_psi_table(self.h, b, which, C.c_void_p(r.data_ptr()), r.shape[0],
                                     C.c_void_p(out.data_ptr()), C.c_void_p(_stream(stream))))
        return out

    def double_layer(self, alpha, X, times, n=8, out=None, stream=None):
        """Retarded double layer potential of the density alpha ((N, M)
        float64 CUDA tensor) at points X ((P, 3) float64 CUDA tensor) and
        times ((nt,) float64 CUDA tensor): (P, nt) float64 CUDA tensor."""
        import torch
        P, nt = X.shape[0], times.shape[0]
        if out is None:
            out = torch.empty((P, nt), dtype=torch.float64, device="cuda")
        _check(lib().tdbem_double_layer(self.h, C.c_void_p(alpha.data_ptr()), C.c_void_p(X.data_ptr()), P,
                                        C.c_void_p(times.data_ptr()), nt, n, C.c_void_p(out.data_ptr()),
                                        C.c_void_p(_stream(stream))))
        return out

    def solve(self, g, restart=50, tol=1e-10, max_iter=2000, stream=None):
        """alpha with A alpha = g by restarted GMRES on the device; returns
        (alpha, iterations, relative residual)."""
        import torch
        alpha = torch.empty_like(g)
        it, rr = C.c_int32(), C.c_double()
        _check(lib().tdbem_solve_gmres(self.h, C.c_void_p(g.data_ptr()), C.c_void_p(alpha.data_ptr()), restart, tol,
                                       max_iter, C.byref(it), C.byref(rr), C.c_void_p(_stream(stream))))
        return alpha, it.value, rr.value

    def solve_dgmres(self, g, restart=30, l=5, r=40, tol=1e-8, max_iter=2000, stream=None):
        """alpha with A alpha = g by DGMRES(restart, l) with at most r
        deflation vectors (Sec. 4.1); returns (alpha, iterations, true
        relative residual, columns of U at the end)."""
        import torch
        alpha = torch.empty_like(g)
        it, rr, nu = C.c_int32(), C.c_double(), C.c_int32()
        _check(lib().tdbem_solve_dgmres(self.h, C.c_void_p(g.data_ptr()), C.c_void_p(alpha.data_ptr()), restart, l, r,
                                        tol, max_iter, C.byref(it), C.byref(rr), C.byref(nu),
                                        C.c_void_p(_stream(stream))))
        return alpha, it.value, rr.value, nu.value

    def solve_fgmres(self, g, restart=50, tol=1e-5, max_iter=20000, inner=(10,), stream=None):
        """alpha with A alpha = g by FGMRES(restart, len(inner)(inner...)) with
        the recursive block-Hessenberg preconditioner (inner = (): no
        preconditioner); returns (alpha, outer iterations, true relative
        residual)."""
        import torch
        alpha = torch.empty_like(g)
        inn = (C.c_int32 * max(1, len(inner)))(*inner)
        it, rr = C.c_int32(), C.c_double()
        _check(lib().tdbem_solve_fgmres(self.h, C.c_void_p(g.data_ptr()), C.c_void_p(alpha.data_ptr()), restart, tol,
                                        max_iter, len(inner), inn if len(inner) else None, C.byref(it), C.byref(rr),
                                        C.c_void_p(_stream(stream))))
        return alpha, it.value, rr.value

    def precondition(self, r, inner=(10,), tol=1e-5, out=None, stream=None):
        """z = M^-1 r, one application of the recursive preconditioner with
        len(inner) levels."""
        import torch
        z = torch.empty_like(r) if out is None else out
        inn = (C.c_int32 * max(1, len(inner)))(*inner)
        _check(lib().tdbem_precond_apply(self.h, len(inner), inn if len(inner) else None, tol,
                                         C.c_void_p(r.data_ptr()), C.c_void_p(z.data_ptr()),
                                         C.c_void_p(_stream(stream))))
        return z

    def stats(self):
        s = Stats()
        _check(lib().tdbem_stats(self.h, C.byref(s)))
        return {f: getattr(s, f) for f, _ in Stats._fields_}
