// Flexible GMRES (Saad's FGMRES, the solver of Sec. 4.2) with the recursive
// algebraic block-Hessenberg preconditioner (Sec. 4.2, Algorithm 1).
//
// Splitting: a diagonal range [lo, hi) of block rows and columns is cut at
// h = lo + ceil((hi - lo) / 2); the preconditioner M drops the block
// (h - 1, h) above the diagonal at the cut, so
//   M^-1 r = (M11^-1 r1, M22^-1 (r2 - M21 M11^-1 r1)).
// The two diagonal systems are solved approximately by one FGMRES cycle of
// inner[l - 1] steps at level l, from zero and with the solver's relative
// tolerance, preconditioned by the level-(l + 1) splitting of the half while
// l < levels and the half spans two blocks or more. The outer solve is the
// restarted FGMRES(m) preconditioned by the level-1 splitting of the whole
// range (levels = 0: plain GMRES(m) through the same code).
//
// Device-resident iteration: the Hessenberg columns, Givens rotations,
// residual estimate and the stop decision of every solve live in a KState
// in device memory and are updated by single-thread kernels. Every kernel
// of a solve reads that solve's `run` flag and does nothing once it is
// zero, and an inner solve starts only if its caller is running. So the
// whole preconditioner application is one fixed launch sequence with no
// host round trip: it is recorded once per solve as a CUDA graph (fixed
// input and output vectors) and replayed at every outer step. The host
// reads back one small status record per outer step. All reductions are the
// fixed-order two-pass sums of solve.cu: repeated solves are bitwise equal.
#include <cstring>
#include <vector>

#include "tdbem_internal.h"

namespace tdbem {

__global__ void kr_begin_kernel(KState *s, const int *parent, int m, double tol, int set_ref) {
    const double beta = sqrt(s->r2);
    if (set_ref) {
        s->bref = beta;
        s->iters = 0;
    }
    const int on = (!parent || *parent) && beta > tol * s->bref;
    s->run = on;
    s->stop = on ? 0 : 1;
    s->jdone = 0;
    s->m = m;
    s->e[0] = beta;
    for (int i = 1; i <= m; ++i) s->e[i] = 0.0;
    s->inv = on ? 1.0 / beta : 0.0;
    s->resid = s->bref > 0.0 ? beta / s->bref : 0.0;
}

// v = w / |w| of the current step (or of the start residual; v may be w)
__global__ void kr_scale_kernel(const KState *__restrict__ s, const double *w, double *v, int64_t n) {
    if (!s->run) return;
    const double ib = s->inv;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = w[e] * ib;
}

// column j of the Hessenberg matrix from the two Gram-Schmidt passes, the
// earlier rotations on it, a new rotation that zeroes h_{j+1,j}, and the
// stop decision: residual estimate |e_{j+1}| <= tol |b|, breakdown
// (h_{j+1,j} = 0) or the last step of the cycle
__global__ void kr_step_kernel(KState *s, int j, double tol) {
    if (!s->run) return;
    constexpr int L = KR_MAXM;
    double *H = s->H;
    for (int i = 0; i <= j; ++i) H[i * L + j] = s->hc[i] + s->hc[GM_MAXV + i];
    const double hn = sqrt(s->w2);
    H[(j + 1) * L + j] = hn;
    for (int i = 0; i < j; ++i) {
        const double a = H[i * L + j], b = H[(i + 1) * L + j];
        H[i * L + j] = s->cs[i] * a + s->sn[i] * b;
        H[(i + 1) * L + j] = -s->sn[i] * a + s->cs[i] * b;
    }
    const double a = H[j * L + j], b = H[(j + 1) * L + j];
    const double rho = hypot(a, b);
    s->cs[j] = rho > 0.0 ? a / rho : 1.0;
    s->sn[j] = rho > 0.0 ? b / rho : 0.0;
    H[j * L + j] = rho;
    H[(j + 1) * L + j] = 0.0;
    s->e[j + 1] = -s->sn[j] * s->e[j];
    s->e[j] = s->cs[j] * s->e[j];
    s->jdone = j + 1;
    s->iters += 1;
    const double r = fabs(s->e[j + 1]);
    s->resid = s->bref > 0.0 ? r / s->bref : 0.0;
    const bool conv = r <= tol * s->bref || hn == 0.0;
    if (conv || j + 1 >= s->m) {
        s->run = 0;
        s->stop = conv ? 1 : 0;
    } else {
        s->inv = 1.0 / hn;
    }
}

// R y = e over the steps done (back substitution)
__global__ void kr_finish_kernel(KState *s) {
    constexpr int L = KR_MAXM;
    const int jd = s->jdone;
    for (int i = jd - 1; i >= 0; --i) {
        double v = s->e[i];
        for (int k = i + 1; k < jd; ++k) v -= s->H[i * L + k] * s->y[k];
        s->y[i] = s->H[i * L + i] != 0.0 ? v / s->H[i * L + i] : 0.0;
    }
}

// x = Z y (assign) or x += Z y over the steps done
__global__ void __launch_bounds__(256) kr_update_kernel(const KState *__restrict__ s, const double *__restrict__ Z,
                                                        int64_t ld, double *__restrict__ x, int64_t n, int assign) {
    __shared__ double ys[KR_MAXM];
    const int jd = s->jdone;
    if (threadIdx.x < jd) ys[threadIdx.x] = s->y[threadIdx.x];
    __syncthreads();
    if (!assign && jd == 0) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double acc = 0.0;
        for (int i = 0; i < jd; ++i) acc = fma(ys[i], Z[(int64_t)i * ld + e], acc);
        x[e] = assign ? acc : x[e] + acc;
    }
}

// out = a - b
__global__ void kr_sub_kernel(const double *__restrict__ a, const double *__restrict__ b, double *__restrict__ out,
                              int64_t n, const int *__restrict__ active) {
    if (active && !*active) return;
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        out[e] = a[e] - b[e];
}

static int vgrid(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

// ------------------------------------------------------------------ plan

static size_t align256(size_t b) { return (b + 255) & ~(size_t)255; }

cudaError_t KrylovSolver::layout(void *ws, size_t *bytes) {
    // level sizes in blocks: the larger half at every level
    nblk[0] = op.N;
    for (int l = 1; l <= levels; ++l) nblk[l] = (nblk[l - 1] + 1) / 2;
    char *p = (char *)ws;
    size_t off = 0;
    auto take = [&](size_t b) -> char * {
        char *q = p ? p + off : nullptr;
        off += align256(b);
        return q;
    };
    states = (KState *)take((size_t)(levels + 1) * sizeof(KState));
    partial = (double *)take((size_t)GM_BLOCKS * GM_MAXV * sizeof(double));
    for (int l = 0; l <= levels; ++l) {
        const int64_t n = (int64_t)nblk[l] * op.M;
        V[l] = (double *)take((size_t)(m[l] + 1) * n * sizeof(double));
        Z[l] = l < levels ? (double *)take((size_t)m[l] * n * sizeof(double)) : nullptr;
        w[l] = (double *)take((size_t)n * sizeof(double));
        t[l] = l >= 1 ? (double *)take((size_t)n * sizeof(double)) : nullptr;
    }
    const int64_t n0 = (int64_t)op.N * op.M;
    pin = levels >= 1 ? (double *)take((size_t)n0 * sizeof(double)) : nullptr;
    pout = levels >= 1 ? (double *)take((size_t)n0 * sizeof(double)) : nullptr;
    *bytes = off;
    return cudaSuccess;
}

cudaError_t KrylovSolver::matvec(const double *x, double *y, int ka, int nk, int ia, int nx, const int *active,
                                 cudaStream_t st) {
    return launch_hessenberg_range(op.blk, op.nb, op.far_fp64, x, op.xT, y, op.M, ka, nk, ia, nx, active, op.nsm,
                                   op.variant, st);
}

// one Arnoldi step j of the solve at level l on block range [lo, hi) with
// the preconditioned vector z
cudaError_t KrylovSolver::arnoldi(int l, int lo, int hi, int j, const double *z, cudaStream_t st) {
    KState *s = states + l;
    const int64_t n = (int64_t)(hi - lo) * op.M;
    const int nbk = hi - lo;
    cudaError_t e = matvec(z, w[l], lo, nbk, lo, nbk, &s->run, st);
    if (e != cudaSuccess) return e;
    for (int pass = 0; pass < 2; ++pass) {
        launch_multi_dot(V[l], n, j + 1, w[l], n, partial, s->hc + pass * GM_MAXV, st, &s->run);
        launch_multi_axpy(V[l], n, j + 1, s->hc + pass * GM_MAXV, -1.0, w[l], n, st, &s->run);
    }
    launch_multi_dot(w[l], n, 1, w[l], n, partial, &s->w2, st, &s->run);
    kr_step_kernel<<<1, 1, 0, st>>>(s, j, tol);
    if (j + 1 < m[l]) kr_scale_kernel<<<vgrid(n), 256, 0, st>>>(s, w[l], V[l] + (int64_t)(j + 1) * n, n);
    return cudaGetLastError();
}

// x = approximate solution of A[lo:hi, lo:hi] x = rhs: one FGMRES cycle of
// m[l] steps from zero at level l >= 1, started only if *parent is set
cudaError_t KrylovSolver::inner_solve(int l, int lo, int hi, const double *rhs, double *x, const int *parent,
                                      cudaStream_t st) {
    KState *s = states + l;
    const int64_t n = (int64_t)(hi - lo) * op.M;
    launch_multi_dot(rhs, n, 1, rhs, n, partial, &s->r2, st, parent);
    kr_begin_kernel<<<1, 1, 0, st>>>(s, parent, m[l], tol, 1);
    kr_scale_kernel<<<vgrid(n), 256, 0, st>>>(s, rhs, V[l], n);
    const bool pre = l < levels && hi - lo >= 2;
    cudaError_t e = cudaSuccess;
    for (int j = 0; j < m[l] && e == cudaSuccess; ++j) {
        const double *vj = V[l] + (int64_t)j * n;
        const double *z = vj;
        if (pre) {
            double *zj = Z[l] + (int64_t)j * n;
            e = precondition(l + 1, lo, hi, vj, zj, &s->run, st);
            z = zj;
        }
        if (e == cudaSuccess) e = arnoldi(l, lo, hi, j, z, st);
    }
    if (e != cudaSuccess) return e;
    kr_finish_kernel<<<1, 1, 0, st>>>(s);
    kr_update_kernel<<<vgrid(n), 256, 0, st>>>(s, pre ? Z[l] : V[l], n, x, n, 1);
    return cudaGetLastError();
}

// out = M^-1 in for the level-l splitting of block range [lo, hi)
cudaError_t KrylovSolver::precondition(int l, int lo, int hi, const double *in, double *out, const int *parent,
                                       cudaStream_t st) {
    const int64_t n = (int64_t)(hi - lo) * op.M;
    if (hi - lo < 2) return cudaMemcpyAsync(out, in, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    const int h = lo + (hi - lo + 1) / 2;
    const int64_t n1 = (int64_t)(h - lo) * op.M, n2 = n - n1;
    cudaError_t e = inner_solve(l, lo, h, in, out, parent, st);
    // t = r2 - M21 y1 (w[l] is free between the two half solves)
    if (e == cudaSuccess) e = matvec(out, w[l], h, hi - h, lo, h - lo, parent, st);
    if (e != cudaSuccess) return e;
    kr_sub_kernel<<<vgrid(n2), 256, 0, st>>>(in + n1, w[l], t[l], n2, parent);
    return inner_solve(l, h, hi, t[l], out + n1, parent, st);
}

cudaError_t KrylovSolver::read_head(KHead *h, cudaStream_t st) {
    cudaError_t e = cudaMemcpyAsync(h, states, sizeof(KHead), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    return e;
}

cudaError_t KrylovSolver::apply_preconditioner(const double *r, double *z, cudaStream_t st) {
    // one application outside any outer solve: no caller flag
    if (levels < 1) {
        return cudaMemcpyAsync(z, r, (size_t)op.N * op.M * sizeof(double), cudaMemcpyDeviceToDevice, st);
    }
    return precondition(1, 0, op.N, r, z, nullptr, st);
}

cudaError_t KrylovSolver::solve(const double *g, double *x, int max_iter, cudaStream_t st, cudaStream_t cap,
                                int *iters, double *rel_res) {
    const int64_t n = (int64_t)op.N * op.M;
    KState *s0 = states;
    cudaError_t e = cudaMemsetAsync(x, 0, n * sizeof(double), st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(V[0], g, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    launch_multi_dot(V[0], n, 1, V[0], n, partial, &s0->r2, st);
    kr_begin_kernel<<<1, 1, 0, st>>>(s0, nullptr, m[0], tol, 1);
    KHead h{};
    if ((e = read_head(&h, st)) != cudaSuccess) return e;
    *iters = 0;
    *rel_res = 0.0;
    if (h.run == 0 && h.resid == 0.0) return cudaGetLastError();  // g = 0: alpha = 0
    // the preconditioner application, recorded once and replayed per step
    cudaGraphExec_t gexec = nullptr;
    if (levels >= 1) {
        cudaGraph_t gr = nullptr;
        e = cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed);
        if (e != cudaSuccess) return e;
        const cudaError_t ec = precondition(1, 0, op.N, pin, pout, &s0->run, cap);
        e = cudaStreamEndCapture(cap, &gr);
        if (e == cudaSuccess) e = ec;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&gexec, gr, 0);
        if (e == cudaSuccess) {
            size_t nn = 0;
            if (cudaGraphGetNodes(gr, nullptr, &nn) == cudaSuccess) graph_nodes = (int64_t)nn;
        }
        if (gr) cudaGraphDestroy(gr);
        if (e != cudaSuccess) return e;
    }
    int total = 0;
    bool done = h.run == 0;
    while (!done && e == cudaSuccess) {
        kr_scale_kernel<<<vgrid(n), 256, 0, st>>>(s0, V[0], V[0], n);
        bool stop = false;
        for (int j = 0; j < m[0] && e == cudaSuccess; ++j) {
            const double *vj = V[0] + (int64_t)j * n;
            const double *z = vj;
            if (levels >= 1) {
                double *zj = Z[0] + (int64_t)j * n;
                e = cudaMemcpyAsync(pin, vj, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                if (e == cudaSuccess) e = cudaGraphLaunch(gexec, st);
                if (e == cudaSuccess) e = cudaMemcpyAsync(zj, pout, n * sizeof(double), cudaMemcpyDeviceToDevice, st);
                z = zj;
            }
            if (e == cudaSuccess) e = arnoldi(0, 0, op.N, j, z, st);
            if (e == cudaSuccess) e = read_head(&h, st);
            if (e != cudaSuccess) break;
            ++total;
            if (h.run == 0 || total >= max_iter) {
                stop = h.stop != 0 || total >= max_iter;
                break;
            }
        }
        if (e != cudaSuccess) break;
        kr_finish_kernel<<<1, 1, 0, st>>>(s0);
        kr_update_kernel<<<vgrid(n), 256, 0, st>>>(s0, levels >= 1 ? Z[0] : V[0], n, x, n, 0);
        if (stop) break;
        // restart from the true residual
        e = matvec(x, w[0], 0, op.N, 0, op.N, nullptr, st);
        if (e != cudaSuccess) break;
        kr_sub_kernel<<<vgrid(n), 256, 0, st>>>(g, w[0], V[0], n, nullptr);
        launch_multi_dot(V[0], n, 1, V[0], n, partial, &s0->r2, st);
        kr_begin_kernel<<<1, 1, 0, st>>>(s0, nullptr, m[0], tol, 0);
        if ((e = read_head(&h, st)) != cudaSuccess) break;
        done = h.run == 0 || total >= max_iter;
    }
    if (e == cudaSuccess) {
        // the true residual of the final iterate
        e = matvec(x, w[0], 0, op.N, 0, op.N, nullptr, st);
        if (e == cudaSuccess) {
            kr_sub_kernel<<<vgrid(n), 256, 0, st>>>(g, w[0], V[0], n, nullptr);
            launch_multi_dot(V[0], n, 1, V[0], n, partial, &s0->r2, st);
            double r2 = 0.0, bref = 0.0;
            e = cudaMemcpyAsync(&r2, &s0->r2, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaMemcpyAsync(&bref, &s0->bref, sizeof(double), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e == cudaSuccess) *rel_res = bref > 0.0 ? sqrt(r2) / bref : 0.0;
        }
    }
    if (gexec) cudaGraphExecDestroy(gexec);
    *iters = total;
    return e == cudaSuccess ? cudaGetLastError() : e;
}

}  // namespace tdbem
