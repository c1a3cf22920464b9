// Vector kernels of the restarted GMRES solver for the block-Hessenberg
// system A alpha = g (the iterative solution of Sec. 4 with the matrix-vector
// product of Sec. 5.1). FP64 throughout; every reduction is a fixed-order
// two-pass block sum, so repeated solves are bitwise identical. The dot and
// axpy kernels take an optional device flag `active`: when it is given and
// zero they do nothing (the converged inner solves of fgmres.cu).
#include "tdbem_internal.h"

namespace tdbem {

// partial[b][v] = sum over block b's elements of V[v][e] w[e], v < nv
__global__ void __launch_bounds__(256) multi_dot_partial(const double *__restrict__ V, int64_t ld, int nv,
                                                         const double *__restrict__ w, int64_t n,
                                                         double *__restrict__ partial,
                                                         const int *__restrict__ active) {
    if (active && !*active) return;
    __shared__ double red[256];
    for (int v = 0; v < nv; ++v) {
        const double *vv = V + (int64_t)v * ld;
        double s = 0.0;
        for (int64_t e = (int64_t)blockIdx.x * 256 + threadIdx.x; e < n; e += (int64_t)gridDim.x * 256)
            s = fma(vv[e], w[e], s);
        red[threadIdx.x] = s;
        __syncthreads();
        for (int o = 128; o > 0; o >>= 1) {
            if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
            __syncthreads();
        }
        if (threadIdx.x == 0) partial[(int64_t)blockIdx.x * GM_MAXV + v] = red[0];
        __syncthreads();
    }
}

// h[v] = sum_b partial[b][v], in block order
__global__ void multi_dot_final(const double *__restrict__ partial, int nb, int nv, double *__restrict__ h,
                                const int *__restrict__ active) {
    if (active && !*active) return;
    const int v = threadIdx.x;
    if (v >= nv) return;
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += partial[(int64_t)b * GM_MAXV + v];
    h[v] = s;
}

// w[e] += sign * sum_v h[v] V[v][e]
__global__ void multi_axpy_kernel(const double *__restrict__ V, int64_t ld, int nv, const double *__restrict__ h,
                                  double sign, double *__restrict__ w, int64_t n, const int *__restrict__ active) {
    if (active && !*active) return;
    __shared__ double hs[GM_MAXV];
    if (threadIdx.x < nv) hs[threadIdx.x] = h[threadIdx.x];
    __syncthreads();
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int v = 0; v < nv; ++v) s = fma(hs[v], V[(int64_t)v * ld + e], s);
        w[e] = fma(sign, s, w[e]);
    }
}

// v = w / beta[0]
__global__ void scale_copy_kernel(const double *__restrict__ w, const double *__restrict__ beta,
                                  double *__restrict__ v, int64_t n) {
    const double ib = 1.0 / beta[0];
    for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x)
        v[e] = w[e] * ib;
}

static int grid_for(int64_t n) { return (int)std::min<int64_t>((n + 255) / 256, 4096); }

void launch_multi_dot(const double *V, int64_t ld, int nv, const double *w, int64_t n, double *partial, double *h,
                      cudaStream_t st, const int *active) {
    const int nb = (int)std::min<int64_t>((n + 255) / 256, GM_BLOCKS);
    multi_dot_partial<<<nb, 256, 0, st>>>(V, ld, nv, w, n, partial, active);
    multi_dot_final<<<1, GM_MAXV, 0, st>>>(partial, nb, nv, h, active);
}

void launch_multi_axpy(const double *V, int64_t ld, int nv, const double *h, double sign, double *w, int64_t n,
                       cudaStream_t st, const int *active) {
    multi_axpy_kernel<<<grid_for(n), 256, 0, st>>>(V, ld, nv, h, sign, w, n, active);
}

void launch_scale_copy(const double *w, const double *beta, double *v, int64_t n, cudaStream_t st) {
    scale_copy_kernel<<<grid_for(n), 256, 0, st>>>(w, beta, v, n);
}

}  // namespace tdbem
