// Block-Hessenberg matrix-vector product y = A x of the whole space-time
// system (Sec. 5.1, Eq. Apartitioned). Only the unique blocks are stored;
// every other block is one of them by Eq. relationAtildeBlock, so each
// unique block b is applied to a run of cnt_b positions (k0 + p, i0 + p),
// p < cnt_b, along its diagonal: cnt_b = N - 1 - k for the inner blocks of
// the second block column (0-based (k, 1)), N - 3 for block (1, 2), one for
// every other block.
//
// x and y are (N, M) FP64, block row k = y[k * M .. k * M + M). x is first
// transposed into the scratch xT (M, N) so that a warp reads the values of
// one trial vertex at consecutive time indices with one coalesced load. One
// warp owns one test vertex l: it keeps y[:, l] in shared memory, walks the
// far and the near CSR row l of every unique block and adds
//   y[k0 + p, l] += sum_j A_b(l, j) xT[j, i0 + p].
// Runs of 16 or more positions map lanes to positions (broadcast of the
// nonzero by shuffle); shorter runs map lanes to nonzeros and reduce across
// the warp. FP64 path: x, products and sums in FP64. Mixed path (FP32 far
// values): x is rounded to FP32 in the transpose, far products are FP32 and
// summed in FP32 over at most 32 products, and these partial sums are
// accumulated as FP32 pairs with an error-free two-sum and added into the
// FP64 row once per row and block (the FP64 pipe runs at 1/64 of the FP32
// rate here); the FP64 near values multiply the same x in FP64. Every y entry is written by
// its owning warp only, in a fixed order: the result is deterministic and
// needs no atomics.
#include <type_traits>

#include "tdbem_internal.h"

namespace tdbem {

// launch shape (positions per lane in one pass of the wide mapping, warps
// per CTA) is a template parameter chosen by the autotuner (MV_VARIANTS)

template <typename XT>
__global__ void __launch_bounds__(1024) transpose_kernel(const double *__restrict__ x, XT *__restrict__ xT, int64_t N,
                                                         int64_t M, const int *__restrict__ active) {
    if (active && !*active) return;
    __shared__ double tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
    if (i0 + ty < N && j0 + tx < M) tile[ty][tx] = x[(i0 + ty) * M + j0 + tx];
    __syncthreads();
    if (j0 + ty < M && i0 + tx < N) xT[(j0 + ty) * N + i0 + tx] = (XT)tile[tx][ty];
}

// Accumulators of the sums over a row: FP64 in the FP64 path; in the mixed
// path an unevaluated FP32 pair (hi, lo) updated with an error-free two-sum,
// so the FP64 pipe (1/64 of the FP32 rate) is used once per row and block.
struct AccPair {
    float h, l;
};
__device__ __forceinline__ void acc_zero(double &a) { a = 0.0; }
__device__ __forceinline__ void acc_zero(AccPair &a) { a.h = 0.f; a.l = 0.f; }
__device__ __forceinline__ void acc_add(double &a, double v) { a += v; }
__device__ __forceinline__ void acc_add(AccPair &a, float v) {
    const float s = a.h + v;
    const float bb = s - a.h;
    a.l += (a.h - (s - bb)) + (v - bb);
    a.h = s;
}
__device__ __forceinline__ void acc_add(AccPair &a, AccPair v) {
    acc_add(a, v.h);
    a.l += v.l;
}
__device__ __forceinline__ double acc_value(double a) { return a; }
__device__ __forceinline__ double acc_value(AccPair a) { return (double)a.h + (double)a.l; }
__device__ __forceinline__ double shfl_xor(double v, int o) { return __shfl_xor_sync(0xffffffffu, v, o); }
__device__ __forceinline__ AccPair shfl_xor(AccPair v, int o) {
    return AccPair{__shfl_xor_sync(0xffffffffu, v.h, o), __shfl_xor_sync(0xffffffffu, v.l, o)};
}

// x value of trial vertex j at time index i: from the transposed copy xT
// (M, N) of type XT, or (XD) from x itself ((N, M) FP64, row stride M),
// rounded to XT so that both reads give the same value
template <typename XT, bool XD>
__device__ __forceinline__ XT x_at(const void *__restrict__ xs, int64_t j, int64_t i, int N, int64_t M) {
    if constexpr (XD) return (XT)((const double *)xs)[i * M + j];
    else return ((const XT *)xs)[j * N + i];
}

// products and sums of one CSR row of one block for the positions of its run.
// F32: FP32 products of FP32 values and FP32 x, partial sums of at most 32
// products in FP32, accumulated as FP32 pairs (two-sum) and added into the
// FP64 row once; otherwise FP64 products and sums.
template <typename VT, typename XT, bool F32, int PP, bool XD>
__device__ __forceinline__ void row_apply(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const VT *__restrict__ val, int64_t l, int k0, int i0, int cnt,
                                          const void *__restrict__ xs, int N, int64_t M, double *ys, int lane) {
    typedef typename std::conditional<F32, float, double>::type AT;
    typedef typename std::conditional<F32, AccPair, double>::type ACC;
    const int64_t a = rp[l], e = rp[l + 1];
    if (a == e) return;
    if (cnt >= 16) {
        for (int p0 = 0; p0 < cnt; p0 += 32 * PP) {
            ACC acc[PP];
#pragma unroll
            for (int m = 0; m < PP; ++m) acc_zero(acc[m]);
            const int pl = p0 + lane;
            for (int64_t base = a; base < e; base += 32) {
                const int n = (int)min((int64_t)32, e - base);
                int cj = 0;
                AT cv = 0;
                if (lane < n) { cj = col[base + lane]; cv = (AT)val[base + lane]; }
                AT part[PP];
#pragma unroll
                for (int m = 0; m < PP; ++m) part[m] = 0;
                for (int t = 0; t < n; ++t) {
                    const int j = __shfl_sync(0xffffffffu, cj, t);
                    const AT v = __shfl_sync(0xffffffffu, cv, t);
#pragma unroll
                    for (int m = 0; m < PP; ++m)
                        if (pl + 32 * m < cnt)
                            part[m] = fma(v, (AT)x_at<XT, XD>(xs, j, i0 + pl + 32 * m, N, M), part[m]);
                }
#pragma unroll
                for (int m = 0; m < PP; ++m) acc_add(acc[m], part[m]);
            }
#pragma unroll
            for (int m = 0; m < PP; ++m)
                if (pl + 32 * m < cnt) ys[k0 + pl + 32 * m] += acc_value(acc[m]);
        }
    } else {
        for (int p = 0; p < cnt; ++p) {
            ACC acc;
            acc_zero(acc);
            for (int64_t c0 = a; c0 < e; c0 += 32 * 32) {
                const int64_t c1 = min(e, c0 + 32 * 32);
                AT part = 0;
                for (int64_t nz = c0 + lane; nz < c1; nz += 32)
                    part = fma((AT)val[nz], (AT)x_at<XT, XD>(xs, col[nz], i0 + p, N, M), part);
                acc_add(acc, part);
            }
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc_add(acc, shfl_xor(acc, o));
            if (lane == 0) ys[k0 + p] += acc_value(acc);
        }
    }
    __syncwarp();
}

// VT: far value type. F32 (mixed path): x in FP32, far products in FP32 with
// FP64 sums of 32-product partials; the FP64 near values multiply the same
// FP32 x in FP64. Otherwise (FP64 path) everything is FP64.
//
// Block ranges: only block rows ka <= k < ka + nk and block columns
// ia <= i < ia + nx take part (the diagonal and off-diagonal parts of the
// splitting of Sec. 4.2); x is then (nx, M) and y (nk, M). The whole product
// is ka = ia = 0, nk = nx = N. Each run is cut to the positions p with both
// k0 + p and i0 + p inside the ranges. active: if given and zero, the
// kernel does nothing (a converged solve, see fgmres.cu).
//
// XD: x is read directly in its (N, M) layout instead of the transposed copy
// (the blocks that are not part of a diagonal run: consecutive columns of a
// CSR row are then consecutive addresses).
template <typename VT, bool F32, int PP, int WARPS, bool XD>
__global__ void __launch_bounds__(WARPS * 32) hessenberg_kernel(const MvBlock *__restrict__ blk, int nb,
                                                                const void *__restrict__ xs,
                                                                double *__restrict__ y, int64_t M, int ka, int nk,
                                                                int ia, int nx, const int *__restrict__ active) {
    typedef typename std::conditional<F32, float, double>::type XT;
    if (active && !*active) return;
    extern __shared__ double ys_all[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *ys = ys_all + (size_t)w * nk;
    for (int64_t l = (int64_t)blockIdx.x * WARPS + w; l < M; l += (int64_t)gridDim.x * WARPS) {
        for (int k = lane; k < nk; k += 32) ys[k] = 0.0;
        __syncwarp();
        for (int b = 0; b < nb; ++b) {
            const MvBlock B = blk[b];
            const int plo = max(0, max(ka - B.k0, ia - B.i0));
            const int phi = min(B.cnt, min(ka + nk - B.k0, ia + nx - B.i0));
            if (phi <= plo) continue;
            const int k0 = B.k0 + plo - ka, i0 = B.i0 + plo - ia, cnt = phi - plo;
            row_apply<VT, XT, F32, PP, XD>(B.rp_far, B.col_far, (const VT *)B.val_far, l, k0, i0, cnt, xs, nx, M, ys,
                                           lane);
            row_apply<double, XT, false, PP, XD>(B.rp_near, B.col_near, B.val_near, l, k0, i0, cnt, xs, nx, M, ys,
                                                 lane);
        }
        for (int k = lane; k < nk; k += 32) y[(int64_t)k * M + l] = ys[k];
        __syncwarp();
    }
}

// The tunable launch shapes: (positions per lane, warps per CTA).
static const int MV_VARIANTS[MV_NVARIANTS][2] = {{4, 8}, {2, 8}, {8, 8}, {4, 4}, {2, 4}, {8, 4}};

template <typename VT, bool F32, int PP, int WARPS, bool XD = false>
static cudaError_t launch_mv_shape(const MvBlock *blk, int nb, const void *xT, double *y, int64_t M, int ka, int nk,
                                   int ia, int nx, const int *active, int nsm, cudaStream_t st) {
    const size_t smem = (size_t)WARPS * nk * sizeof(double);
    const int64_t ctas = (M + WARPS - 1) / WARPS;
    const int grid = (int)std::min<int64_t>(ctas, (int64_t)nsm * 16);
    cudaError_t e = cudaFuncSetAttribute(hessenberg_kernel<VT, F32, PP, WARPS, XD>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    hessenberg_kernel<VT, F32, PP, WARPS, XD>
        <<<grid, WARPS * 32, smem, st>>>(blk, nb, xT, y, M, ka, nk, ia, nx, active);
    return cudaGetLastError();
}

// the blocks outside the Toeplitz class in the mixed path, x read directly
cudaError_t launch_hessenberg_rest(const MvBlock *blk, int nb, const double *x, double *y, int64_t M, int N, int nsm,
                                   int variant, cudaStream_t st) {
    switch (variant) {
        case 1: return launch_mv_shape<float, true, 2, 8, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
        case 2: return launch_mv_shape<float, true, 8, 8, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
        case 3: return launch_mv_shape<float, true, 4, 4, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
        case 4: return launch_mv_shape<float, true, 2, 4, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
        case 5: return launch_mv_shape<float, true, 8, 4, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
        default: return launch_mv_shape<float, true, 4, 8, true>(blk, nb, x, y, M, 0, N, 0, N, nullptr, nsm, st);
    }
}

template <typename VT, bool F32>
static cudaError_t launch_mv(const MvBlock *blk, int nb, const double *x, void *xT, double *y, int64_t M, int ka,
                             int nk, int ia, int nx, const int *active, int nsm, int variant, cudaStream_t st) {
    typedef typename std::conditional<F32, float, double>::type XT;
    const dim3 tg((unsigned)((M + 31) / 32), (unsigned)((nx + 31) / 32));
    transpose_kernel<XT><<<tg, dim3(32, 32), 0, st>>>(x, (XT *)xT, nx, M, active);
    switch (variant) {
        case 1: return launch_mv_shape<VT, F32, 2, 8>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
        case 2: return launch_mv_shape<VT, F32, 8, 8>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
        case 3: return launch_mv_shape<VT, F32, 4, 4>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
        case 4: return launch_mv_shape<VT, F32, 2, 4>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
        case 5: return launch_mv_shape<VT, F32, 8, 4>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
        default: return launch_mv_shape<VT, F32, 4, 8>(blk, nb, xT, y, M, ka, nk, ia, nx, active, nsm, st);
    }
}

cudaError_t launch_hessenberg(const MvBlock *blk, int nb, bool far_fp64, const double *x, double *xT, double *y,
                              int64_t M, int N, int nsm, int variant, cudaStream_t st) {
    return launch_hessenberg_range(blk, nb, far_fp64, x, xT, y, M, 0, N, 0, N, nullptr, nsm, variant, st);
}

cudaError_t launch_hessenberg_range(const MvBlock *blk, int nb, bool far_fp64, const double *x, double *xT, double *y,
                                    int64_t M, int ka, int nk, int ia, int nx, const int *active, int nsm, int variant,
                                    cudaStream_t st) {
    if (far_fp64) return launch_mv<double, false>(blk, nb, x, xT, y, M, ka, nk, ia, nx, active, nsm, variant, st);
    return launch_mv<float, true>(blk, nb, x, xT, y, M, ka, nk, ia, nx, active, nsm, variant, st);
}

}  // namespace tdbem
