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
// the warp. Products and sums are FP64 (far values are widened from FP32 in
// the mixed path). Every y entry is written by its owning warp only, in a
// fixed order: the result is deterministic and needs no atomics.
#include "tdbem_internal.h"

namespace tdbem {

constexpr int MV_WARPS = 8;
constexpr int MV_PP = 4;  // positions per lane in one pass of the wide mapping

__global__ void __launch_bounds__(1024) transpose_kernel(const double *__restrict__ x, double *__restrict__ xT,
                                                         int64_t N, int64_t M) {
    __shared__ double tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32, i0 = (int64_t)blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 32
    if (i0 + ty < N && j0 + tx < M) tile[ty][tx] = x[(i0 + ty) * M + j0 + tx];
    __syncthreads();
    if (j0 + ty < M && i0 + tx < N) xT[(j0 + ty) * N + i0 + tx] = tile[tx][ty];
}

template <typename VT>
__device__ __forceinline__ void row_apply(const int64_t *__restrict__ rp, const int32_t *__restrict__ col,
                                          const VT *__restrict__ val, int64_t l, int k0, int i0, int cnt,
                                          const double *__restrict__ xT, int N, double *ys, int lane) {
    const int64_t a = rp[l], e = rp[l + 1];
    if (a == e) return;
    if (cnt >= 16) {
        for (int p0 = 0; p0 < cnt; p0 += 32 * MV_PP) {
            double acc[MV_PP];
#pragma unroll
            for (int m = 0; m < MV_PP; ++m) acc[m] = 0.0;
            const int pl = p0 + lane;
            for (int64_t base = a; base < e; base += 32) {
                const int n = (int)min((int64_t)32, e - base);
                int cj = 0;
                double cv = 0.0;
                if (lane < n) { cj = col[base + lane]; cv = (double)val[base + lane]; }
                for (int t = 0; t < n; ++t) {
                    const int j = __shfl_sync(0xffffffffu, cj, t);
                    const double v = __shfl_sync(0xffffffffu, cv, t);
                    const double *xr = xT + (int64_t)j * N + i0 + pl;
#pragma unroll
                    for (int m = 0; m < MV_PP; ++m)
                        if (pl + 32 * m < cnt) acc[m] = fma(v, xr[32 * m], acc[m]);
                }
            }
#pragma unroll
            for (int m = 0; m < MV_PP; ++m)
                if (pl + 32 * m < cnt) ys[k0 + pl + 32 * m] += acc[m];
        }
    } else {
        for (int p = 0; p < cnt; ++p) {
            double acc = 0.0;
            for (int64_t nz = a + lane; nz < e; nz += 32) acc = fma((double)val[nz], xT[(int64_t)col[nz] * N + i0 + p], acc);
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
            if (lane == 0) ys[k0 + p] += acc;
        }
    }
    __syncwarp();
}

template <typename VT>
__global__ void __launch_bounds__(MV_WARPS * 32) hessenberg_kernel(const MvBlock *__restrict__ blk, int nb,
                                                                   const double *__restrict__ xT,
                                                                   double *__restrict__ y, int64_t M, int N) {
    extern __shared__ double ys_all[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    double *ys = ys_all + (size_t)w * N;
    for (int64_t l = (int64_t)blockIdx.x * MV_WARPS + w; l < M; l += (int64_t)gridDim.x * MV_WARPS) {
        for (int k = lane; k < N; k += 32) ys[k] = 0.0;
        __syncwarp();
        for (int b = 0; b < nb; ++b) {
            const MvBlock B = blk[b];
            row_apply<VT>(B.rp_far, B.col_far, (const VT *)B.val_far, l, B.k0, B.i0, B.cnt, xT, N, ys, lane);
            row_apply<double>(B.rp_near, B.col_near, B.val_near, l, B.k0, B.i0, B.cnt, xT, N, ys, lane);
        }
        for (int k = lane; k < N; k += 32) y[(int64_t)k * M + l] = ys[k];
        __syncwarp();
    }
}

size_t hessenberg_smem(int N) { return (size_t)MV_WARPS * N * sizeof(double); }

cudaError_t launch_hessenberg(const MvBlock *blk, int nb, bool far_fp64, const double *x, double *xT, double *y,
                              int64_t M, int N, int nsm, cudaStream_t st) {
    const dim3 tg((unsigned)((M + 31) / 32), (unsigned)((N + 31) / 32));
    transpose_kernel<<<tg, dim3(32, 32), 0, st>>>(x, xT, N, M);
    const size_t smem = hessenberg_smem(N);
    const int64_t ctas = (M + MV_WARPS - 1) / MV_WARPS;
    const int grid = (int)std::min<int64_t>(ctas, (int64_t)nsm * 8);
    cudaError_t e;
    if (far_fp64) {
        if ((e = cudaFuncSetAttribute(hessenberg_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        hessenberg_kernel<double><<<grid, MV_WARPS * 32, smem, st>>>(blk, nb, xT, y, M, N);
    } else {
        if ((e = cudaFuncSetAttribute(hessenberg_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem)))
            return e;
        hessenberg_kernel<float><<<grid, MV_WARPS * 32, smem, st>>>(blk, nb, xT, y, M, N);
    }
    return cudaGetLastError();
}

}  // namespace tdbem
