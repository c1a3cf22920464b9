// Toeplitz part of the mixed-precision block-Hessenberg product (Sec. 5.1,
// Eq. relationAtildeBlock). On an equidistant grid the inner blocks of the
// second block column, (d + 1, 1) for d >= 0, and block (1, 2) (d = -1) stand
// for every block (m, i) with 1 <= m, i <= N - 2 and lag d = m - i >= -1.
// Per test vertex l and inner row m = u + 1 (u = 0 .. N - 3) their share of
// the product is
//
//   y[u + 1, l] += sum_j sum_d A_d(l, j) x[u + 1 - d, j],   0 <= u - d < N - 2.
//
// For one vertex pair (l, j) the lags d with A_d(l, j) in the pattern form
// one window [a, b] of a few lags (the support of psi at lag d is
// [(d - 2) dt, (d + 2) dt], the distances of the pair one interval: Eq.
// SparsitySmallBlock), which the assembler keeps as the pair's lag window.
// This file stores every window in entries of TW lags: the pair's trial
// vertex j, the first lag, and TW values, zero past the end of the window
// (a window longer than TW takes several entries). The far values are FP32
// (the CSR values of the mixed path, hi + lo of the accumulated pair), the
// near values FP64.
//
// One warp handles one test vertex l; lane L owns the outputs
// u = u0 + 4 L .. u0 + 4 L + 3 of a chunk of 128. For an entry (j, a) these
// outputs meet x_j at the 4 + TW - 1 inner time indices
// u0 + 4 L - a - (TW - 1) .. u0 + 4 L + 3 - a, which the lane reads with
// aligned float4 loads from a padded FP32 copy of x (zeros outside the inner
// indices, so the bounds need no test) and then applies all TW lags from
// registers. Each x value is thus read once per vertex pair and used for up
// to 4 TW products; the per-block CSR product reads it once per (pair, lag)
// and position run. Far products are FP32 and summed in FP32 over four
// entries (at most 4 TW products), and these partial sums are accumulated as
// FP32 pairs with an error-free two-sum; near products and sums are FP64.
// Each y entry is written by its own warp only, after the product of the
// other blocks has written it: the result is deterministic.
#include "tdbem_internal.h"

namespace tdbem {

constexpr int TW_WARPS = 8;

// xP[j S + PADL + c] = x[(c + 1) M + j] rounded to FP32 for the inner time
// indices c = 0 .. N - 3, zero at every other position of the row
__global__ void __launch_bounds__(256) tw_transpose_kernel(const double *__restrict__ x, float *__restrict__ xP,
                                                           int64_t N, int64_t M, int S, int PADL) {
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int q0 = blockIdx.y * 32;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int64_t nin = N - 2;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int q = q0 + ty + 8 * s;
        const int64_t c = (int64_t)q - PADL;
        float v = 0.f;
        if (c >= 0 && c < nin && j0 + tx < M) v = (float)x[(c + 1) * M + j0 + tx];
        tile[ty + 8 * s][tx] = v;
    }
    __syncthreads();
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t j = j0 + ty + 8 * s;
        const int q = q0 + tx;
        if (j < M && q < S) xP[j * S + q] = tile[tx][ty + 8 * s];
    }
}

// ------------------------------------------------------------ layout build
// Entries per row: set 0 = far (every trial vertex j), set 1 = near (the
// neighbour list of l); a non-empty window [a, b] gives ceil((b - a + 1) / TW)
// entries. One warp per (set, row).
__global__ void tw_count_kernel(int64_t M, const int16_t *__restrict__ dlo, const int16_t *__restrict__ dhi,
                                const int64_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr, int TW,
                                int64_t *__restrict__ cnt) {
    const int lane = threadIdx.x & 31;
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= 2 * M) return;
    const int set = (int)(item / M);
    const int64_t l = item % M;
    const int64_t k0 = set ? nbr_ptr[l] : 0, k1 = set ? nbr_ptr[l + 1] : M;
    int64_t n = 0;
    for (int64_t k = k0 + lane; k < k1; k += 32) {
        const int64_t j = set ? nbr[k] : k;
        const int a = dlo[l * M + j], b = dhi[l * M + j];
        if (a <= b) n += (b - a + TW) / TW;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n += __shfl_xor_sync(0xffffffffu, n, o);
    if (lane == 0) cnt[set * M + l] = n;
}

// Entries of row l in order of the trial vertex, then of the first lag; the
// positions come from an exclusive scan of the counts (ptr, 2 x (M + 1)).
// dense: the far windows of the class, FP32 pairs (hi, lo) at
// ((l M + j) KW + d - a); ndense: the near windows, FP64 at
// ((l NB + k - nbr_ptr[l]) KW + d - a).
__global__ void tw_fill_kernel(int64_t M, const int16_t *__restrict__ dlo, const int16_t *__restrict__ dhi,
                               const int64_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr, int TW,
                               const int64_t *__restrict__ ptr, const float2 *__restrict__ dense,
                               const double *__restrict__ ndense, int KW, int NB, int2 *__restrict__ fhdr,
                               float *__restrict__ fval, int2 *__restrict__ nhdr, double *__restrict__ nval) {
    const int lane = threadIdx.x & 31;
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= 2 * M) return;
    const int set = (int)(item / M);
    const int64_t l = item % M;
    const int64_t k0 = set ? nbr_ptr[l] : 0, k1 = set ? nbr_ptr[l + 1] : M;
    int64_t pos = ptr[set * (M + 1) + l];
    for (int64_t kb = k0; kb < k1; kb += 32) {
        const int64_t k = kb + lane;
        int a = 0, b = -1;
        int64_t j = 0;
        if (k < k1) {
            j = set ? nbr[k] : k;
            a = dlo[l * M + j];
            b = dhi[l * M + j];
        }
        const int n = a <= b ? (b - a + TW) / TW : 0;
        int incl = n;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        const int64_t my = pos + incl - n;
        for (int q = 0; q < n; ++q) {
            const int a0 = a + TW * q;
            const int64_t e = my + q;
            if (set == 0) {
                fhdr[e] = make_int2((int)j, a0);
                const float2 *w = dense + (l * M + j) * KW;
                for (int t = 0; t < TW; ++t) {
                    const int d = a0 + t;
                    fval[e * TW + t] = d <= b ? w[d - a].x + w[d - a].y : 0.f;
                }
            } else {
                nhdr[e] = make_int2((int)j, a0);
                const double *w = ndense + (l * NB + (k - k0)) * KW;
                for (int t = 0; t < TW; ++t) {
                    const int d = a0 + t;
                    nval[e * TW + t] = d <= b ? w[d - a] : 0.0;
                }
            }
        }
        pos += __shfl_sync(0xffffffffu, incl, 31);
    }
}

// ------------------------------------------------------------ product
template <int TW>
struct TwShape {
    static constexpr int NW = TW + 3;             // x values one lane meets per entry
    static constexpr int NV4 = (NW + 3 + 3) / 4;  // aligned float4 loads covering them at any shift
};

// acc[r] += sum_t a[t] v[SH + TW - 1 + r - t]: output u0 + 4 L + r, lag a0 + t
template <int TW, int SH, typename T, typename A>
__device__ __forceinline__ void tw_apply(const float (&v)[4 * TwShape<TW>::NV4], const A (&a)[TW], T (&acc)[4]) {
#pragma unroll
    for (int t = 0; t < TW; ++t)
#pragma unroll
        for (int r = 0; r < 4; ++r) acc[r] = fma((T)a[t], (T)v[SH + TW - 1 + r - t], acc[r]);
}

template <int TW, typename T, typename A>
__device__ __forceinline__ void tw_entry(const float *__restrict__ row, int base, const A (&a)[TW], T (&acc)[4]) {
    constexpr int NV4 = TwShape<TW>::NV4;
    const int sh = base & 3;  // the same in every lane of the warp
    const float4 *r4 = reinterpret_cast<const float4 *>(row + (base - sh));
    float v[4 * NV4];
#pragma unroll
    for (int q = 0; q < NV4; ++q) {
        const float4 t = __ldg(r4 + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
    switch (sh) {
        case 0: tw_apply<TW, 0>(v, a, acc); break;
        case 1: tw_apply<TW, 1>(v, a, acc); break;
        case 2: tw_apply<TW, 2>(v, a, acc); break;
        default: tw_apply<TW, 3>(v, a, acc); break;
    }
}

__device__ __forceinline__ void two_sum_add(float &h, float &l, float v) {
    const float s = h + v;
    const float bb = s - h;
    l += (h - (s - bb)) + (v - bb);
    h = s;
}

template <int TW>
__global__ void __launch_bounds__(TW_WARPS * 32) toeplitz_kernel(TwArgs g, const float *__restrict__ xP,
                                                                 double *__restrict__ y) {
    const int lane = threadIdx.x & 31;
    const int64_t nwarp = (int64_t)gridDim.x * TW_WARPS;
    const int nin = g.nin;
    for (int64_t l = (int64_t)blockIdx.x * TW_WARPS + (threadIdx.x >> 5); l < g.M; l += nwarp) {
        for (int u0 = 0; u0 < nin; u0 += 128) {
            float acc[4] = {0.f, 0.f, 0.f, 0.f}, ph[4] = {0.f, 0.f, 0.f, 0.f}, pl[4] = {0.f, 0.f, 0.f, 0.f};
            double ad[4] = {0.0, 0.0, 0.0, 0.0};
            const int lbase = g.PADL + u0 + 4 * lane - (TW - 1);
            // far entries, headers fetched 32 at a time and broadcast by shuffle
            const int64_t e0 = g.fptr[l], e1 = g.fptr[l + 1];
            int pend = 0;
            for (int64_t eb = e0; eb < e1; eb += 32) {
                const int ne = (int)min((int64_t)32, e1 - eb);
                int2 hv = make_int2(0, 0);
                if (lane < ne) hv = g.fhdr[eb + lane];
                for (int t = 0; t < ne; ++t) {
                    const int j = __shfl_sync(0xffffffffu, hv.x, t);
                    const int a0 = __shfl_sync(0xffffffffu, hv.y, t);
                    // outputs of this chunk all below the window, or all past it
                    if (a0 > u0 + 127 || u0 - (a0 + TW - 1) > nin - 1) continue;
                    const float4 *vp = reinterpret_cast<const float4 *>(g.fval + (eb + t) * TW);
                    float a[TW];
#pragma unroll
                    for (int q = 0; q < TW / 4; ++q) {
                        const float4 w = __ldg(vp + q);
                        a[4 * q] = w.x;
                        a[4 * q + 1] = w.y;
                        a[4 * q + 2] = w.z;
                        a[4 * q + 3] = w.w;
                    }
                    tw_entry<TW>(xP + (int64_t)j * g.S, lbase - a0, a, acc);
                    if (++pend == 4) {
#pragma unroll
                        for (int r = 0; r < 4; ++r) {
                            two_sum_add(ph[r], pl[r], acc[r]);
                            acc[r] = 0.f;
                        }
                        pend = 0;
                    }
                }
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) two_sum_add(ph[r], pl[r], acc[r]);
            // near entries: FP64 values and sums
            const int64_t n0 = g.nptr[l], n1 = g.nptr[l + 1];
            for (int64_t e = n0; e < n1; ++e) {
                const int2 h = g.nhdr[e];
                if (h.y > u0 + 127 || u0 - (h.y + TW - 1) > nin - 1) continue;
                double a[TW];
#pragma unroll
                for (int t = 0; t < TW; ++t) a[t] = g.nval[e * TW + t];
                tw_entry<TW>(xP + (int64_t)h.x * g.S, lbase - h.y, a, ad);
            }
#pragma unroll
            for (int r = 0; r < 4; ++r) {
                const int u = u0 + 4 * lane + r;
                if (u < nin) y[(int64_t)(u + 1) * g.M + l] += ((double)ph[r] + (double)pl[r]) + ad[r];
            }
        }
    }
}

int tw_lags(int KW) { return KW <= 8 ? 8 : (KW <= 12 ? 12 : 16); }

void tw_geometry(int TW, int max_lag, int N, int *PADL, int *S) {
    const int nch = (N - 2 + 127) / 128;
    const int nv4 = (TW + 3 + 3 + 3) / 4;
    *PADL = (max_lag + TW + 3 + 3) / 4 * 4;
    *S = (*PADL + 128 * nch + 4 * nv4 + 4 + 3) / 4 * 4;
}

void launch_tw_count(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                     int TW, int64_t *cnt, cudaStream_t st) {
    const int64_t threads = 2 * M * 32;
    tw_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, dlo, dhi, nbr_ptr, nbr, TW, cnt);
}

void launch_tw_fill(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                    int TW, const int64_t *ptr, const float2 *dense, const double *ndense, int KW, int NB, int2 *fhdr,
                    float *fval, int2 *nhdr, double *nval, cudaStream_t st) {
    const int64_t threads = 2 * M * 32;
    tw_fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, dlo, dhi, nbr_ptr, nbr, TW, ptr, dense,
                                                                     ndense, KW, NB, fhdr, fval, nhdr, nval);
}

cudaError_t launch_toeplitz(const TwArgs &g, const double *x, float *xP, double *y, int nsm, cudaStream_t st) {
    const dim3 tg((unsigned)((g.M + 31) / 32), (unsigned)((g.S + 31) / 32));
    tw_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(x, xP, (int64_t)g.nin + 2, g.M, g.S, g.PADL);
    if (g.nin <= 0) return cudaGetLastError();
    const int grid = (int)std::min<int64_t>((g.M + TW_WARPS - 1) / TW_WARPS, (int64_t)nsm * 8);
    switch (g.TW) {
        case 8: toeplitz_kernel<8><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
        case 12: toeplitz_kernel<12><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
        default: toeplitz_kernel<16><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
    }
    return cudaGetLastError();
}

}  // namespace tdbem
