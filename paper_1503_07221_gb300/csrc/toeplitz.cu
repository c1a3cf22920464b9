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
// This file stores every window as one entry of TL lags (TL the smallest of
// 8, 9, 10, 12, 16 that holds the widest window; the assembler keeps windows
// of at most 16 lags): the pair's trial vertex j, the first lag, and TL
// values, zero past the end of the window. The far values are FP32
// (the CSR values of the mixed path, hi + lo of the accumulated pair), the
// near values FP64.
//
// One warp handles one test vertex l and a chunk of 128 outputs u. With R
// outputs per lane (R = 4, 8 or 16, the autotuner's choice), 128 / R lanes
// share one entry and the warp applies R / 4 entries at a time. For an entry
// (j, a) the R outputs of a lane meet x_j at the R + TL - 1 consecutive
// inner time indices starting at u - a - (TL - 1); the padded FP32 copy of x
// is kept four times, shifted by 0..3 floats, so that this window is read
// with aligned float4 loads from the copy that matches its start (the same
// code for every entry, no branch on the alignment), with zeros outside the
// inner indices so that the bounds need no test. All TL lags are then applied
// from registers: each x value is read once per vertex pair and used for up
// to R TL products, where the per-block CSR product reads it once per (pair,
// lag) and position run. Far products are FP32 and summed in FP32 over four
// steps (at most 4 TL products per output), and these partial sums are
// accumulated as FP32 pairs with an error-free two-sum; near products and
// sums, and the sum over the entries applied side by side, are FP64.
// Each y entry is written by its own warp only, after the product of the
// other blocks has written it: the result is deterministic.
#include "tdbem_internal.h"

namespace tdbem {

constexpr int TW_WARPS = 8;

// X[j][q] = x[(q - PADL + 1) M + j] rounded to FP32 for q - PADL in the inner
// time indices 0 .. N - 3, zero at every other q < S; copy c (blockIdx.z)
// holds X shifted by c: xP[c M S + j S + q] = X[j][q + c] (zero past S)
__global__ void __launch_bounds__(256) tw_transpose_kernel(const double *__restrict__ x, float *__restrict__ xP,
                                                           int64_t N, int64_t M, int S, int PADL) {
    __shared__ float tile[32][33];
    const int64_t j0 = (int64_t)blockIdx.x * 32;
    const int q0 = blockIdx.y * 32, c = blockIdx.z;
    const int tx = threadIdx.x, ty = threadIdx.y;  // 32 x 8
    const int64_t nin = N - 2;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int q = q0 + ty + 8 * s + c;
        const int64_t ci = (int64_t)q - PADL;
        float v = 0.f;
        if (q < S && ci >= 0 && ci < nin && j0 + tx < M) v = (float)x[(ci + 1) * M + j0 + tx];
        tile[ty + 8 * s][tx] = v;
    }
    __syncthreads();
    float *dst = xP + (int64_t)c * M * S;
#pragma unroll
    for (int s = 0; s < 4; ++s) {
        const int64_t j = j0 + ty + 8 * s;
        const int q = q0 + tx;
        if (j < M && q < S) dst[j * S + q] = tile[tx][ty + 8 * s];
    }
}

// ------------------------------------------------------------ layout build
// Entries per row: set 0 = far (every trial vertex j), set 1 = near (the
// neighbour list of l); one entry per pair with a non-empty window [a, b].
// *maxw: the widest window (b - a + 1) of either set. One warp per (set, row).
__global__ void tw_count_kernel(int64_t M, const int16_t *__restrict__ dlo, const int16_t *__restrict__ dhi,
                                const int64_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr,
                                int64_t *__restrict__ cnt, unsigned long long *__restrict__ maxw) {
    const int lane = threadIdx.x & 31;
    const int64_t item = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (item >= 2 * M) return;
    const int set = (int)(item / M);
    const int64_t l = item % M;
    const int64_t k0 = set ? nbr_ptr[l] : 0, k1 = set ? nbr_ptr[l + 1] : M;
    int64_t n = 0;
    int wmax = 0;
    for (int64_t k = k0 + lane; k < k1; k += 32) {
        const int64_t j = set ? nbr[k] : k;
        const int a = dlo[l * M + j], b = dhi[l * M + j];
        if (a <= b) {
            ++n;
            wmax = max(wmax, b - a + 1);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        n += __shfl_xor_sync(0xffffffffu, n, o);
        wmax = max(wmax, __shfl_xor_sync(0xffffffffu, wmax, o));
    }
    if (lane == 0) {
        cnt[set * M + l] = n;
        if (wmax > 0) atomicMax(maxw, (unsigned long long)wmax);
    }
}

// Entries of row l in order of the trial vertex; the positions come from
// an exclusive scan of the counts (ptr, 2 x (M + 1)). Every window fits in
// TL lags; an entry holds its TL values at stride TS (zero past the window).
// dense: the far windows of the class, FP32 pairs (hi, lo) at
// ((l M + j) KW + d - a); ndense: the near windows, FP64 at
// ((l NB + k - nbr_ptr[l]) KW + d - a).
__global__ void tw_fill_kernel(int64_t M, const int16_t *__restrict__ dlo, const int16_t *__restrict__ dhi,
                               const int64_t *__restrict__ nbr_ptr, const int32_t *__restrict__ nbr, int TL, int TS,
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
        const bool in = a <= b;
        const unsigned bal = __ballot_sync(0xffffffffu, in);
        if (in) {
            const int64_t e = pos + __popc(bal & ((1u << lane) - 1u));
            if (set == 0) {
                fhdr[e] = make_int2((int)j, a);
                const float2 *w = dense + (l * M + j) * KW;
                for (int t = 0; t < TS; ++t) fval[e * TS + t] = (t < TL && a + t <= b) ? w[t].x + w[t].y : 0.f;
            } else {
                nhdr[e] = make_int2((int)j, a);
                const double *w = ndense + (l * NB + (k - k0)) * KW;
                for (int t = 0; t < TS; ++t) nval[e * TS + t] = (t < TL && a + t <= b) ? w[t] : 0.0;
            }
        }
        pos += __popc(bal);
    }
}

// ------------------------------------------------------------ product
template <int TL, int R>
struct TwCfg {
    static constexpr int TS = (TL + 3) / 4 * 4;        // stored values per entry
    static constexpr int LPE = 128 / R;                // lanes per entry
    static constexpr int EPW = 32 / LPE;               // entries a warp applies at once
    static constexpr int NV4 = (R + TL - 1 + 3) / 4;   // float4 loads of one window
    static constexpr int NVF = 4 * NV4;
};

// acc[r] += sum_t a[t] v[TL - 1 + r - t]: output u + r, lag a0 + t
template <int TL, int R, typename T, typename A>
__device__ __forceinline__ void tw_fma(const float (&v)[TwCfg<TL, R>::NVF], const A (&a)[TL], T (&acc)[R]) {
#pragma unroll
    for (int t = 0; t < TL; ++t)
#pragma unroll
        for (int r = 0; r < R; ++r) acc[r] = fma((T)a[t], (T)v[TL - 1 + r - t], acc[r]);
}

// v[i] = X[j][base + i]: aligned float4 loads from the copy shifted by base mod 4
template <int TL, int R>
__device__ __forceinline__ void tw_window(const float *__restrict__ xP, int64_t MS, int S, int j, int base,
                                          float (&v)[TwCfg<TL, R>::NVF]) {
    const int c = base & 3;
    const float4 *r4 = reinterpret_cast<const float4 *>(xP + c * MS + (int64_t)j * S + (base - c));
#pragma unroll
    for (int q = 0; q < TwCfg<TL, R>::NV4; ++q) {
        const float4 t = __ldg(r4 + q);
        v[4 * q] = t.x;
        v[4 * q + 1] = t.y;
        v[4 * q + 2] = t.z;
        v[4 * q + 3] = t.w;
    }
}

__device__ __forceinline__ void two_sum_add(float &h, float &l, float v) {
    const float s = h + v;
    const float bb = s - h;
    l += (h - (s - bb)) + (v - bb);
    h = s;
}

// Far entries are taken 32 at a time: their headers into registers (one per
// lane) and their values into the warp's slice of shared memory, both with
// coalesced loads, so that applying an entry waits on no global value load.
template <int TL, int R>
__global__ void __launch_bounds__(TW_WARPS * 32) toeplitz_kernel(TwArgs g, const float *__restrict__ xP,
                                                                 double *__restrict__ y) {
    typedef TwCfg<TL, R> C;
    __shared__ __align__(16) float sval_all[TW_WARPS][32 * C::TS];
    const int lane = threadIdx.x & 31, sub = lane % C::LPE, grp = lane / C::LPE;
    float *sval = sval_all[threadIdx.x >> 5];
    const int64_t nwarp = (int64_t)gridDim.x * TW_WARPS, MS = g.M * (int64_t)g.S;
    const int nin = g.nin;
    for (int64_t l = (int64_t)blockIdx.x * TW_WARPS + (threadIdx.x >> 5); l < g.M; l += nwarp) {
        for (int u0 = 0; u0 < nin; u0 += 128) {
            const int lb = g.PADL + u0 + R * sub - (TL - 1);
            float acc[R], ph[R], pl[R];
#pragma unroll
            for (int r = 0; r < R; ++r) acc[r] = ph[r] = pl[r] = 0.f;
            const int64_t e0 = g.fptr[l], e1 = g.fptr[l + 1];
            int pend = 0;
            for (int64_t eb = e0; eb < e1; eb += 32) {
                const int ne = (int)min((int64_t)32, e1 - eb);
                int2 hv = make_int2(0, 0);
                __syncwarp();
                if (lane < ne) {
                    hv = g.fhdr[eb + lane];
                    const float4 *src = reinterpret_cast<const float4 *>(g.fval + (eb + lane) * C::TS);
                    float4 *dst = reinterpret_cast<float4 *>(sval + lane * C::TS);
#pragma unroll
                    for (int q = 0; q < C::TS / 4; ++q) dst[q] = __ldg(src + q);
                }
                __syncwarp();
                for (int t0 = 0; t0 < ne; t0 += C::EPW) {
                    const int t = t0 + grp;
                    const int j = __shfl_sync(0xffffffffu, hv.x, min(t, 31));
                    const int a0 = __shfl_sync(0xffffffffu, hv.y, min(t, 31));
                    // outputs of this chunk all below the window, or all past it
                    if (t < ne && a0 <= u0 + 127 && u0 - (a0 + TL - 1) <= nin - 1) {
                        float v[C::NVF];
                        tw_window<TL, R>(xP, MS, g.S, j, lb - a0, v);
                        float a[TL];
                        const float *sv = sval + t * C::TS;
#pragma unroll
                        for (int q = 0; q < TL; ++q) a[q] = sv[q];
                        tw_fma<TL, R>(v, a, acc);
                    }
                    if (++pend == 4) {
#pragma unroll
                        for (int r = 0; r < R; ++r) {
                            two_sum_add(ph[r], pl[r], acc[r]);
                            acc[r] = 0.f;
                        }
                        pend = 0;
                    }
                }
            }
            double out[R];
#pragma unroll
            for (int r = 0; r < R; ++r) {
                two_sum_add(ph[r], pl[r], acc[r]);
                out[r] = (double)ph[r] + (double)pl[r];
            }
            // near entries: FP64 values and sums
            const int64_t n0 = g.nptr[l], n1 = g.nptr[l + 1];
            for (int64_t ebn = n0; ebn < n1; ebn += C::EPW) {
                const int64_t e = ebn + grp;
                if (e >= n1) continue;
                const int2 h = g.nhdr[e];
                if (h.y > u0 + 127 || u0 - (h.y + TL - 1) > nin - 1) continue;
                double a[TL];
#pragma unroll
                for (int t = 0; t < TL; ++t) a[t] = g.nval[e * C::TS + t];
                float v[C::NVF];
                tw_window<TL, R>(xP, MS, g.S, h.x, lb - h.y, v);
                tw_fma<TL, R>(v, a, out);
            }
            // sum over the entries applied side by side, then each lane writes 4 outputs
#pragma unroll
            for (int o = C::LPE; o < 32; o <<= 1)
#pragma unroll
                for (int r = 0; r < R; ++r) out[r] += __shfl_xor_sync(0xffffffffu, out[r], o);
#pragma unroll
            for (int r = 0; r < R; ++r) {
                const int u = u0 + R * sub + r;
                if (r / 4 == grp && u < nin) y[(int64_t)(u + 1) * g.M + l] += out[r];
            }
        }
    }
}

int tw_lags(int maxw) {
    static const int opts[] = {8, 9, 10, 12, 16};
    for (int o : opts)
        if (maxw <= o) return o;
    return -1;
}

int tw_variant_outputs(int variant) { return variant % 3 == 0 ? 4 : (variant % 3 == 1 ? 8 : 16); }

void tw_geometry(int TL, int max_lag, int N, int *PADL, int *S) {
    const int nch = (N - 2 + 127) / 128;
    *PADL = (max_lag + TL + 3) / 4 * 4;
    *S = (*PADL + 128 * nch + 8 + 3) / 4 * 4;
}

void launch_tw_count(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                     int64_t *cnt, unsigned long long *maxw, cudaStream_t st) {
    const int64_t threads = 2 * M * 32;
    tw_count_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, dlo, dhi, nbr_ptr, nbr, cnt, maxw);
}

void launch_tw_fill(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                    int TL, const int64_t *ptr, const float2 *dense, const double *ndense, int KW, int NB, int2 *fhdr,
                    float *fval, int2 *nhdr, double *nval, cudaStream_t st) {
    const int64_t threads = 2 * M * 32;
    tw_fill_kernel<<<(unsigned)((threads + 255) / 256), 256, 0, st>>>(M, dlo, dhi, nbr_ptr, nbr, TL, (TL + 3) / 4 * 4,
                                                                     ptr, dense, ndense, KW, NB, fhdr, fval, nhdr,
                                                                     nval);
}

template <int TL>
static void launch_tw_shape(const TwArgs &g, const float *xP, double *y, int R, int grid, cudaStream_t st) {
    switch (R) {
        case 4: toeplitz_kernel<TL, 4><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
        case 8: toeplitz_kernel<TL, 8><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
        default: toeplitz_kernel<TL, 16><<<grid, TW_WARPS * 32, 0, st>>>(g, xP, y); break;
    }
}

cudaError_t launch_toeplitz(const TwArgs &g, const double *x, float *xP, double *y, int R, int nsm, cudaStream_t st) {
    const dim3 tg((unsigned)((g.M + 31) / 32), (unsigned)((g.S + 31) / 32), 4);
    tw_transpose_kernel<<<tg, dim3(32, 8), 0, st>>>(x, xP, (int64_t)g.nin + 2, g.M, g.S, g.PADL);
    if (g.nin <= 0) return cudaGetLastError();
    const int grid = (int)std::min<int64_t>((g.M + TW_WARPS - 1) / TW_WARPS, (int64_t)nsm * 8);
    switch (g.TL) {
        case 8: launch_tw_shape<8>(g, xP, y, R, grid, st); break;
        case 9: launch_tw_shape<9>(g, xP, y, R, grid, st); break;
        case 10: launch_tw_shape<10>(g, xP, y, R, grid, st); break;
        case 12: launch_tw_shape<12>(g, xP, y, R, grid, st); break;
        default: launch_tw_shape<16>(g, xP, y, R, grid, st); break;
    }
    return cudaGetLastError();
}

}  // namespace tdbem
