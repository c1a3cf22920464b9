// Far-field quadrature in mixed precision (FP32 arithmetic, FP64 element-
// pair anchor), element pairs without a shared vertex, 7-point rule on both
// triangles (Eq. MatrixEntries).
//
// CTA = 14 warps over 32 trial triangles sigma (lanes) and the 7 test points
// x_w of the test triangle tau: warps 0..6 evaluate psi for test point w and
// keep t_b = sum_y w_y lambda_b(y) psi / r (b = 0, 1, 2) per lag slot; warps
// 7..13 evaluate psi~ for test point w - 7 and keep s~ = sum_y w_y psi~ / r.
// Both halves share the retarded argument: on an equidistant grid every
// block class sees q = r / dt in one unit cell, so one Chebyshev argument
// u = frac(q) serves every panel of every class and only the lag a panel
// feeds depends on floor(q) (Sec. 3.1, Eq. psiTildeRed); the panel
// coefficients come from the constant bank, uniform across the warp.
//
// r - R0 = (2 D.e + e.e) / (R0 + r), with D = c_tau - c_sigma and R0 = |D| in
// FP64 per element pair and e the FP32 difference of the points' offsets
// from their centroids. The CTA then forms
//   L_ab = |tau||sigma|/(4 pi) [ n_tau.n_sigma sum_x w_x lambda_a(x) t_b(x)
//                               + curl_a.curl_b sum_x w_x s~(x) ]
// per trial triangle and lag slot, and scatter_chunk adds them into the FP64
// vertex-pair lag windows (launches per colour of a vertex-disjoint
// triangle colouring: no two CTAs of a launch touch the same row).
#include <math.h>

#include "far_common.cuh"

namespace tdbem {

constexpr int F32_XW = 7;
constexpr int F32_WARPS = 2 * F32_XW;
constexpr int F32_THREADS = F32_WARPS * 32;
constexpr int F32_THREADS_ALL = F32_THREADS + 32;  // + one producer warp

struct Setup32 {
    float scale[32];
    float nn[32];
    int base[32];
    int valid[32];
    float f0[32];
    float D[32][3];
    float R0[32];
    float dqy[32][7][3];
    float curl[32][9];
};

// Chebyshev sums of NP consecutive panels (psi: COMP 0, psi~: COMP 1) at
// argument x. The terms n >= NLOW (at most a few 1e-3 of the panel maximum)
// are summed forward while the T_n recurrence runs; then the FP32 residuals
// of the leading coefficients and the terms n < NLOW are added from n =
// NLOW-1 down to 0 from the kept T_n. Small terms therefore enter before the
// large leading ones, and the rounding of the leading coefficients does not
// become a fixed perturbation of psi, which the quadrature would not average
// away and the cancellation in the odd prototype would amplify.
constexpr int NLOW = 8;
template <int NP, int COMP>
__device__ __forceinline__ void panel_values(const ChebF32 &C, int p0, float x, float *out) {
    float T[NLOW];
    T[0] = 1.f;
    T[1] = x;
    const float x2 = x + x;
#pragma unroll
    for (int n = 2; n < NLOW; ++n) T[n] = x2 * T[n - 1] - T[n - 2];
    float hi[NP];
#pragma unroll
    for (int j = 0; j < NP; ++j) hi[j] = 0.f;
    float tm = T[NLOW - 2], t = T[NLOW - 1];
#pragma unroll
    for (int n = NLOW; n < NCHEB; ++n) {
        const float tn = x2 * t - tm;
        tm = t;
        t = tn;
#pragma unroll
        for (int j = 0; j < NP; ++j) hi[j] += C.c[p0 + j][n][COMP] * tn;
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        float a = 0.f;
#pragma unroll
        for (int n = 0; n < NCHEB_LO; ++n) a += C.lo[p0 + j][n][COMP] * T[n];
        a += hi[j];
#pragma unroll
        for (int n = NLOW - 1; n >= 0; --n) a += C.c[p0 + j][n][COMP] * T[n];
        out[j] = a;
    }
}

// the ten panels of the three lag classes, sharing one recurrence
template <int COMP>
__device__ __forceinline__ void lag_panels(const ChebF32 &C, float x, float *v1, float *v2, float *v3) {
    float v[10];
    panel_values<10, COMP>(C, cls_panel0(C1), x, v);  // C1 (3), C2 (4), C3 (3) are panels 0..9
#pragma unroll
    for (int j = 0; j < 3; ++j) { v1[j] = v[j]; v3[j] = v[7 + j]; }
#pragma unroll
    for (int j = 0; j < 4; ++j) v2[j] = v[3 + j];
}

// Accumulate the P panel values of lag class CL at cell offset K = cell + OFF
// into slots slot0(CL) + K + P - 1 - j: NV = 3 (t_0, t_1, t_2) or 1 (s~).
template <int OFF, int NV, int CL, int K>
__device__ __forceinline__ void acc_lag(float (&acc)[slot0<OFF>(NLAG)][NV], const float *v, const float *f) {
    constexpr int P = cls_P(CL);
#pragma unroll
    for (int j = 0; j < P; ++j) {
        constexpr int s0 = slot0<OFF>(CL) + K + P - 1;
#pragma unroll
        for (int b = 0; b < NV; ++b) acc[s0 - j][b] += v[j] * f[b];
    }
}

template <int OFF, int NV, int K>
__device__ __forceinline__ void acc_cell(float (&acc)[slot0<OFF>(NLAG)][NV], const float *v1, const float *v2,
                                         const float *v3, const float *f) {
    acc_lag<OFF, NV, C1, K>(acc, v1, f);
    acc_lag<OFF, NV, C2, K>(acc, v2, f);
    acc_lag<OFF, NV, C3, K>(acc, v3, f);
}

template <int OFF, int NV>
__device__ __forceinline__ void acc_switch32(float (&acc)[slot0<OFF>(NLAG)][NV], int k, const float *v1,
                                             const float *v2, const float *v3, const float *f) {
    switch (k) {
        case 0: acc_cell<OFF, NV, 0>(acc, v1, v2, v3, f); break;
        case 1: acc_cell<OFF, NV, 1>(acc, v1, v2, v3, f); break;
        case 2: acc_cell<OFF, NV, 2>(acc, v1, v2, v3, f); break;
        case 3: if constexpr (OFF >= 2) acc_cell<OFF, NV, 3>(acc, v1, v2, v3, f); break;
        case 4: if constexpr (OFF >= 2) acc_cell<OFF, NV, 4>(acc, v1, v2, v3, f); break;
        case 5: if constexpr (OFF >= 3) acc_cell<OFF, NV, 5>(acc, v1, v2, v3, f); break;
        case 6: if constexpr (OFF >= 3) acc_cell<OFF, NV, 6>(acc, v1, v2, v3, f); break;
        default: break;
    }
}

// One warp role: COMP 0 (psi, NV = 3) or 1 (psi~, NV = 1). Writes its
// accumulators to red[xw][lane][slot][4] at components [COMP ? 3 : 0, ...).
template <int OFF, int COMP>
__device__ __forceinline__ void quad_role(const FarArgs &A, const ChebF32 &C, const Setup32 &su, int xw, int lane,
                                          float dx0, float dx1, float dx2, float *red) {
    constexpr int NS = slot0<OFF>(NLAG);
    constexpr int NV = COMP == 0 ? 3 : 1;
    float acc[NS][NV];
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int b = 0; b < NV; ++b) acc[s][b] = 0.f;
    const int valid = su.valid[lane];
    const float f0 = su.f0[lane], R0 = su.R0[lane];
    const float D0 = su.D[lane][0], D1 = su.D[lane][1], D2 = su.D[lane][2];
    const float inv_dt = (float)A.lt.inv_dt;
#pragma unroll 1
    for (int y = 0; y < 7; ++y) {
        const float e0 = dx0 - su.dqy[lane][y][0];
        const float e1 = dx1 - su.dqy[lane][y][1];
        const float e2 = dx2 - su.dqy[lane][y][2];
        const float sv = 2.f * (D0 * e0 + D1 * e1 + D2 * e2) + (e0 * e0 + e1 * e1 + e2 * e2);
        const float dr = sv * __frcp_rn(R0 + sqrtf(fmaxf(R0 * R0 + sv, 0.f)));
        const float ir = __frcp_rn(R0 + dr);
        const float q = f0 + dr * inv_dt;
        const float cf = floorf(q);
        int cell = (int)cf;
        const float u = q - cf;
        const float x = u + u - 1.f;
        const float wr = valid ? A.rw32[y] * ir : 0.f;
        float f[NV];
        if constexpr (COMP == 0) {
            f[0] = wr * A.rl32[3 * y]; f[1] = wr * A.rl32[3 * y + 1]; f[2] = wr * A.rl32[3 * y + 2];
        } else {
            f[0] = wr;
        }
        if (cell < -OFF || cell > OFF) {
            if (valid) A.status[0] = ST_OFF_RANGE;
            cell = 0;
        }
        float v1[3], v2[4], v3[3];
        lag_panels<COMP>(C, x, v1, v2, v3);
        acc_switch32<OFF, NV>(acc, cell + OFF, v1, v2, v3, f);
    }
    float *rp = red + ((size_t)(xw * 32 + lane) * NS) * 4 + (COMP == 0 ? 0 : 3);
#pragma unroll
    for (int s = 0; s < NS; ++s)
#pragma unroll
        for (int b = 0; b < NV; ++b) rp[4 * s + b] = acc[s][b];
}

// Element-pair setup of one chunk (32 trial triangles) for test triangle tau:
// FP64 centroid distance, lag base and fraction, FP32 anchor, trial points
// and curls.
__device__ __forceinline__ void chunk_setup(const FarArgs &A, int64_t tau, int64_t ch, int lane, Setup32 &su) {
    const Geo &g = A.g;
    const int64_t E = g.E;
    const int64_t sg = ch * 32 + lane;
    const int32_t Ft0 = g.F[3 * tau], Ft1 = g.F[3 * tau + 1], Ft2 = g.F[3 * tau + 2];
    int valid = 0, base = 0;
    float f0 = 0.f, R0 = 1.f, D0 = 0.f, D1 = 0.f, D2 = 0.f, scale = 0.f, nn = 0.f;
    if (sg < E) {
        const int32_t *B = g.F + 3 * sg;
        int shared = 0;
        for (int b = 0; b < 3; ++b) shared += (B[b] == Ft0) + (B[b] == Ft1) + (B[b] == Ft2);
        valid = shared == 0;
        const double d0 = g.cen[3 * tau] - g.cen[3 * sg];
        const double d1 = g.cen[3 * tau + 1] - g.cen[3 * sg + 1];
        const double d2 = g.cen[3 * tau + 2] - g.cen[3 * sg + 2];
        const double r0 = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
        const double q0 = r0 * A.lt.inv_dt;
        const double fb = floor(q0);
        base = (int)fb;
        f0 = (float)(q0 - fb);
        R0 = (float)r0; D0 = (float)d0; D1 = (float)d1; D2 = (float)d2;
        const float *gt = g.geo32 + 16 * tau, *gs = g.geo32 + 16 * sg;
        scale = gt[3] * gs[3] * 0.07957747f;  // 1/(4 pi)
        nn = gt[0] * gs[0] + gt[1] * gs[1] + gt[2] * gs[2];
        for (int k = 0; k < 9; ++k) su.curl[lane][k] = gs[4 + k];
        for (int k = 0; k < 21; ++k) su.dqy[lane][k / 3][k % 3] = g.dq32[sg * 21 + k];
    } else {
        for (int k = 0; k < 9; ++k) su.curl[lane][k] = 0.f;
        for (int k = 0; k < 21; ++k) su.dqy[lane][k / 3][k % 3] = 0.f;
    }
    su.valid[lane] = valid; su.base[lane] = base; su.f0[lane] = f0; su.R0[lane] = R0;
    su.D[lane][0] = D0; su.D[lane][1] = D1; su.D[lane][2] = D2;
    su.scale[lane] = scale; su.nn[lane] = nn;
}

// Special blocks (cell 0 and the first/last-row corner) are not evaluated
// here: the few far pairs that reach them go through the FP64 pass in near.cu.
// Warps 0..13 compute (two roles x seven test points); warp 14 prepares the
// next chunk's setup in the other buffer while they do, so the FP64 setup
// and its loads stay off the critical path.
template <int OFF>
__global__ void __launch_bounds__(F32_THREADS_ALL, 1)
far32_kernel(const FarArgs A, const __grid_constant__ ChebF32 C) {
    constexpr int NS = slot0<OFF>(NLAG);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Setup32 *sub = reinterpret_cast<Setup32 *>(smem_raw);                                       // [2]
    float *red = reinterpret_cast<float *>(smem_raw + ((2 * sizeof(Setup32) + 15) / 16) * 16);  // [7][32][NS][4]
    float *Lb = red + (size_t)F32_XW * 32 * NS * 4;                                             // [32][NS][9]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = w == F32_WARPS;
    const int role = w / F32_XW, xw = w % F32_XW;
    const Geo &g = A.g;
    const int64_t nch = A.nchunks;
    // flattened sequence of (tau, chunk) items of this CTA
    const int64_t ntau = A.ncolor > blockIdx.x ? (A.ncolor - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nit = ntau * nch;
    if (nit == 0) return;
    if (producer) chunk_setup(A, A.color_tris[blockIdx.x], 0, lane, sub[0]);
    __syncthreads();
    int64_t cur_tau = -1;
    int32_t Ft0 = 0, Ft1 = 0, Ft2 = 0;
    float dx0 = 0.f, dx1 = 0.f, dx2 = 0.f;
    for (int64_t it = 0; it < nit; ++it) {
        const int64_t tix = it / nch, ch = it % nch;
        const int64_t tau = A.color_tris[blockIdx.x + tix * gridDim.x];
        Setup32 &su = sub[it & 1];
        if (tau != cur_tau) {
            cur_tau = tau;
            Ft0 = g.F[3 * tau]; Ft1 = g.F[3 * tau + 1]; Ft2 = g.F[3 * tau + 2];
            if (!producer) {
                dx0 = g.dq32[(tau * 7 + xw) * 3 + 0];
                dx1 = g.dq32[(tau * 7 + xw) * 3 + 1];
                dx2 = g.dq32[(tau * 7 + xw) * 3 + 2];
            }
        }
        if (producer) {
            if (it + 1 < nit) {
                const int64_t t2 = A.color_tris[blockIdx.x + ((it + 1) / nch) * gridDim.x];
                chunk_setup(A, t2, (it + 1) % nch, lane, sub[(it + 1) & 1]);
            }
        } else {
            if (role == 0) quad_role<OFF, 0>(A, C, su, xw, lane, dx0, dx1, dx2, red);
            else quad_role<OFF, 1>(A, C, su, xw, lane, dx0, dx1, dx2, red);
        }
        __syncthreads();
        // ---- sum over the 7 test points -> local 3x3 per (sigma, slot)
        for (int k = threadIdx.x; k < 32 * NS; k += F32_THREADS_ALL) {
            const int sl = k / NS, s = k % NS;
            float Sab[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, St = 0.f;
#pragma unroll
            for (int x = 0; x < 7; ++x) {
                const float *q = red + ((size_t)(x * 32 + sl) * NS + s) * 4;
                const float wx = A.rw32[x];
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    const float ga = wx * A.rl32[3 * x + a];
#pragma unroll
                    for (int b = 0; b < 3; ++b) Sab[a][b] += ga * q[b];
                }
                St += wx * q[3];
            }
            const float *gt = g.geo32 + 16 * tau + 4, *gs = su.curl[sl];
            const float sc = su.scale[sl], nn = su.nn[sl];
            float *lp = Lb + ((size_t)sl * NS + s) * 9;
#pragma unroll
            for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int b = 0; b < 3; ++b) {
                    const float cc = gt[3 * a] * gs[3 * b] + gt[3 * a + 1] * gs[3 * b + 1] + gt[3 * a + 2] * gs[3 * b + 2];
                    lp[3 * a + b] = sc * (nn * Sab[a][b] + cc * St);
                }
        }
        __syncthreads();
        scatter_chunk<float, OFF, F32_THREADS_ALL, Setup32, false>(A, ch, Ft0, Ft1, Ft2, su, Lb);
        __syncthreads();
    }
}

template <int OFF>
static void launch32(const FarArgs &a, const ChebF32 &c32, int grid, cudaStream_t st) {
    constexpr int NS = slot0<OFF>(NLAG);
    const size_t smem = ((2 * sizeof(Setup32) + 15) / 16) * 16 + sizeof(float) * ((size_t)F32_XW * 32 * NS * 4 + 32 * NS * 9);
    cudaFuncSetAttribute(far32_kernel<OFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    far32_kernel<OFF><<<grid, F32_THREADS_ALL, smem, st>>>(a, c32);
}

void launch_far32(const FarArgs &a, const ChebF32 &c32, int off, int grid, cudaStream_t st) {
    if (off == 1) launch32<1>(a, c32, grid, st);
    else if (off == 2) launch32<2>(a, c32, grid, st);
    else launch32<3>(a, c32, grid, st);
}

}  // namespace tdbem
