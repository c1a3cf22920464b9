// Far-field quadrature in mixed precision (FP32 arithmetic, FP64 element-
// pair anchor), element pairs without a shared vertex, 7-point rule on both
// triangles (Eq. MatrixEntries).
//
// CTA = 7 compute warps over 32 trial triangles sigma (lanes) and the 7 test
// points x_w of the test triangle tau (warp w), plus one producer warp that
// prepares the next chunk's FP64 setup in a second buffer.
//
// Every block class shares the retarded argument: on an equidistant grid all
// classes see q = r / dt in one unit cell, so one Chebyshev argument
// u = frac(q) serves every panel of every class and only the lag a panel
// feeds depends on floor(q) (Sec. 3.1, Eq. psiTildeRed). A thread evaluates
// psi and psi~ of a panel together as one packed FP32 pair (fma.rn.f32x2):
// the coefficients are stored as (psi, psi~) pairs, so one instruction adds a
// Chebyshev term of both functions, and the distance and T_n are computed
// once per point pair. It keeps, per lag slot, the pairs
//   (t_0, t_1) and (t_2, s~),  t_b = sum_y w_y lambda_b(y) psi / r,
//                              s~  = sum_y w_y psi~ / r.
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
constexpr int F32_THREADS_ALL = (F32_XW + 1) * 32;

typedef unsigned long long f2;  // two packed floats (lo, hi)

__device__ __forceinline__ f2 pk(float lo, float hi) {
    f2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void upk(f2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// d = a * b + c on both halves, round to nearest
__device__ __forceinline__ f2 fma2(f2 a, f2 b, f2 c) {
    f2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ f2 coef2(const ChebF32 &C, int p, int n) {
    return *reinterpret_cast<const f2 *>(&C.c[p][n][0]);
}
__device__ __forceinline__ f2 lo2(const ChebF32 &C, int p, int n) {
    return *reinterpret_cast<const f2 *>(&C.lo[p][n][0]);
}

struct Setup32 {
    int64_t tau, ch;
    int32_t Ft[3];
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

// (psi, psi~) of the ten lag-class panels (C1: 3, C2: 4, C3: 3) at argument
// x, sharing one T_n recurrence. The terms n >= NLOW (at most a few 1e-3 of
// the panel maximum) are summed forward while the recurrence runs; then the
// FP32 residuals of the leading coefficients and the terms n < NLOW are added
// from n = NLOW-1 down to 0 from the kept T_n. Small terms therefore enter
// before the large leading ones, and the rounding of the leading coefficients
// does not become a fixed perturbation of psi, which the quadrature would not
// average away and the cancellation in the odd prototype would amplify.
constexpr int NLOW = 8;
__device__ __forceinline__ void lag_panels(const ChebF32 &C, float x, f2 (&v)[10]) {
    f2 T[NLOW];
    float t0 = 1.f, t1 = x;
    const float x2 = x + x;
    T[0] = pk(1.f, 1.f);
    T[1] = pk(x, x);
#pragma unroll
    for (int n = 2; n < NLOW; ++n) {
        const float tn = x2 * t1 - t0;
        t0 = t1;
        t1 = tn;
        T[n] = pk(tn, tn);
    }
    f2 hi[10];
#pragma unroll
    for (int j = 0; j < 10; ++j) hi[j] = 0ull;
#pragma unroll
    for (int n = NLOW; n < NCHEB; ++n) {
        const float tn = x2 * t1 - t0;
        t0 = t1;
        t1 = tn;
        const f2 tt = pk(tn, tn);
#pragma unroll
        for (int j = 0; j < 10; ++j) hi[j] = fma2(coef2(C, j, n), tt, hi[j]);
    }
#pragma unroll
    for (int j = 0; j < 10; ++j) {
        f2 a = 0ull;
#pragma unroll
        for (int n = 0; n < NCHEB_LO; ++n) a = fma2(lo2(C, j, n), T[n], a);
        a = fma2(pk(1.f, 1.f), hi[j], a);
#pragma unroll
        for (int n = NLOW - 1; n >= 0; --n) a = fma2(coef2(C, j, n), T[n], a);
        v[j] = a;
    }
}

// Accumulate the P panels of lag class CL at cell offset K = cell + OFF: slot
// slot0(CL) + K + P - 1 - j gets (t_0, t_1) += psi (F_0, F_1) and
// (t_2, s~) += (psi, psi~) (F_2, w r^-1), with F_b = w r^-1 lambda_b(y).
template <int OFF, int CL, int K>
__device__ __forceinline__ void accp(f2 (&a01)[slot0<OFF>(NLAG)], f2 (&a2s)[slot0<OFF>(NLAG)], const f2 (&v)[10],
                                     f2 F01, f2 F2W) {
    constexpr int P = cls_P(CL);
    constexpr int pj = cls_panel0(CL);
#pragma unroll
    for (int j = 0; j < P; ++j) {
        constexpr int s0 = slot0<OFF>(CL) + K + P - 1;
        float ps, pt;
        upk(v[pj + j], ps, pt);
        a01[s0 - j] = fma2(pk(ps, ps), F01, a01[s0 - j]);
        a2s[s0 - j] = fma2(v[pj + j], F2W, a2s[s0 - j]);
    }
}

template <int OFF, int K>
__device__ __forceinline__ void accp_cell(f2 (&a01)[slot0<OFF>(NLAG)], f2 (&a2s)[slot0<OFF>(NLAG)], const f2 (&v)[10],
                                          f2 F01, f2 F2W) {
    accp<OFF, C1, K>(a01, a2s, v, F01, F2W);
    accp<OFF, C2, K>(a01, a2s, v, F01, F2W);
    accp<OFF, C3, K>(a01, a2s, v, F01, F2W);
}

// Quadrature of one (test point x_w, trial triangle = lane) pair over the 7
// trial points; writes red[xw][lane][slot][0..3] = (t_0, t_1, t_2, s~).
template <int OFF>
__device__ __forceinline__ void quad_packed(const FarArgs &A, const ChebF32 &C, const Setup32 &su, int xw, int lane,
                                            float dx0, float dx1, float dx2, float *red) {
    constexpr int NS = slot0<OFF>(NLAG);
    f2 a01[NS], a2s[NS];
#pragma unroll
    for (int s = 0; s < NS; ++s) { a01[s] = 0ull; a2s[s] = 0ull; }
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
        const f2 F01 = pk(wr * A.rl32[3 * y], wr * A.rl32[3 * y + 1]);
        const f2 F2W = pk(wr * A.rl32[3 * y + 2], wr);
        if (cell < -OFF || cell > OFF) {
            if (valid) A.status[0] = ST_OFF_RANGE;
            cell = 0;
        }
        f2 v[10];
        lag_panels(C, x, v);
        switch (cell + OFF) {
            case 0: accp_cell<OFF, 0>(a01, a2s, v, F01, F2W); break;
            case 1: accp_cell<OFF, 1>(a01, a2s, v, F01, F2W); break;
            case 2: accp_cell<OFF, 2>(a01, a2s, v, F01, F2W); break;
            case 3: if constexpr (OFF >= 2) accp_cell<OFF, 3>(a01, a2s, v, F01, F2W); break;
            case 4: if constexpr (OFF >= 2) accp_cell<OFF, 4>(a01, a2s, v, F01, F2W); break;
            case 5: if constexpr (OFF >= 3) accp_cell<OFF, 5>(a01, a2s, v, F01, F2W); break;
            case 6: if constexpr (OFF >= 3) accp_cell<OFF, 6>(a01, a2s, v, F01, F2W); break;
            default: break;
        }
    }
    f2 *rp = reinterpret_cast<f2 *>(red + ((size_t)(xw * 32 + lane) * NS) * 4);
#pragma unroll
    for (int s = 0; s < NS; ++s) { rp[2 * s] = a01[s]; rp[2 * s + 1] = a2s[s]; }
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
    if (lane == 0) { su.tau = tau; su.ch = ch; su.Ft[0] = Ft0; su.Ft[1] = Ft1; su.Ft[2] = Ft2; }
}

// Special blocks (cell 0 and the first/last-row corner) are not evaluated
// here: the few far pairs that reach them go through the FP64 pass in near.cu.
template <int OFF>
__global__ void __launch_bounds__(F32_THREADS_ALL, 1)
far32_kernel(const FarArgs A, const __grid_constant__ ChebF32 C) {
    constexpr int NS = slot0<OFF>(NLAG);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    Setup32 *sub = reinterpret_cast<Setup32 *>(smem_raw);                                       // [2]
    float *red = reinterpret_cast<float *>(smem_raw + ((2 * sizeof(Setup32) + 15) / 16) * 16);  // [7][32][NS][4]
    float *Lb = red + (size_t)F32_XW * 32 * NS * 4;                                             // [32][NS][9]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = w == F32_XW;
    const int xw = w;
    const Geo &g = A.g;
    const int64_t nch = A.nchunks;
    const int64_t ntau = A.ncolor > blockIdx.x ? (A.ncolor - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nit = ntau * nch;
    if (nit == 0) return;
    if (producer) chunk_setup(A, A.color_tris[blockIdx.x], 0, lane, sub[0]);
    __syncthreads();
    int64_t cur_tau = -1;
    float dx0 = 0.f, dx1 = 0.f, dx2 = 0.f;
    for (int64_t it = 0; it < nit; ++it) {
        Setup32 &su = sub[it & 1];
        if (producer) {
            if (it + 1 < nit) {
                const int64_t t2 = A.color_tris[blockIdx.x + ((it + 1) / nch) * gridDim.x];
                chunk_setup(A, t2, (it + 1) % nch, lane, sub[(it + 1) & 1]);
            }
        } else {
            if (su.tau != cur_tau) {
                cur_tau = su.tau;
                dx0 = g.dq32[(cur_tau * 7 + xw) * 3 + 0];
                dx1 = g.dq32[(cur_tau * 7 + xw) * 3 + 1];
                dx2 = g.dq32[(cur_tau * 7 + xw) * 3 + 2];
            }
            quad_packed<OFF>(A, C, su, xw, lane, dx0, dx1, dx2, red);
        }
        __syncthreads();
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
            const float *gt = g.geo32 + 16 * su.tau + 4, *gs = su.curl[sl];
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
        scatter_chunk<float, OFF, F32_THREADS_ALL, Setup32, false>(A, su.ch, su.Ft[0], su.Ft[1], su.Ft[2], su, Lb);
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
