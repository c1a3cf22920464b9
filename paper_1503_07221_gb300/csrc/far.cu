// Far-field quadrature (element pairs without a shared vertex) of Eq.
// MatrixEntries with the 7-point degree-5 triangle rule on both triangles.
//
// CTA = 7 warps: warp w owns quadrature point x_w of the test triangle tau,
// lane s owns trial triangle sigma = chunk * 32 + s. For each of the 7 trial
// points y, a thread evaluates every panel of every block class at one
// Chebyshev argument: on an equidistant grid all blocks see q = r / dt in
// the same unit cell, so the local argument u = frac(q) is shared and only
// the lag that a panel feeds depends on floor(q) (Sec. 3.1, Eq.
// psiTildeRed). The panels' coefficients are therefore uniform across the
// warp (constant bank in the FP32 path). Per lag slot the thread keeps
//   t_b = sum_y w_y lambda_b(y) psi / r  (b = 0, 1, 2),
//   s~  = sum_y w_y psi~ / r,
// and the CTA forms the local 3x3 matrix
//   L_ab = |tau||sigma|/(4 pi) [ n_tau.n_sigma sum_x w_x lambda_a(x) t_b(x)
//                               + curl_a.curl_b sum_x w_x s~(x) ].
// The sum over the triangles sharing a trial vertex is reduced in shared
// memory with a host-built per-chunk plan and added (read-modify-write,
// no atomics) into the FP64 vertex-pair lag windows of the test triangle's
// three rows, so the long sums over test triangles and chunks do not
// accumulate FP32 rounding. Launches are per colour of a vertex-disjoint triangle colouring, so
// no two CTAs of a launch touch the same row.
#include <math.h>

#include "far_common.cuh"

namespace tdbem {

// Chebyshev coefficient of panel p, sub-panel sub, index n, component k.
template <typename R>
__device__ __forceinline__ R coef(const ChebF32 &c32, const double *c64, int S, int sub, int p, int n, int k);
template <>
__device__ __forceinline__ float coef<float>(const ChebF32 &c32, const double *, int, int, int p, int n, int k) {
    return c32.c[p][n][k];
}
template <>
__device__ __forceinline__ double coef<double>(const ChebF32 &, const double *c64, int S, int sub, int p, int n, int k) {
    return __ldg(c64 + (((size_t)(p * S + sub) * NCHEB + n) * 2 + k));
}

// Dot products of the panels [p0, p0 + NP) at Chebyshev argument x:
// out[2 j + k] = sum_n c_{p0+j, n, k} T_n(x). In FP32 the T_n are kept and
// each sum runs from n = 32 down to 0, so the small high-order terms are
// added before the large leading ones (a third of the rounding error of the
// forward order at the same number of FMAs), and it starts from the FP32
// residuals of the leading coefficients: their rounding would otherwise be a
// fixed perturbation of psi, which the quadrature does not average away and
// the cancellation in the odd prototype amplifies.
template <typename R, int NP>
__device__ __forceinline__ void cheb_dots(const ChebF32 &c32, const double *c64, int S, int sub,
                                          int p0, R x, R out[2 * NP]) {
    if constexpr (sizeof(R) == 4) {
        R T[NCHEB];
        T[0] = R(1);
        T[1] = x;
        const R x2 = x + x;
#pragma unroll
        for (int n = 2; n < NCHEB; ++n) T[n] = x2 * T[n - 1] - T[n - 2];
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            R a = R(0), b = R(0);
#pragma unroll
            for (int n = 0; n < NCHEB_LO; ++n) {
                a += c32.lo[p0 + j][n][0] * T[n];
                b += c32.lo[p0 + j][n][1] * T[n];
            }
#pragma unroll
            for (int n = NCHEB - 1; n >= 0; --n) {
                a += coef<R>(c32, c64, S, sub, p0 + j, n, 0) * T[n];
                b += coef<R>(c32, c64, S, sub, p0 + j, n, 1) * T[n];
            }
            out[2 * j] = a;
            out[2 * j + 1] = b;
        }
        return;
    }
#pragma unroll
    for (int j = 0; j < NP; ++j) {
        out[2 * j] = coef<R>(c32, c64, S, sub, p0 + j, 0, 0) + coef<R>(c32, c64, S, sub, p0 + j, 1, 0) * x;
        out[2 * j + 1] = coef<R>(c32, c64, S, sub, p0 + j, 0, 1) + coef<R>(c32, c64, S, sub, p0 + j, 1, 1) * x;
    }
    R tm = R(1), t = x;
    const R x2 = x + x;
#pragma unroll
    for (int n = 2; n < NCHEB; ++n) {
        const R tn = x2 * t - tm;
        tm = t;
        t = tn;
#pragma unroll
        for (int j = 0; j < NP; ++j) {
            out[2 * j] += coef<R>(c32, c64, S, sub, p0 + j, n, 0) * tn;
            out[2 * j + 1] += coef<R>(c32, c64, S, sub, p0 + j, n, 1) * tn;
        }
    }
}

// Accumulator array of the classes [AB, AE): slot of class c is
// slot0(c) - slot0(AB) + (cell + OFF) + (P_c - 1 - j) for lag classes.
template <int OFF, int AB, int AE>
struct Grp {
    static constexpr int NS = slot0<OFF>(AE) - slot0<OFF>(AB);
    static constexpr int off(int c) { return slot0<OFF>(c) - slot0<OFF>(AB); }
};

// Add the P panel values of lag class C for cell offset K = cell + OFF:
// t_b += psi w lambda_b / r (b = 0, 1, 2) and s~ += psi~ w / r.
template <typename R, int OFF, int AB, int AE, int C, int K>
__device__ __forceinline__ void acc_class(R (&acc)[Grp<OFF, AB, AE>::NS][4], const R *v, R f0, R f1, R f2, R wr) {
    if constexpr (C >= AB && C < AE) {
        constexpr int P = cls_P(C);
#pragma unroll
        for (int j = 0; j < P; ++j) {
            const int s = Grp<OFF, AB, AE>::off(C) + K + P - 1 - j;
            const R ps = v[2 * j], pt = v[2 * j + 1];
            acc[s][0] += ps * f0;
            acc[s][1] += ps * f1;
            acc[s][2] += ps * f2;
            acc[s][3] += pt * wr;
        }
    }
}

template <typename R, int OFF, int AB, int AE, int K>
__device__ __forceinline__ void acc_case(R (&acc)[Grp<OFF, AB, AE>::NS][4], const R *v1, const R *v2,
                                         const R *v3, R f0, R f1, R f2, R wr) {
    acc_class<R, OFF, AB, AE, C1, K>(acc, v1, f0, f1, f2, wr);
    acc_class<R, OFF, AB, AE, C2, K>(acc, v2, f0, f1, f2, wr);
    acc_class<R, OFF, AB, AE, C3, K>(acc, v3, f0, f1, f2, wr);
}

template <typename R, int OFF, int AB, int AE>
__device__ __forceinline__ void acc_switch(R (&acc)[Grp<OFF, AB, AE>::NS][4], int k, const R *v1,
                                           const R *v2, const R *v3, R f0, R f1, R f2, R wr) {
    switch (k) {
        case 0: acc_case<R, OFF, AB, AE, 0>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 1: acc_case<R, OFF, AB, AE, 1>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 2: acc_case<R, OFF, AB, AE, 2>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 3: if constexpr (OFF >= 2) acc_case<R, OFF, AB, AE, 3>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 4: if constexpr (OFF >= 2) acc_case<R, OFF, AB, AE, 4>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 5: if constexpr (OFF >= 3) acc_case<R, OFF, AB, AE, 5>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        case 6: if constexpr (OFF >= 3) acc_case<R, OFF, AB, AE, 6>(acc, v1, v2, v3, f0, f1, f2, wr); break;
        default: break;
    }
}

template <typename R, int OFF, int AB, int AE, int C>
__device__ __forceinline__ void acc_special(R (&acc)[Grp<OFF, AB, AE>::NS][4], R ps, R pt, R fa, R fb, R fc, R wr) {
    if constexpr (C >= AB && C < AE) {
        constexpr int s = Grp<OFF, AB, AE>::off(C);
        acc[s][0] += ps * fa;
        acc[s][1] += ps * fb;
        acc[s][2] += ps * fc;
        acc[s][3] += pt * wr;
    }
}

// Per-thread view of the current (tau, x_w, sigma) triple.
struct Pt {
    int64_t sg;
    int valid, base;
    float f0, R0, D0, D1, D2;
    float dx0, dx1, dx2;
    double xw0, xw1, xw2;
};

// Quadrature over the 7 trial points for the classes [AB, AE).
template <typename R, int OFF, int AB, int AE>
__device__ __forceinline__ void quad_classes(const FarArgs &A, const ChebF32 &C32, int S, const Pt &p,
                                             R (&acc)[Grp<OFF, AB, AE>::NS][4]) {
    constexpr int NS = Grp<OFF, AB, AE>::NS;
    const Geo &g = A.g;
    const double *c64 = A.cheb64;
    const double inv_dt = A.lt.inv_dt;
    const R inv_dtR = (R)inv_dt;
    const int rhoSN0 = A.lt.rho[SN0];
    const int64_t sg = p.sg;
#pragma unroll
    for (int s = 0; s < NS; ++s) acc[s][0] = acc[s][1] = acc[s][2] = acc[s][3] = R(0);
#pragma unroll 1
    for (int y = 0; y < 7; ++y) {
        R q, rr;
        if constexpr (sizeof(R) == 4) {
            // r = |D + e|, e = (x - c_tau) - (y - c_sigma), D = c_tau - c_sigma:
            // r - R0 = (2 D.e + e.e) / (R0 + r) with D, R0 from the FP64 setup
            const float e0 = p.dx0 - g.dq32[(sg * 7 + y) * 3 + 0];
            const float e1 = p.dx1 - g.dq32[(sg * 7 + y) * 3 + 1];
            const float e2 = p.dx2 - g.dq32[(sg * 7 + y) * 3 + 2];
            const float sv = 2.f * (p.D0 * e0 + p.D1 * e1 + p.D2 * e2) + (e0 * e0 + e1 * e1 + e2 * e2);
            const float dr = sv / (p.R0 + sqrtf(fmaxf(p.R0 * p.R0 + sv, 0.f)));
            rr = p.R0 + dr;
            q = p.f0 + dr * inv_dtR;
        } else {
            const double y0 = g.cen[3 * sg] + g.dq[(sg * 7 + y) * 3 + 0];
            const double y1 = g.cen[3 * sg + 1] + g.dq[(sg * 7 + y) * 3 + 1];
            const double y2 = g.cen[3 * sg + 2] + g.dq[(sg * 7 + y) * 3 + 2];
            const double a0 = p.xw0 - y0, a1 = p.xw1 - y1, a2 = p.xw2 - y2;
            rr = sqrt(a0 * a0 + a1 * a1 + a2 * a2);
            q = rr * inv_dt - (double)p.base;
        }
        const R cf = floor(q);
        int cell = (int)cf;
        R u = q - cf;
        int sub = 0;
        if (S > 1) {
            const R us = u * (R)S;
            sub = min((int)floor(us), S - 1);
            u = us - (R)sub;
        }
        const R x = u + u - R(1);
        const R wr = p.valid ? rule_w<R>(A, y) / rr : R(0);
        const R fa = wr * rule_l<R>(A, 3 * y), fb = wr * rule_l<R>(A, 3 * y + 1), fc = wr * rule_l<R>(A, 3 * y + 2);
        if (cell < -OFF || cell > OFF) {
            if (p.valid) A.status[0] = ST_OFF_RANGE;
            cell = 0;
        }
        if constexpr (AB < NLAG) {
            R v1[6], v2[8], v3[6];
            if constexpr (C1 >= AB && C1 < AE) cheb_dots<R, 3>(C32, c64, S, sub, cls_panel0(C1), x, v1);
            if constexpr (C2 >= AB && C2 < AE) cheb_dots<R, 4>(C32, c64, S, sub, cls_panel0(C2), x, v2);
            if constexpr (C3 >= AB && C3 < AE) cheb_dots<R, 3>(C32, c64, S, sub, cls_panel0(C3), x, v3);
            acc_switch<R, OFF, AB, AE>(acc, cell + OFF, v1, v2, v3, fa, fb, fc, wr);
        }
        if constexpr (AE == NCLASS) {
            // special blocks: absolute cell 0 (four of them) or N-3, N-2 (SN0)
            const int absc = p.base + cell;
            if (__any_sync(0xffffffffu, p.valid && absc == 0)) {
                R vs[8];
                cheb_dots<R, 2>(C32, c64, S, sub, cls_panel0(S00), x, vs);      // S00, S01
                cheb_dots<R, 2>(C32, c64, S, sub, cls_panel0(SNN), x, vs + 4);  // SNN, SN1N
                if (absc == 0) {
                    acc_special<R, OFF, AB, AE, S00>(acc, vs[0], vs[1], fa, fb, fc, wr);
                    acc_special<R, OFF, AB, AE, S01>(acc, vs[2], vs[3], fa, fb, fc, wr);
                    acc_special<R, OFF, AB, AE, SNN>(acc, vs[4], vs[5], fa, fb, fc, wr);
                    acc_special<R, OFF, AB, AE, SN1N>(acc, vs[6], vs[7], fa, fb, fc, wr);
                }
            }
            if (__any_sync(0xffffffffu, p.valid && (absc == rhoSN0 || absc == rhoSN0 + 1))) {
                R vs[4];
                cheb_dots<R, 2>(C32, c64, S, sub, cls_panel0(SN0), x, vs);
                if (absc == rhoSN0 || absc == rhoSN0 + 1) {
                    const bool j1 = absc != rhoSN0;
                    acc_special<R, OFF, AB, AE, SN0>(acc, j1 ? vs[2] : vs[0], j1 ? vs[3] : vs[1], fa, fb, fc, wr);
                }
            }
        }
    }
}

// Write the classes [GB, GE) of the accumulator array to shared memory, sum
// over the 7 test points and store the local 3x3 matrices into Lb.
template <typename R, int OFF, int AB, int AE, int GB, int GE>
__device__ __forceinline__ void reduce_group(const FarArgs &A, int64_t tau, int64_t ch, const FarSetup<R> &su,
                                             R (&acc)[Grp<OFF, AB, AE>::NS][4], R *red, R *Lb) {
    constexpr int NG = slot0<OFF>(GE) - slot0<OFF>(GB);
    constexpr int NS = total_slots<OFF>();
    constexpr int G0 = Grp<OFF, AB, AE>::off(GB);
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Geo &g = A.g;
    R *rp = red + ((size_t)(w * 32 + lane) * NG) * 4;
#pragma unroll
    for (int s = 0; s < NG; ++s) {
        rp[4 * s + 0] = acc[G0 + s][0]; rp[4 * s + 1] = acc[G0 + s][1];
        rp[4 * s + 2] = acc[G0 + s][2]; rp[4 * s + 3] = acc[G0 + s][3];
    }
    __syncthreads();
    for (int it = threadIdx.x; it < 32 * NG; it += FAR_THREADS) {
        const int sl = it / NG, s = it % NG;
        const int64_t sg = ch * 32 + sl < g.E ? ch * 32 + sl : 0;
        R Sab[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, St = 0;
#pragma unroll
        for (int xw = 0; xw < 7; ++xw) {
            const R *q = red + ((size_t)(xw * 32 + sl) * NG + s) * 4;
            const R tb[3] = {q[0], q[1], q[2]};
            const R wx = rule_w<R>(A, xw);
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const R ga = wx * rule_l<R>(A, 3 * xw + a);
#pragma unroll
                for (int b = 0; b < 3; ++b) Sab[a][b] += ga * tb[b];
            }
            St += wx * q[3];
        }
        const R sc = su.scale[sl], nn = su.nn[sl];
        R *lp = Lb + ((size_t)sl * NS + slot0<OFF>(GB) + s) * 9;
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R cc;
                if constexpr (sizeof(R) == 4) {
                    const float *gt = g.geo32 + 16 * tau + 4, *gs = g.geo32 + 16 * sg + 4;
                    cc = gt[3 * a] * gs[3 * b] + gt[3 * a + 1] * gs[3 * b + 1] + gt[3 * a + 2] * gs[3 * b + 2];
                } else {
                    const double *gt = g.geo64 + 16 * tau + 4, *gs = g.geo64 + 16 * sg + 4;
                    cc = gt[3 * a] * gs[3 * b] + gt[3 * a + 1] * gs[3 * b + 1] + gt[3 * a + 2] * gs[3 * b + 2];
                }
                lp[3 * a + b] = sc * (nn * Sab[a][b] + cc * St);
            }
    }
    __syncthreads();
}

template <int OFF>
constexpr int max_group_slots() {
    constexpr int a = slot0<OFF>(C2) - slot0<OFF>(C1);
    constexpr int b = slot0<OFF>(C3) - slot0<OFF>(C2);
    constexpr int c = slot0<OFF>(NCLASS) - slot0<OFF>(C3);
    return a > b ? (a > c ? a : c) : (b > c ? b : c);
}

template <typename R, int OFF>
__global__ void __launch_bounds__(FAR_THREADS, 1)
far_kernel(const FarArgs A, const __grid_constant__ ChebF32 C32, int S) {
    constexpr int NS = total_slots<OFF>();
    constexpr int NGMAX = max_group_slots<OFF>();
    extern __shared__ __align__(16) unsigned char smem_raw[];
    FarSetup<R> &su = *reinterpret_cast<FarSetup<R> *>(smem_raw);
    R *red = reinterpret_cast<R *>(smem_raw + ((sizeof(FarSetup<R>) + 15) / 16) * 16);  // [7][32][NGMAX][4]
    R *Lb = red + (size_t)FAR_WARPS * 32 * NGMAX * 4;                                    // [32][NS][9]

    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, MM = M * M;
    const double inv_dt = A.lt.inv_dt;

    for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
        const int64_t tau = A.color_tris[ti];
        const int32_t Ft0 = g.F[3 * tau], Ft1 = g.F[3 * tau + 1], Ft2 = g.F[3 * tau + 2];
        Pt p;
        p.dx0 = g.dq32[(tau * 7 + w) * 3 + 0];
        p.dx1 = g.dq32[(tau * 7 + w) * 3 + 1];
        p.dx2 = g.dq32[(tau * 7 + w) * 3 + 2];
        p.xw0 = g.cen[3 * tau] + g.dq[(tau * 7 + w) * 3 + 0];
        p.xw1 = g.cen[3 * tau + 1] + g.dq[(tau * 7 + w) * 3 + 1];
        p.xw2 = g.cen[3 * tau + 2] + g.dq[(tau * 7 + w) * 3 + 2];

        for (int64_t ch = 0; ch < A.nchunks; ++ch) {
            // ---- element-pair setup (FP64 centroid distance), warp 0
            if (w == 0) {
                const int64_t sg = ch * 32 + lane;
                int valid = 0, base = 0;
                float f0 = 0.f, R0 = 1.f, D0 = 0.f, D1 = 0.f, D2 = 0.f;
                R scale = R(0), nn = R(0);
                if (sg < E) {
                    const int32_t *B = g.F + 3 * sg;
                    int shared = 0;
                    for (int b = 0; b < 3; ++b) shared += (B[b] == Ft0) + (B[b] == Ft1) + (B[b] == Ft2);
                    valid = shared == 0;
                    const double d0 = g.cen[3 * tau] - g.cen[3 * sg];
                    const double d1 = g.cen[3 * tau + 1] - g.cen[3 * sg + 1];
                    const double d2 = g.cen[3 * tau + 2] - g.cen[3 * sg + 2];
                    const double r0 = sqrt(d0 * d0 + d1 * d1 + d2 * d2);
                    const double q0 = r0 * inv_dt;
                    const double fb = floor(q0);
                    base = (int)fb;
                    f0 = (float)(q0 - fb);
                    R0 = (float)r0; D0 = (float)d0; D1 = (float)d1; D2 = (float)d2;
                    if constexpr (sizeof(R) == 8) {
                        const double *gt = g.geo64 + 16 * tau, *gs = g.geo64 + 16 * sg;
                        scale = gt[3] * gs[3] * 0.07957747154594767;  // 1/(4 pi)
                        nn = gt[0] * gs[0] + gt[1] * gs[1] + gt[2] * gs[2];
                    } else {
                        const float *gt = g.geo32 + 16 * tau, *gs = g.geo32 + 16 * sg;
                        scale = gt[3] * gs[3] * 0.07957747f;
                        nn = gt[0] * gs[0] + gt[1] * gs[1] + gt[2] * gs[2];
                    }
                }
                su.valid[lane] = valid; su.base[lane] = base; su.f0[lane] = f0; su.R0[lane] = R0;
                su.D[lane][0] = D0; su.D[lane][1] = D1; su.D[lane][2] = D2;
                su.scale[lane] = scale; su.nn[lane] = nn;
            }
            __syncthreads();
            p.sg = ch * 32 + lane < E ? ch * 32 + lane : 0;
            p.valid = su.valid[lane]; p.base = su.base[lane];
            p.f0 = su.f0[lane]; p.R0 = su.R0[lane];
            p.D0 = su.D[lane][0]; p.D1 = su.D[lane][1]; p.D2 = su.D[lane][2];

            if constexpr (sizeof(R) == 4) {
                // one sweep over the trial points feeds every class
                R acc[NS][4];
                quad_classes<R, OFF, 0, NCLASS>(A, C32, 1, p, acc);
                reduce_group<R, OFF, 0, NCLASS, C1, C2>(A, tau, ch, su, acc, red, Lb);
                reduce_group<R, OFF, 0, NCLASS, C2, C3>(A, tau, ch, su, acc, red, Lb);
                reduce_group<R, OFF, 0, NCLASS, C3, NCLASS>(A, tau, ch, su, acc, red, Lb);
            } else {
                // FP64: one sweep per class group keeps the accumulators in registers
                {
                    R acc[Grp<OFF, C1, C2>::NS][4];
                    quad_classes<R, OFF, C1, C2>(A, C32, S, p, acc);
                    reduce_group<R, OFF, C1, C2, C1, C2>(A, tau, ch, su, acc, red, Lb);
                }
                {
                    R acc[Grp<OFF, C2, C3>::NS][4];
                    quad_classes<R, OFF, C2, C3>(A, C32, S, p, acc);
                    reduce_group<R, OFF, C2, C3, C2, C3>(A, tau, ch, su, acc, red, Lb);
                }
                {
                    R acc[Grp<OFF, C3, NCLASS>::NS][4];
                    quad_classes<R, OFF, C3, NCLASS>(A, C32, S, p, acc);
                    reduce_group<R, OFF, C3, NCLASS, C3, NCLASS>(A, tau, ch, su, acc, red, Lb);
                }
            }

            scatter_chunk<R, OFF, FAR_THREADS>(A, ch, Ft0, Ft1, Ft2, su, Lb);
            __syncthreads();
        }
    }
}

template <typename R, int OFF>
static void launch_t(const FarArgs &a, const ChebF32 &c32, int S, int grid, cudaStream_t st) {
    constexpr int NS = total_slots<OFF>();
    constexpr int NG = max_group_slots<OFF>();
    const size_t smem = ((sizeof(FarSetup<R>) + 15) / 16) * 16 + sizeof(R) * ((size_t)FAR_WARPS * 32 * NG * 4 + 32 * NS * 9);
    cudaFuncSetAttribute(far_kernel<R, OFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    far_kernel<R, OFF><<<grid, FAR_THREADS, smem, st>>>(a, c32, S);
}

void launch_far(const FarArgs &a, const ChebF32 &c32, bool fp64, int off, int S, int grid,
                cudaStream_t st) {
    if (fp64) {
        if (off == 1) launch_t<double, 1>(a, c32, S, grid, st);
        else if (off == 2) launch_t<double, 2>(a, c32, S, grid, st);
        else launch_t<double, 3>(a, c32, S, grid, st);
    } else {
        if (off == 1) launch_t<float, 1>(a, c32, 1, grid, st);
        else if (off == 2) launch_t<float, 2>(a, c32, 1, grid, st);
        else launch_t<float, 3>(a, c32, 1, grid, st);
    }
}

}  // namespace tdbem
