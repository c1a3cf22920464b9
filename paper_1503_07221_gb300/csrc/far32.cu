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
__device__ __forceinline__ f2 add2(f2 a, f2 b) {
    f2 d;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 sub2(f2 a, f2 b) {
    f2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
__device__ __forceinline__ f2 mul2(f2 a, f2 b) {
    f2 d;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}
// (h, l) += (gh + gl) t on both halves: exact product error of gh t, two-sum
// into h, the rest into l
__device__ __forceinline__ void ff_acc(f2 &h, f2 &l, f2 gh, f2 gl, f2 t) {
    const f2 p = mul2(gh, t);
    const f2 pe = fma2(gh, t, sub2(0ull, p));
    const f2 s = add2(h, p);
    const f2 bb = sub2(s, h);
    const f2 e = add2(sub2(h, sub2(s, bb)), sub2(p, bb));
    l = fma2(gl, t, add2(l, add2(e, pe)));
    h = s;
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
    float sch[32], scl[32];          // |tau||sigma| / (4 pi) as an FP32 pair
    float nnh[32], nnl[32];          // n_tau . n_sigma as an FP32 pair
    int base[32];
    int valid[32];
    float f0h[32], f0l[32];  // frac(R0 / dt) as an FP32 pair
    float Dh[32][3];         // unit vector (c_tau - c_sigma) / R0 as an FP32 pair
    float Dl[32][3];
    float R0[32];
    float dqy[32][7][3];
    float cch[32][9], ccl[32][9];   // curl_a(tau) . curl_b(sigma) as FP32 pairs
};

// (psi, psi~) of the ten lag-class panels (C1: 3, C2: 4, C3: 3) at argument
// x, sharing one T_n recurrence. The terms n >= NLOW (at most a few 1e-3 of
// the panel maximum) are summed forward while the recurrence runs; then the
// FP32 residuals of the leading coefficients and the terms n < NLOW are added
// from n = NLOW-1 down to 0 from the kept T_n. Small terms therefore enter
// before the large leading ones, and the rounding of the leading coefficients
// does not become a fixed perturbation of psi, which the quadrature would not
// average away and the cancellation in the odd prototype would amplify. The
// last three additions (n = 2, 1, 0) carry a Kahan compensation term.
constexpr int NLOW = 8;
// Low-order part of one directly evaluated panel j (terms n < NLOW, the
// leading residuals, and the sum hj of the terms n >= NLOW).
__device__ __forceinline__ f2 panel_low(const ChebF32 &C, int j, const f2 (&T)[NLOW], f2 hj) {
    f2 a = 0ull;
#pragma unroll
    for (int n = 0; n < NCHEB_LO; ++n) a = fma2(lo2(C, j, n), T[n], a);
    a = fma2(pk(1.f, 1.f), hj, a);
#pragma unroll
    for (int n = NLOW - 1; n >= 3; --n) a = fma2(coef2(C, j, n), T[n], a);
    // the three largest terms with Kahan compensation: their partial sums
    // are of the size of psi, and their FP32 roundings would otherwise
    // dominate the error of the panel value
    f2 y = mul2(coef2(C, j, 2), T[2]);
    f2 t = add2(a, y);
    f2 nc = sub2(y, sub2(t, a));  // minus the rounding error of t
    a = t;
    y = fma2(coef2(C, j, 1), T[1], nc);
    t = add2(a, y);
    nc = sub2(y, sub2(t, a));
    return add2(t, add2(coef2(C, j, 0), nc));
}

__device__ __forceinline__ void lag_panels(const ChebF32 &C, float x, f2 (&v)[10]) {
    // Evaluated directly: C1 (panels 0-2) and C3 (7-9), and the first two C2
    // panels (3, 4) with their even and odd terms kept apart. The inner
    // prototype is antisymmetric about the centre of its support (Eq.
    // symmetryXi, p = 0), so C2 panel 3 - s at x is minus panel s at -x:
    // O_s(x) - E_s(x). Two of the ten Chebyshev sums are thereby saved.
    constexpr int DIR[6] = {0, 1, 2, 7, 8, 9};
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
    f2 hi[6], hE[2], hO[2];
#pragma unroll
    for (int d = 0; d < 6; ++d) hi[d] = 0ull;
#pragma unroll
    for (int q = 0; q < 2; ++q) { hE[q] = 0ull; hO[q] = 0ull; }
#pragma unroll
    for (int n = NLOW; n < NCHEB; ++n) {
        const float tn = x2 * t1 - t0;
        t0 = t1;
        t1 = tn;
        const f2 tt = pk(tn, tn);
#pragma unroll
        for (int d = 0; d < 6; ++d) hi[d] = fma2(coef2(C, DIR[d], n), tt, hi[d]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (n & 1) hO[q] = fma2(coef2(C, 3 + q, n), tt, hO[q]);
            else hE[q] = fma2(coef2(C, 3 + q, n), tt, hE[q]);
        }
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) v[DIR[d]] = panel_low(C, DIR[d], T, hi[d]);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = 3 + q;
        f2 aE = fma2(lo2(C, j, 2), T[2], mul2(lo2(C, j, 0), T[0]));
        f2 aO = fma2(lo2(C, j, 3), T[3], mul2(lo2(C, j, 1), T[1]));
        aE = add2(aE, hE[q]);
        aO = add2(aO, hO[q]);
        aO = fma2(coef2(C, j, 7), T[7], aO);
        aE = fma2(coef2(C, j, 6), T[6], aE);
        aO = fma2(coef2(C, j, 5), T[5], aO);
        aE = fma2(coef2(C, j, 4), T[4], aE);
        aO = fma2(coef2(C, j, 3), T[3], aO);
        // Kahan compensation of the largest terms, as in panel_low
        f2 y = mul2(coef2(C, j, 2), T[2]);
        f2 t = add2(aE, y);
        f2 nc = sub2(y, sub2(t, aE));
        aE = add2(t, add2(coef2(C, j, 0), nc));
        y = mul2(coef2(C, j, 1), T[1]);
        t = add2(aO, y);
        nc = sub2(y, sub2(t, aO));
        aO = add2(t, nc);
        v[j] = add2(aE, aO);
        v[6 - q] = sub2(aO, aE);
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
    const float f0h = su.f0h[lane], f0l = su.f0l[lane], R0 = su.R0[lane];
    const float Dh0 = su.Dh[lane][0], Dh1 = su.Dh[lane][1], Dh2 = su.Dh[lane][2];
    const float Dl0 = su.Dl[lane][0], Dl1 = su.Dl[lane][1], Dl2 = su.Dl[lane][2];
    const float ih = (float)A.lt.inv_dt, il = (float)(A.lt.inv_dt - (double)ih);
#pragma unroll 1
    for (int y = 0; y < 7; ++y) {
        // r - R0 = u + e_perp^2 / ((R0 + u) + r) with u = D^.e, e the offset
        // difference and e_perp^2 = e.e - u^2; the FP32 rounding of the
        // small correction term is harmless, and u carries the low part of
        // the unit vector D^
        const float e0 = dx0 - su.dqy[lane][y][0];
        const float e1 = dx1 - su.dqy[lane][y][1];
        const float e2 = dx2 - su.dqy[lane][y][2];
        const float u = fmaf(Dh2, e2, fmaf(Dh1, e1, Dh0 * e0));
        const float ul = fmaf(Dl2, e2, fmaf(Dl1, e1, Dl0 * e0));
        const float ee = fmaf(e2, e2, fmaf(e1, e1, e0 * e0));
        const float ep = fmaf(-u, u, ee);
        const float tt = R0 + u;
        const float rr = sqrtf(fmaxf(fmaf(tt, tt, ep), 0.f));
        const float corr = ep * __frcp_rn(tt + rr);
        const float ir = __frcp_rn(tt + corr);
        // q = f0 + (u + corr + ul) / dt as an FP32 pair (two-sums and exact
        // product error); floor of the high part, fraction plus low part
        const float du = u + corr;
        const float b1 = du - u;
        const float de = (u - (du - b1)) + (corr - b1);
        const float wh = du * ih;
        const float wl = fmaf(du, ih, -wh);
        const float sh = f0h + wh;
        const float b2 = sh - f0h;
        const float se = (f0h - (sh - b2)) + (wh - b2);
        const float low = (se + (wl + fmaf(de + ul, ih, du * il))) + f0l;
        const float cf = floorf(sh);
        int cell = (int)cf;
        const float uq = (sh - cf) + low;
        const float x = uq + uq - 1.f;
        // weights w_y lambda_b(y) and w_y carried as FP32 pairs, so that
        // their rounding is not a fixed bias shared by all element pairs
        const float irv = valid ? ir : 0.f;
        const float F0 = fmaf(irv, A.gwl[3 * y], irv * A.gwh[3 * y]);
        const float F1 = fmaf(irv, A.gwl[3 * y + 1], irv * A.gwh[3 * y + 1]);
        const float F2 = fmaf(irv, A.gwl[3 * y + 2], irv * A.gwh[3 * y + 2]);
        const float wr = fmaf(irv, A.wwl[y], irv * A.wwh[y]);
        const f2 F01 = pk(F0, F1);
        const f2 F2W = pk(F2, wr);
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
    float f0h = 0.f, f0l = 0.f, R0 = 1.f;
    float Dh[3] = {0.f, 0.f, 0.f}, Dl[3] = {0.f, 0.f, 0.f};
    double scale = 0.0, nn = 0.0, cc[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
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
        const double f0 = q0 - fb;
        f0h = (float)f0;
        f0l = (float)(f0 - (double)f0h);
        R0 = (float)r0;
        const double ir0 = 1.0 / r0;
        const double dd[3] = {d0 * ir0, d1 * ir0, d2 * ir0};
        for (int k = 0; k < 3; ++k) {
            Dh[k] = (float)dd[k];
            Dl[k] = (float)(dd[k] - (double)Dh[k]);
        }
        // geometric factors of the element pair in FP64, kept as FP32 pairs:
        // the n.n and curl.curl parts of a block cancel to a small fraction
        // of either, so their FP32 rounding would be amplified
        const double *gt = g.geo64 + 16 * tau, *gs = g.geo64 + 16 * sg;
        scale = gt[3] * gs[3] * 0.079577471545947668;  // 1/(4 pi)
        nn = gt[0] * gs[0] + gt[1] * gs[1] + gt[2] * gs[2];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                cc[3 * a + b] = gt[4 + 3 * a] * gs[4 + 3 * b] + gt[5 + 3 * a] * gs[5 + 3 * b] + gt[6 + 3 * a] * gs[6 + 3 * b];
        for (int k = 0; k < 21; ++k) su.dqy[lane][k / 3][k % 3] = g.dq32[sg * 21 + k];
    } else {
        for (int k = 0; k < 21; ++k) su.dqy[lane][k / 3][k % 3] = 0.f;
    }
    su.sch[lane] = (float)scale;
    su.scl[lane] = (float)(scale - (double)su.sch[lane]);
    su.nnh[lane] = (float)nn;
    su.nnl[lane] = (float)(nn - (double)su.nnh[lane]);
    for (int k = 0; k < 9; ++k) {
        su.cch[lane][k] = (float)cc[k];
        su.ccl[lane][k] = (float)(cc[k] - (double)su.cch[lane][k]);
    }
    su.valid[lane] = valid; su.base[lane] = base; su.f0h[lane] = f0h; su.f0l[lane] = f0l; su.R0[lane] = R0;
    for (int k = 0; k < 3; ++k) { su.Dh[lane][k] = Dh[k]; su.Dl[lane][k] = Dl[k]; }
    if (lane == 0) { su.tau = tau; su.ch = ch; su.Ft[0] = Ft0; su.Ft[1] = Ft1; su.Ft[2] = Ft2; }
}

// a + b for FP32 pairs: two-sum of the high parts, renormalised
__device__ __forceinline__ FF ff_plus(FF a, FF b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb);
    const float l = (a.l + b.l) + e;
    const float h = s + l;
    return FF{h, l - (h - s)};
}

// Staging of the current chunk's scatter inputs, issued by the producer warp
// while the compute warps run the quadrature: the lag-window bounds of every
// (trial vertex, test corner, class) item and the window values themselves
// (asynchronous 8-byte copies into shared memory), so that the scatter phase
// reads only shared memory and writes global memory.
__device__ __forceinline__ void stage_scatter(const FarArgs &A, const Setup32 &su, int lane, double *stg,
                                              int16_t *swlo, int16_t *swhi) {
    const Geo &g = A.g;
    const int64_t M = g.M, MM = M * M;
    const int KW = A.KW;
    const int v0 = A.chunk_vptr[su.ch], nitems = (A.chunk_vptr[su.ch + 1] - v0) * 3 * NLAG;
    constexpr int SPL = 8;  // items per lane per batch: independent loads in flight
    for (int b0 = 0; b0 < nitems; b0 += 32 * SPL) {
        int64_t o[SPL];
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            const int it = b0 + q * 32 + lane;
            o[q] = -1;
            if (it < nitems) {
                const int v = it / (3 * NLAG), rem = it % (3 * NLAG);
                const int a = rem / NLAG, c = rem % NLAG;
                o[q] = c * MM + (int64_t)su.Ft[a] * M + A.chunk_vert[v0 + v];
            }
        }
        int16_t wl[SPL], wh[SPL];
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            wl[q] = o[q] >= 0 ? A.dlo[o[q]] : (int16_t)0;
            wh[q] = o[q] >= 0 ? A.dhi[o[q]] : (int16_t)0;
        }
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            if (o[q] < 0) continue;
            const int it = b0 + q * 32 + lane;
            const double *src = A.dense + o[q] * KW;
            const unsigned dst = (unsigned)__cvta_generic_to_shared(stg + (size_t)it * KW);
            for (int k = 0; k < KW; ++k)
                asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst + 8 * k), "l"(src + k));
        }
#pragma unroll
        for (int q = 0; q < SPL; ++q) {
            if (o[q] < 0) continue;
            const int it = b0 + q * 32 + lane;
            swlo[it] = wl[q];
            swhi[it] = wh[q];
        }
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
}

// Scatter of one chunk's lag-class values into the FP64 lag windows of the
// CTA's test rows from the staged windows: thread per (trial vertex, test
// corner, class), sums over the chunk's triangles at that vertex.
template <int OFF>
__device__ __forceinline__ void scatter_staged(const FarArgs &A, const Setup32 &su, const FF *Lb,
                                               const double *stg, const int16_t *swlo, const int16_t *swhi) {
    constexpr int NS = slot0<OFF>(NLAG);
    const Geo &g = A.g;
    const int64_t M = g.M, MM = M * M;
    const int KW = A.KW;
    const int v0 = A.chunk_vptr[su.ch], nitems = (A.chunk_vptr[su.ch + 1] - v0) * 3 * NLAG;
    for (int it = threadIdx.x; it < nitems; it += F32_THREADS_ALL) {
        const int v = it / (3 * NLAG), rem = it % (3 * NLAG);
        const int a = rem / NLAG, c = rem % NLAG;
        const int s0 = A.chunk_sptr[v0 + v], s1 = A.chunk_sptr[v0 + v + 1];
        const int P = cls_P(c), K = 2 * OFF + P;
        const int rho = A.lt.rho[c];
        const int so = c == C1 ? slot0<OFF>(C1) : c == C2 ? slot0<OFF>(C2) : slot0<OFF>(C3);
        const int wlo = swlo[it], whi = swhi[it];
        // the mixed path keeps its far lag windows as FP32 pairs (hi, lo):
        // updated with two-sums on the FP32 pipe, exact enough for the FP64
        // sums they stand for, and no FP64 add on this critical phase
        FF *dst = reinterpret_cast<FF *>(A.dense) + (c * MM + (int64_t)su.Ft[a] * M + A.chunk_vert[v0 + v]) * KW;
        const FF *cur = reinterpret_cast<const FF *>(stg) + (size_t)it * KW;
        // the vertex's triangles in this chunk, 3 per batch, in registers (a batch of
        // 3 keeps the predicated sums short; most vertices need one or two)
        constexpr int MAXS = 3;
        for (int x0 = s0; x0 < s1; x0 += MAXS) {
            int lbi[MAXS], off[MAXS];
            bool has[MAXS];
            int dmn = 1 << 30, dmx = -(1 << 30);
#pragma unroll
            for (int q = 0; q < MAXS; ++q) {
                has[q] = false;
                lbi[q] = 0;
                off[q] = 0;
                if (x0 + q < s1) {
                    const int src = A.chunk_src[x0 + q], sl = src / 3, b = src % 3;
                    if (su.valid[sl]) {
                        has[q] = true;
                        off[q] = su.base[sl] - rho - (P - 1) - OFF;
                        lbi[q] = (sl * NS + so) * 9 + 3 * a + b;
                        dmn = min(dmn, off[q]);
                        dmx = max(dmx, off[q] + K - 1);
                    }
                }
            }
            dmn = max(dmn, wlo);
            dmx = min(min(dmx, whi), wlo + KW - 1);
            for (int d = dmn; d <= dmx; ++d) {
                FF sum{};
#pragma unroll
                for (int q = 0; q < MAXS; ++q) {
                    const int slot = d - off[q];
                    if (has[q] && slot >= 0 && slot < K) lb_add(sum, Lb[lbi[q] + slot * 9]);
                }
                // first batch adds to the staged value, later ones to what the
                // previous batch stored
                const FF base_v = x0 == s0 ? cur[d - wlo] : dst[d - wlo];
                dst[d - wlo] = ff_plus(base_v, sum);
            }
        }
    }
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
    FF *Lb = reinterpret_cast<FF *>(red + (size_t)F32_XW * 32 * NS * 4);                        // [32][NS][9]
    double *stg = reinterpret_cast<double *>(Lb + (size_t)32 * NS * 9);                        // [max_nv * 9][KW]
    int16_t *swlo = reinterpret_cast<int16_t *>(stg + (size_t)A.max_nv * 3 * NLAG * A.KW);     // [max_nv * 9]
    int16_t *swhi = swlo + A.max_nv * 3 * NLAG;
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
            stage_scatter(A, su, lane, stg, swlo, swhi);
            if (it + 1 < nit) {
                const int64_t t2 = A.color_tris[blockIdx.x + ((it + 1) / nch) * gridDim.x];
                chunk_setup(A, t2, (it + 1) % nch, lane, sub[(it + 1) & 1]);
            }
            asm volatile("cp.async.wait_all;" ::: "memory");
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
            FF *lp = Lb + ((size_t)sl * NS + s) * 9;
            f2 q01[7], q2s[7];
            unsigned long long any = 0ull;
#pragma unroll
            for (int x = 0; x < 7; ++x) {
                const f2 *q = reinterpret_cast<const f2 *>(red + ((size_t)(x * 32 + sl) * NS + s) * 4);
                q01[x] = q[0];
                q2s[x] = q[1];
                any |= q01[x] | q2s[x];
            }
            if (any == 0ull) {  // slot not reached by this element pair
#pragma unroll
                for (int i = 0; i < 9; ++i) lp[i] = FF{0.f, 0.f};
                continue;
            }
            // S_ab = sum_x w_x lambda_a(x) t_b(x) and S~ = sum_x w_x s~(x)
            // as FP32 pairs: packed (S_a0, S_a1) for a = 0..2, (S_02, S_12)
            // and (S_22, S~)
            f2 h[5] = {0ull, 0ull, 0ull, 0ull, 0ull}, l[5] = {0ull, 0ull, 0ull, 0ull, 0ull};
#pragma unroll
            for (int x = 0; x < 7; ++x) {
                const float g0h = A.gwh[3 * x], g1h = A.gwh[3 * x + 1], g2h = A.gwh[3 * x + 2];
                const float g0l = A.gwl[3 * x], g1l = A.gwl[3 * x + 1], g2l = A.gwl[3 * x + 2];
                float t2, st;
                upk(q2s[x], t2, st);
                ff_acc(h[0], l[0], pk(g0h, g0h), pk(g0l, g0l), q01[x]);
                ff_acc(h[1], l[1], pk(g1h, g1h), pk(g1l, g1l), q01[x]);
                ff_acc(h[2], l[2], pk(g2h, g2h), pk(g2l, g2l), q01[x]);
                ff_acc(h[3], l[3], pk(g0h, g1h), pk(g0l, g1l), pk(t2, t2));
                ff_acc(h[4], l[4], pk(g2h, A.wwh[x]), pk(g2l, A.wwl[x]), q2s[x]);
            }
            float Sh[9], Sl[9], Th, Tl;
            upk(h[0], Sh[0], Sh[1]); upk(l[0], Sl[0], Sl[1]);
            upk(h[1], Sh[3], Sh[4]); upk(l[1], Sl[3], Sl[4]);
            upk(h[2], Sh[6], Sh[7]); upk(l[2], Sl[6], Sl[7]);
            upk(h[3], Sh[2], Sh[5]); upk(l[3], Sl[2], Sl[5]);
            upk(h[4], Sh[8], Th); upk(l[4], Sl[8], Tl);
            // L_ab = scale (n.n S_ab + curl_a.curl_b S~) in FP32-pair arithmetic
            const float sch = su.sch[sl], scl = su.scl[sl], nh = su.nnh[sl], nl = su.nnl[sl];
#pragma unroll
            for (int i = 0; i < 9; ++i) {
                const float ch = su.cch[sl][i], cl = su.ccl[sl][i];
                const float ph = nh * Sh[i];
                const float pl = fmaf(nh, Sh[i], -ph) + fmaf(nh, Sl[i], nl * Sh[i]);
                const float qh = ch * Th;
                const float ql = fmaf(ch, Th, -qh) + fmaf(ch, Tl, cl * Th);
                const float th = ph + qh;
                const float bb = th - ph;
                const float tl = ((ph - (th - bb)) + (qh - bb)) + (pl + ql);
                const float lh = sch * th;
                const float ll = fmaf(sch, th, -lh) + fmaf(sch, tl, scl * th);
                lp[i] = FF{lh, ll};
            }
        }
        __syncthreads();
        scatter_staged<OFF>(A, su, Lb, stg, swlo, swhi);
        __syncthreads();
    }
}

template <int OFF>
static void launch32(const FarArgs &a, const ChebF32 &c32, int grid, cudaStream_t st) {
    constexpr int NS = slot0<OFF>(NLAG);
    const size_t smem = ((2 * sizeof(Setup32) + 15) / 16) * 16 + sizeof(float) * (size_t)F32_XW * 32 * NS * 4 +
                        sizeof(FF) * 32 * NS * 9 + (sizeof(double) * a.KW + 2 * sizeof(int16_t)) * (size_t)a.max_nv * 3 * NLAG;
    cudaFuncSetAttribute(far32_kernel<OFF>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    far32_kernel<OFF><<<grid, F32_THREADS_ALL, smem, st>>>(a, c32);
}

void launch_far32(const FarArgs &a, const ChebF32 &c32, int off, int grid, cudaStream_t st) {
    if (off == 1) launch32<1>(a, c32, grid, st);
    else if (off == 2) launch32<2>(a, c32, grid, st);
    else launch32<3>(a, c32, grid, st);
}

}  // namespace tdbem
