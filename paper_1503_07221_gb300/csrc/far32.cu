// Far-field quadrature in mixed precision (FP32 arithmetic, FP32-pair
// element-pair anchor) for element pairs without a shared vertex: 7-point
// rule on both triangles (Eq. MatrixEntries), psi and psi~ from the degree-32
// Chebyshev panels of the lag classes (Sec. 3.1).
//
// CTA = 8 warps, two CTAs per SM. Warps 0..6 are the 7 test points x_w of the
// test triangle tau, lanes the 32 trial triangles sigma of a chunk; warp 7 is
// the producer. Per chunk:
//   P1  thread (x_w, sigma) runs the 7 trial points y: distance, one T_n
//       recurrence, 8 Chebyshev sums of (psi, psi~) pairs (fma.rn.f32x2 with
//       the coefficient pair straight from the constant bank), and the
//       accumulation into its own window of W unit cells of the retarded
//       argument q = r / dt. Meanwhile the producer copies the chunk's
//       vertex-pair lag windows into shared memory (cp.async) and prepares
//       the element-pair setup of the next chunk;
//   P2  per (sigma, lag slot): the sums over the 7 test points with the
//       weights w_x lambda_a(x) and the combination
//         L_ab = |tau||sigma|/(4 pi) [ n.n S_ab + curl_a.curl_b S~ ];
//   P3  the 3x3 values of the chunk's triangles that share a trial vertex
//       are summed, added to the staged window and stored to the FP32-pair
//       vertex-pair lag windows of the test rows (one launch per colour of a
//       vertex-disjoint triangle colouring: no two CTAs share a row; no
//       atomics).
// While one CTA of an SM is in P2 / P3 or at a barrier, the other one keeps
// the FMA pipe busy with P1.
//
// Every lag class sees the same local argument: on an equidistant grid all
// class prototypes have their breakpoints at integer q, so u = frac(q) serves
// every panel of every class and only the lag a panel feeds depends on
// floor(q) (Sec. 3.1, Eq. psiTildeRed). A thread keeps, per lag slot,
//   (t_0, t_1) and (t_2, s~),   t_b = sum_y w_y lambda_b(y) psi / r,
//                               s~  = sum_y w_y psi~ / r.
//
// Precision: the distance is anchored at the centroid distance R0 of the
// element pair (FP32-pair arithmetic), r - R0 = u + e_perp^2 / ((R0 + u) + r)
// from FP32 offsets, and q = frac(R0/dt) + (r - R0)/dt is formed with
// two-sums; the leading Chebyshev coefficients carry their FP32 residuals
// (their rounding would be a fixed perturbation shared by every point pair);
// the test-point weights and the geometric factors are FP32 pairs, because
// the n.n and curl.curl parts of a block cancel to a small fraction of
// either part and a fixed rounding of a weight would not average out.
#include <math.h>

#include <algorithm>

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
__device__ __forceinline__ f2 coef2(const ChebLag32 &C, int p, int n) {
    return *reinterpret_cast<const f2 *>(&C.c[n][p][0]);
}
__device__ __forceinline__ f2 lo2(const ChebLag32 &C, int p, int n) {
    return *reinterpret_cast<const f2 *>(&C.lo[n][p][0]);
}

// mbarrier helpers: completion of the scatter (P3) of a chunk, awaited
// before its shared memory is reused. The wait gives up after a bounded
// number of polls and flags the status word instead of hanging.
__device__ __forceinline__ void mbar_init(unsigned addr, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(addr), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned addr) {
    unsigned long long st;
    asm volatile("mbarrier.arrive.shared::cta.b64 %0, [%1];" : "=l"(st) : "r"(addr) : "memory");
    (void)st;
}
__device__ __forceinline__ void mbar_wait(unsigned addr, unsigned parity, int *status) {
    for (int i = 0; i < (1 << 22); ++i) {
        unsigned done;
        asm volatile(
            "{ .reg .pred p; mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2; selp.u32 %0, 1, 0, p; }"
            : "=r"(done)
            : "r"(addr), "r"(parity)
            : "memory");
        if (done) return;
    }
    *status = ST_WAIT;
}

// ---- FP32-pair (double-float) arithmetic of the element-pair setup --------
// values h + l with |l| <= ulp(h) / 2; error-free transformations with FMA
struct DF {
    float h, l;
};
__device__ __forceinline__ DF df_fast(float a, float b) {  // |a| >= |b|
    const float s = a + b;
    return DF{s, b - (s - a)};
}
__device__ __forceinline__ DF df_add(DF a, DF b) {
    const float s = a.h + b.h;
    const float bb = s - a.h;
    const float e = (a.h - (s - bb)) + (b.h - bb);
    return df_fast(s, e + (a.l + b.l));
}
__device__ __forceinline__ DF df_mul(DF a, DF b) {
    const float p = a.h * b.h;
    const float e = fmaf(a.h, b.h, -p);
    return df_fast(p, fmaf(a.h, b.l, fmaf(a.l, b.h, e)));
}
__device__ __forceinline__ DF df_dot3(const DF *a, const DF *b) {
    return df_add(df_add(df_mul(a[0], b[0]), df_mul(a[1], b[1])), df_mul(a[2], b[2]));
}
// a / b with ib an approximation of 1 / b.h: quotient of the high parts, one
// correction from the exact remainder (the correction absorbs the error of q)
__device__ __forceinline__ DF df_div(DF a, DF b, float ib) {
    const float q = a.h * ib;
    const DF r = df_add(a, df_mul(DF{-q, 0.f}, b));
    return df_add(DF{q, 0.f}, DF{r.h * ib, 0.f});
}
__device__ __forceinline__ DF df_sqrt(DF a) {
    const float s = a.h * rsqrtf(a.h);
    const float p = s * s;
    const float e = fmaf(s, s, -p);
    return df_add(DF{s, 0.f}, DF{((a.h - p) - e + a.l) * (0.5f * rsqrtf(a.h)), 0.f});
}

// Per-thread window of W unit cells of q: the 7 trial points of sigma lie
// within rho_sigma of its centroid, so for a fixed test point their q span
// at most 2 rho / dt < W - 1 cells. Slots of class c: P_c + W - 1 per thread;
// over the 7 test points the thread windows start within W - 1 cells of
// each other, so the union has P_c + 2 W - 2 slots.
template <int W>
struct Win {
    static constexpr int NT = TOTAL_LAG_PANELS + 3 * (W - 1);
    static constexpr int NU = TOTAL_LAG_PANELS + 3 * (2 * W - 2);
    __host__ __device__ static constexpr int pt(int c) { return cls_P(c) + W - 1; }
    __host__ __device__ static constexpr int pu(int c) { return cls_P(c) + 2 * W - 2; }
    __host__ __device__ static constexpr int ot(int c) { return c == C1 ? 0 : c == C2 ? pt(C1) : pt(C1) + pt(C2); }
    __host__ __device__ static constexpr int ou(int c) { return c == C1 ? 0 : c == C2 ? pu(C1) : pu(C1) + pu(C2); }
};

struct Setup32 {
    int64_t tau, ch;
    int32_t Ft[3];
    int base[32];            // floor(R0 / dt)
    int valid[32];
    float f0h[32], f0l[32];  // frac(R0 / dt) as an FP32 pair
    float Dh[32][3];         // unit vector (c_tau - c_sigma) / R0 as an FP32 pair
    float Dl[32][3];
    float R0[32];
    float rs[32];            // max |y - c_sigma| / dt over the 7 points, rounded up
    float dqy[32][7][3];
    float nnh[32], nnl[32];        // |tau||sigma|/(4 pi) n_tau.n_sigma as an FP32 pair
    float cch[32][9], ccl[32][9];  // |tau||sigma|/(4 pi) curl_a(tau).curl_b(sigma)
};

// (psi, psi~) of the ten lag-class panels (C1: 0-2, C2: 3-6, C3: 7-9) at x in
// [-1, 1], sharing one recurrence. V_n = s_n T_n(x) with the sign pattern
// s = +, +, -, -, ... obeys V_{n+1} = (-1)^n 2x V_n + V_{n-1}: one packed FMA
// per term yields the operand pair (V_n, V_n) directly. Terms n >= 4 are
// summed as the recurrence runs (they are below 1e-2 of the panel maximum);
// then the FP32 residuals of c_0..c_3 and the terms 3, 2, 1, 0, so that small
// terms enter before the large leading ones. C2 panels 3 and 4 keep even and
// odd terms apart: the inner prototype is antisymmetric about the centre of
// its support (Eq. symmetryXi, p = 0), so C2 panel 3 - s at x is minus panel
// s at -x, O_s(x) - E_s(x), and two of the ten sums are saved.
__device__ __forceinline__ void lag_panels(const ChebLag32 &C, float x, f2 (&v)[TOTAL_LAG_PANELS]) {
    constexpr int DIR[6] = {0, 1, 2, 7, 8, 9};
    const float x2 = x + x;
    const f2 Xp = pk(x2, x2), Xm = pk(-x2, -x2);
    const f2 V1 = pk(x, x);
    const f2 V2 = fma2(Xm, V1, pk(1.f, 1.f));
    const f2 V3 = fma2(Xp, V2, V1);
    f2 hi[6], hE[2], hO[2];
    f2 a = V2, b = V3;
    {
        const f2 V4 = fma2(Xm, b, a);
#pragma unroll
        for (int d = 0; d < 6; ++d) hi[d] = mul2(coef2(C, DIR[d], 4), V4);
#pragma unroll
        for (int q = 0; q < 2; ++q) { hE[q] = mul2(coef2(C, 3 + q, 4), V4); hO[q] = 0ull; }
        a = b;
        b = V4;
    }
#pragma unroll
    for (int n = 5; n < NCHEB; ++n) {
        const f2 Vn = fma2((n & 1) ? Xp : Xm, b, a);  // V_n from V_{n-1} = b, V_{n-2} = a
        a = b;
        b = Vn;
#pragma unroll
        for (int d = 0; d < 6; ++d) hi[d] = fma2(coef2(C, DIR[d], n), Vn, hi[d]);
#pragma unroll
        for (int q = 0; q < 2; ++q) {
            if (n & 1) hO[q] = fma2(coef2(C, 3 + q, n), Vn, hO[q]);
            else hE[q] = fma2(coef2(C, 3 + q, n), Vn, hE[q]);
        }
    }
#pragma unroll
    for (int d = 0; d < 6; ++d) {
        const int j = DIR[d];
        f2 s = add2(lo2(C, j, 0), hi[d]);
        s = fma2(lo2(C, j, 1), V1, s);
        s = fma2(lo2(C, j, 2), V2, s);
        s = fma2(lo2(C, j, 3), V3, s);
        s = fma2(coef2(C, j, 3), V3, s);
        s = fma2(coef2(C, j, 2), V2, s);
        s = fma2(coef2(C, j, 1), V1, s);
        v[j] = add2(coef2(C, j, 0), s);
    }
#pragma unroll
    for (int q = 0; q < 2; ++q) {
        const int j = 3 + q;
        f2 e = add2(lo2(C, j, 0), hE[q]);
        f2 o = fma2(lo2(C, j, 1), V1, hO[q]);
        e = fma2(lo2(C, j, 2), V2, e);
        o = fma2(lo2(C, j, 3), V3, o);
        o = fma2(coef2(C, j, 3), V3, o);
        e = fma2(coef2(C, j, 2), V2, e);
        o = fma2(coef2(C, j, 1), V1, o);
        e = add2(coef2(C, j, 0), e);
        v[j] = add2(e, o);
        v[6 - q] = sub2(o, e);
    }
}

// Accumulation of one point pair into the thread's slots: panel j of class c
// at window cell k feeds slot k + P_c - 1 - j. The value of every slot is
// selected by the cell (no divergent branch), then two packed FMAs add
// (psi F_0, psi F_1) and (psi F_2, psi~ w / r).
template <int W, int CL>
__device__ __forceinline__ void acc_class(f2 *a01, f2 *a2s, const f2 (&v)[TOTAL_LAG_PANELS], int cell, f2 F01,
                                          f2 F2W) {
    constexpr int P = cls_P(CL), p0 = cls_panel0(CL), o = Win<W>::ot(CL);
#pragma unroll
    for (int s = 0; s < P + W - 1; ++s) {
        f2 val = 0ull;
#pragma unroll
        for (int k = 0; k < W; ++k) {
            const int j = k + P - 1 - s;
            if (j >= 0 && j < P) val = cell == k ? v[p0 + j] : val;
        }
        float ps, pt;
        upk(val, ps, pt);
        a01[o + s] = fma2(pk(ps, ps), F01, a01[o + s]);
        a2s[o + s] = fma2(val, F2W, a2s[o + s]);
    }
}

// P1 of one thread: test point x_w (offset dx from the centroid of tau),
// trial triangle = lane. Writes red[(xw NT + s) 32 + lane] = (t_0, t_1, t_2,
// s~) and the window start rbase[xw 32 + lane] (cells above floor(R0 / dt)).
template <int W>
__device__ __forceinline__ void quad_thread(const FarArgs &A, const ChebLag32 &C, const Setup32 &su, int xw,
                                            int lane, float dx0, float dx1, float dx2, float4 *red, int *rbase,
                                            unsigned mbar, int64_t it) {
    constexpr int NT = Win<W>::NT;
    f2 a01[NT], a2s[NT];
#pragma unroll
    for (int s = 0; s < NT; ++s) { a01[s] = 0ull; a2s[s] = 0ull; }
    const int valid = su.valid[lane];
    const float f0h = su.f0h[lane], f0l = su.f0l[lane], R0 = su.R0[lane];
    const float Dh0 = su.Dh[lane][0], Dh1 = su.Dh[lane][1], Dh2 = su.Dh[lane][2];
    const float Dl0 = su.Dl[lane][0], Dl1 = su.Dl[lane][1], Dl2 = su.Dl[lane][2];
    const float ih = (float)A.lt.inv_dt, il = (float)(A.lt.inv_dt - (double)ih);
    // window start: q at the trial centroid minus rho_sigma / dt (and a margin
    // far above the FP32 error of q)
    int bt;
    {
        const float u = fmaf(Dh2, dx2, fmaf(Dh1, dx1, Dh0 * dx0));
        const float ee = fmaf(dx2, dx2, fmaf(dx1, dx1, dx0 * dx0));
        const float tt = R0 + u;
        const float rr = sqrtf(fmaxf(fmaf(tt, tt, fmaf(-u, u, ee)), 0.f));
        const float qc = fmaf(rr - R0, ih, f0h);
        bt = (int)floorf(qc - su.rs[lane] - 1e-4f);
    }
#pragma unroll 1
    for (int y = 0; y < 7; ++y) {
        // r - R0 = u + e_perp^2 / ((R0 + u) + r) with u = D^.e, e the offset
        // difference and e_perp^2 = e.e - u^2; u carries the low part of D^
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
        int cell = (int)cf - bt;
        const float uq = (sh - cf) + low;
        const float x = uq + uq - 1.f;
        // weights w_y lambda_b(y) / r and w_y / r with FP32-pair weights, so
        // that their rounding is not a fixed bias shared by all element pairs
        const float irv = valid ? ir : 0.f;
        const float F0 = fmaf(irv, A.gwl[3 * y], irv * A.gwh[3 * y]);
        const float F1 = fmaf(irv, A.gwl[3 * y + 1], irv * A.gwh[3 * y + 1]);
        const float F2 = fmaf(irv, A.gwl[3 * y + 2], irv * A.gwh[3 * y + 2]);
        const float wr = fmaf(irv, A.wwl[y], irv * A.wwh[y]);
        if (cell < 0 || cell >= W) {
            if (valid) A.status[0] = ST_OFF_RANGE;
            cell = 0;
        }
        f2 v[TOTAL_LAG_PANELS];
        lag_panels(C, x, v);
        const f2 F01 = pk(F0, F1), F2W = pk(F2, wr);
        acc_class<W, C1>(a01, a2s, v, cell, F01, F2W);
        acc_class<W, C2>(a01, a2s, v, cell, F01, F2W);
        acc_class<W, C3>(a01, a2s, v, cell, F01, F2W);
    }
    // red shares its space with the previous chunk's P3 values: wait for it
    if (it > 0) mbar_wait(mbar, (unsigned)((it - 1) & 1), A.status);
#pragma unroll
    for (int s = 0; s < NT; ++s) {
        float t0, t1, t2, st;
        upk(a01[s], t0, t1);
        upk(a2s[s], t2, st);
        red[(xw * NT + s) * 32 + lane] = make_float4(t0, t1, t2, st);
    }
    rbase[xw * 32 + lane] = bt;
}

// Element-pair setup of one chunk (32 trial triangles) for test triangle tau
// in FP32-pair arithmetic from the FP32-pair centroids and geometry:
// centroid distance R0, lag base and fraction of R0 / dt, unit vector,
// trial points, window half-width and the geometric factors (with
// |tau||sigma|/(4 pi) folded in).
__device__ __forceinline__ void chunk_setup(const FarArgs &A, int64_t tau, int64_t ch, int lane, Setup32 &su) {
    const Geo &g = A.g;
    const int64_t E = g.E;
    const int64_t sg = ch * 32 + lane;
    const int32_t Ft0 = g.F[3 * tau], Ft1 = g.F[3 * tau + 1], Ft2 = g.F[3 * tau + 2];
    int valid = 0, base = 0;
    float f0h = 0.f, f0l = 0.f, R0 = 1.f, rs = 0.f;
    DF Dv[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    DF nn{0.f, 0.f}, cc[9];
    for (int k = 0; k < 9; ++k) cc[k] = DF{0.f, 0.f};
    if (sg < E) {
        const int32_t *B = g.F + 3 * sg;
        int shared = 0;
        for (int b = 0; b < 3; ++b) shared += (B[b] == Ft0) + (B[b] == Ft1) + (B[b] == Ft2);
        valid = shared == 0;
        DF d[3];
        for (int k = 0; k < 3; ++k)
            d[k] = df_add(DF{A.cenh[3 * tau + k], A.cenl[3 * tau + k]}, DF{-A.cenh[3 * sg + k], -A.cenl[3 * sg + k]});
        const DF r0 = df_sqrt(df_dot3(d, d));
        if (r0.h > 0.f) {
            const float ih = (float)A.lt.inv_dt, il = (float)(A.lt.inv_dt - (double)ih);
            const DF q0 = df_mul(r0, DF{ih, il});
            float fb = floorf(q0.h);
            DF f0 = df_fast(q0.h - fb, q0.l);  // q0.h - fb is exact
            if (f0.h < 0.f) { fb -= 1.f; f0 = df_add(f0, DF{1.f, 0.f}); }
            if (f0.h >= 1.f) { fb += 1.f; f0 = df_add(f0, DF{-1.f, 0.f}); }
            base = (int)fb;
            f0h = f0.h;
            f0l = f0.l;
            R0 = r0.h;
            const float ir = __frcp_rn(r0.h);
            for (int k = 0; k < 3; ++k) Dv[k] = df_div(d[k], r0, ir);
        }
        // geometric factors: |tau||sigma|/(4 pi) (n.n, curl_a.curl_b)
        const float *gth = A.geoh + 16 * tau, *gtl = A.geol + 16 * tau;
        const float *gsh = A.geoh + 16 * sg, *gsl = A.geol + 16 * sg;
        const DF sc = df_mul(df_mul(DF{gth[3], gtl[3]}, DF{gsh[3], gsl[3]}), DF{0.0795774715f, 3.1471446e-9f});
        DF a3[3], b3[3];
        for (int k = 0; k < 3; ++k) { a3[k] = DF{gth[k], gtl[k]}; b3[k] = DF{gsh[k], gsl[k]}; }
        nn = df_mul(sc, df_dot3(a3, b3));
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) {
                for (int k = 0; k < 3; ++k) {
                    a3[k] = DF{gth[4 + 3 * a + k], gtl[4 + 3 * a + k]};
                    b3[k] = DF{gsh[4 + 3 * b + k], gsl[4 + 3 * b + k]};
                }
                cc[3 * a + b] = df_mul(sc, df_dot3(a3, b3));
            }
        float rmax = 0.f;
        for (int k = 0; k < 7; ++k) {
            const float p0 = g.dq32[sg * 21 + 3 * k], p1 = g.dq32[sg * 21 + 3 * k + 1], p2 = g.dq32[sg * 21 + 3 * k + 2];
            su.dqy[lane][k][0] = p0;
            su.dqy[lane][k][1] = p1;
            su.dqy[lane][k][2] = p2;
            rmax = fmaxf(rmax, sqrtf(fmaf(p2, p2, fmaf(p1, p1, p0 * p0))));
        }
        rs = rmax * 1.0001f * (float)A.lt.inv_dt;
    } else {
        for (int k = 0; k < 21; ++k) su.dqy[lane][k / 3][k % 3] = 0.f;
    }
    su.nnh[lane] = nn.h;
    su.nnl[lane] = nn.l;
    for (int k = 0; k < 9; ++k) {
        su.cch[lane][k] = cc[k].h;
        su.ccl[lane][k] = cc[k].l;
    }
    su.valid[lane] = valid; su.base[lane] = base; su.f0h[lane] = f0h; su.f0l[lane] = f0l; su.R0[lane] = R0;
    su.rs[lane] = rs;
    for (int k = 0; k < 3; ++k) { su.Dh[lane][k] = Dv[k].h; su.Dl[lane][k] = Dv[k].l; }
    if (lane == 0) { su.tau = tau; su.ch = ch; su.Ft[0] = Ft0; su.Ft[1] = Ft1; su.Ft[2] = Ft2; }
}

// The chunk's scatter inputs. Plan: vertex list, sources (sigma_local * 3 +
// corner) per vertex (fetched by the producer during the previous chunk's
// P1), and the lag-window bounds of every (vertex, test corner, class) item
// (fetched by all threads during the previous chunk's P2): read-only inputs,
// so they are fetched one chunk ahead. Window values: copied (cp.async) into
// shared memory by the producer at the start of the chunk's P1, after the
// previous chunk's P3 has stored its windows; P3 then reads only shared
// memory.
struct Stage32 {
    int nv, nitems;
    int32_t vert[64];
    int32_t sptr[65];
    int32_t src[96];
};
// The plan of chunk ch: vertex list and sources (the same for every test
// triangle), fetched by one warp (lane = this thread's lane)
__device__ __forceinline__ void stage_chunk_plan(const FarArgs &A, int64_t ch, int lane, Stage32 &sg) {
    const int4 h = A.chunk_hdr[ch];  // v0, nv, x0, nsrc
    for (int v = lane; v < h.y; v += 32) sg.vert[v] = A.chunk_vert[h.x + v];
    for (int v = lane; v <= h.y; v += 32) sg.sptr[v] = A.chunk_sptr[h.x + v] - h.z;
    for (int x = lane; x < h.w; x += 32) sg.src[x] = A.chunk_src[h.z + x];
    if (lane == 0) { sg.nv = h.y; sg.nitems = h.y * 3 * NLAG; }
}
// the lag-window bounds and window rows (c M^2 + l M + j, below 2^31) of
// every item of a staged plan for test corners (Ft0, Ft1, Ft2), fetched by
// all threads of the CTA
__device__ __forceinline__ void stage_bounds(const FarArgs &A, int32_t Ft0, int32_t Ft1, int32_t Ft2,
                                             const Stage32 &sg, int16_t *swlo, int16_t *swhi, int32_t *srow) {
    const int64_t M = A.g.M, MM = M * M;
    for (int it = threadIdx.x; it < sg.nitems; it += F32_THREADS_ALL) {
        const int v = it / (3 * NLAG), rem = it % (3 * NLAG);
        const int a = rem / NLAG, c = rem % NLAG;
        const int64_t o = c * MM + (int64_t)(a == 0 ? Ft0 : a == 1 ? Ft1 : Ft2) * M + sg.vert[v];
        swlo[it] = A.dlo[o];
        swhi[it] = A.dhi[o];
        srow[it] = (int32_t)o;
    }
}
// row stride of the staged windows in FP32 pairs: odd, so that lanes reading
// different rows hit different shared-memory banks
__device__ __forceinline__ int kw_stride(int KW) { return KW | 1; }
__device__ __forceinline__ void stage_windows(const FarArgs &A, int lane, const Stage32 &sg, const int32_t *srow,
                                              FF *stg) {
    const int KW = A.KW, KS = kw_stride(KW);
    // lane per row: 8-byte copies of its KW words (a mapping of lanes onto
    // consecutive words of a few rows measured slower)
    for (int it = lane; it < sg.nitems; it += 32) {
        const FF *src = reinterpret_cast<const FF *>(A.dense) + (int64_t)srow[it] * KW;
        const unsigned dst = (unsigned)__cvta_generic_to_shared(stg + (size_t)it * KS);
        for (int k = 0; k < KW; ++k)
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;" ::"r"(dst + 8 * k), "l"(src + k));
    }
    asm volatile("cp.async.commit_group;" ::: "memory");
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

// Packed FP32-pair accumulators: value = h + l on both halves
struct F2F {
    f2 h, l;
};
__device__ __forceinline__ void ffp_add(F2F &a, f2 v) {  // a += v, two-sum of the high parts
    const f2 s = add2(a.h, v);
    const f2 bb = sub2(s, a.h);
    const f2 e = add2(sub2(a.h, sub2(s, bb)), sub2(v, bb));
    a.h = s;
    a.l = add2(a.l, e);
}
__device__ __forceinline__ void ffp_mac(F2F &a, f2 ch, f2 cl, f2 v) {  // a += (ch + cl) v
    const f2 p = mul2(ch, v);
    const f2 pe = fma2(cl, v, fma2(ch, v, sub2(0ull, p)));
    ffp_add(a, p);
    a.l = add2(a.l, pe);
}
__device__ __forceinline__ void ffp_macff(F2F &a, f2 ch, f2 cl, F2F v) {  // a += (ch + cl)(v.h + v.l)
    const f2 p = mul2(ch, v.h);
    const f2 pe = fma2(ch, v.l, fma2(cl, v.h, fma2(ch, v.h, sub2(0ull, p))));
    ffp_add(a, p);
    a.l = add2(a.l, pe);
}
__device__ __forceinline__ f2 lo_of(f2 v) {  // (v.lo, v.lo)
    float a, b;
    upk(v, a, b);
    return pk(a, a);
}
__device__ __forceinline__ f2 hi_of(f2 v) {  // (v.hi, v.hi)
    float a, b;
    upk(v, a, b);
    return pk(b, b);
}

// P2 item: union slot ug (0..NU-1) of trial triangle sl (lanes of a warp
// take consecutive trial triangles: conflict-free shared memory). The test
// points of the thread windows that cover the slot contribute their (t_0,
// t_1, t_2, s~) (a window that does not cover it gives zeros: no divergent
// branch). The sums over the 7 test points follow the orbits of the rule:
// with O_o the sum over orbit o and p_{o,a} its point whose distinguished
// corner is a,
//   S_ab = k_0 t_b(c) + k_1 O_1 + k_2 O_2 + d_1 t_b(p_{1,a}) + d_2 t_b(p_{2,a}),
//   S~   = w_0 s~(c) + w_1 O~_1 + w_2 O~_2,
// all in FP32-pair arithmetic; then L_ab = n.n' S_ab + curl_a.curl_b' S~.
template <int W>
__device__ __forceinline__ void reduce_item(const FarArgs &A, const Setup32 &su, const float4 *red, const int *rbase,
                                            int sl, int ug, FF (&L)[9], int &ubase) {
    constexpr int NT = Win<W>::NT;
    const int c = ug < Win<W>::ou(C2) ? C1 : (ug < Win<W>::ou(C3) ? C2 : C3);
    const int u = ug - (c == C1 ? Win<W>::ou(C1) : c == C2 ? Win<W>::ou(C2) : Win<W>::ou(C3));
    const int pt = c == C1 ? Win<W>::pt(C1) : c == C2 ? Win<W>::pt(C2) : Win<W>::pt(C3);
    const int ot = c == C1 ? Win<W>::ot(C1) : c == C2 ? Win<W>::ot(C2) : Win<W>::ot(C3);
    int b[F32_XW];
    ubase = 1 << 30;
#pragma unroll
    for (int x = 0; x < F32_XW; ++x) {
        b[x] = rbase[x * 32 + sl];
        ubase = min(ubase, b[x]);
    }
    f2 QA[F32_XW], QB[F32_XW];  // (t_0, t_1) and (t_2, s~) per test point
#pragma unroll
    for (int x = 0; x < F32_XW; ++x) {
        const int k = u - (b[x] - ubase);
        const bool in = k >= 0 && k < pt;
        const float4 q = red[(x * NT + ot + (in ? k : 0)) * 32 + sl];
        QA[x] = in ? pk(q.x, q.y) : 0ull;
        QB[x] = in ? pk(q.z, q.w) : 0ull;
    }
    // orbit sums
    F2F OA1{QA[1], 0ull}, OB1{QB[1], 0ull}, OA2{QA[4], 0ull}, OB2{QB[4], 0ull};
    ffp_add(OA1, QA[2]); ffp_add(OA1, QA[3]);
    ffp_add(OB1, QB[2]); ffp_add(OB1, QB[3]);
    ffp_add(OA2, QA[5]); ffp_add(OA2, QA[6]);
    ffp_add(OB2, QB[5]); ffp_add(OB2, QB[6]);
    // R = (R_0, R_1) and (R_2, S~)
    F2F RA{0ull, 0ull}, RB{0ull, 0ull};
    ffp_mac(RA, pk(A.okh[0], A.okh[0]), pk(A.okl[0], A.okl[0]), QA[0]);
    ffp_macff(RA, pk(A.okh[1], A.okh[1]), pk(A.okl[1], A.okl[1]), OA1);
    ffp_macff(RA, pk(A.okh[2], A.okh[2]), pk(A.okl[2], A.okl[2]), OA2);
    ffp_mac(RB, pk(A.okh[0], A.owh[0]), pk(A.okl[0], A.owl[0]), QB[0]);
    ffp_macff(RB, pk(A.okh[1], A.owh[1]), pk(A.okl[1], A.owl[1]), OB1);
    ffp_macff(RB, pk(A.okh[2], A.owh[2]), pk(A.okl[2], A.owl[2]), OB2);
    const f2 d1h = pk(A.odh[0], A.odh[0]), d1l = pk(A.odl[0], A.odl[0]);
    const f2 d2h = pk(A.odh[1], A.odh[1]), d2l = pk(A.odl[1], A.odl[1]);
    // (S_a0, S_a1), a = 0..2
    F2F SA[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        SA[a] = RA;
        ffp_mac(SA[a], d1h, d1l, QA[1 + a]);
        ffp_mac(SA[a], d2h, d2l, QA[4 + a]);
    }
    // (S_02, S_12) from (R_2, R_2); (S_22, S~) from (R_2, S~)
    F2F S2{lo_of(RB.h), lo_of(RB.l)};
    {
        float p0, p1, p2, p3, dum;
        upk(QB[1], p0, dum); upk(QB[2], p1, dum);
        ffp_mac(S2, d1h, d1l, pk(p0, p1));
        upk(QB[4], p2, dum); upk(QB[5], p3, dum);
        ffp_mac(S2, d2h, d2l, pk(p2, p3));
    }
    F2F SB = RB;
    {
        float p0, p1, dum;
        upk(QB[3], p0, dum); upk(QB[6], p1, dum);
        ffp_mac(SB, pk(A.odh[0], 0.f), pk(A.odl[0], 0.f), pk(p0, 0.f));
        ffp_mac(SB, pk(A.odh[1], 0.f), pk(A.odl[1], 0.f), pk(p1, 0.f));
    }
    // L_ab = n.n' S_ab + curl_a.curl_b' S~ (the primed factors carry
    // |tau||sigma|/(4 pi)), two entries per packed pair:
    // (L_a0, L_a1) for a = 0..2, (L_02, L_12), (L_22, -)
    const f2 Th = hi_of(SB.h), Tl = hi_of(SB.l);
    const f2 Nh = pk(su.nnh[sl], su.nnh[sl]), Nl = pk(su.nnl[sl], su.nnl[sl]);
    const float *cch = su.cch[sl], *ccl = su.ccl[sl];
    F2F Sv[5] = {SA[0], SA[1], SA[2], S2, SB};
    const int i0[5] = {0, 3, 6, 2, 8}, i1[5] = {1, 4, 7, 5, 8};
#pragma unroll
    for (int m = 0; m < 5; ++m) {
        const f2 Ch = pk(cch[i0[m]], cch[i1[m]]), Cl = pk(ccl[i0[m]], ccl[i1[m]]);
        const f2 ph = mul2(Nh, Sv[m].h);
        const f2 pl = add2(fma2(Nh, Sv[m].h, sub2(0ull, ph)), fma2(Nh, Sv[m].l, mul2(Nl, Sv[m].h)));
        const f2 qh = mul2(Ch, Th);
        const f2 ql = add2(fma2(Ch, Th, sub2(0ull, qh)), fma2(Ch, Tl, mul2(Cl, Th)));
        const f2 th = add2(ph, qh);
        const f2 bb = sub2(th, ph);
        const f2 tl = add2(add2(sub2(ph, sub2(th, bb)), sub2(qh, bb)), add2(pl, ql));
        const f2 lh = add2(th, tl);
        const f2 ll = sub2(tl, sub2(lh, th));
        float h0, h1, l0, l1;
        upk(lh, h0, h1);
        upk(ll, l0, l1);
        L[i0[m]] = FF{h0, l0};
        if (m < 4) L[i1[m]] = FF{h1, l1};
    }
}

// P3: thread per (trial vertex of the chunk, test corner, class): adds the
// values of the chunk's triangles at that vertex to the staged window (its
// own shared-memory copy), then stores the touched lags to the FP32-pair lag
// window of row F[tau][a]. Lb holds [NU][9][32] values, ub[sl] the lag of
// union slot 0 plus rho_c + P_c - 1.
template <int W>
__device__ __forceinline__ void scatter_chunk32(const FarArgs &A, const Setup32 &su, const Stage32 &sg, FF *stg,
                                                const int16_t *swlo, const int16_t *swhi, const int32_t *srow,
                                                const FF *Lb, const int *ub) {
    const int KW = A.KW;
    for (int it = threadIdx.x; it < sg.nitems; it += F32_THREADS_ALL) {
        const int v = it / (3 * NLAG), rem = it % (3 * NLAG);
        const int a = rem / NLAG, c = rem % NLAG;
        const int s0 = sg.sptr[v], s1 = sg.sptr[v + 1];
        const int P = cls_P(c);
        const int pu = c == C1 ? Win<W>::pu(C1) : c == C2 ? Win<W>::pu(C2) : Win<W>::pu(C3);
        const int ou = c == C1 ? Win<W>::ou(C1) : c == C2 ? Win<W>::ou(C2) : Win<W>::ou(C3);
        const int rho = A.lt.rho[c];
        const int wlo = swlo[it], whi = min((int)swhi[it], wlo + KW - 1);
        FF *cur = stg + (size_t)it * kw_stride(KW);
        int dmn = 1 << 30, dmx = -(1 << 30);
        for (int x = s0; x < s1; ++x) {
            const int src = sg.src[x], sl = src / 3, b = src % 3;
            if (!su.valid[sl]) continue;
            const int off = ub[sl] - rho - (P - 1);
            const int u0 = max(0, wlo - off), u1 = min(pu - 1, whi - off);
            if (u0 > u1) continue;
            dmn = min(dmn, off + u0);
            dmx = max(dmx, off + u1);
            const FF *lb = Lb + (ou * 9 + 3 * a + b) * 32 + sl;
            FF *cw = cur + (off - wlo);
#pragma unroll
            for (int u = 0; u < cls_P(C2) + 2 * W - 2; ++u)
                if (u >= u0 && u <= u1) cw[u] = ff_plus(cw[u], lb[u * 9 * 32]);
        }
        if (dmn > dmx) continue;
        FF *dst = reinterpret_cast<FF *>(A.dense) + (int64_t)srow[it] * KW;
        for (int d = dmn; d <= dmx; ++d) dst[d - wlo] = cur[d - wlo];
    }
}

// Special blocks (cell 0 and the first/last-row corner) are not evaluated
// here: the few far pairs that reach them go through farspec32_kernel
// (near32.cu), with FP64 distances and FP32-pair sums.
// Shared memory: two element-pair setups, the thread slots of P1 (reused for
// the 3x3 values of P2 once they are read), the window starts, the staged
// chunk plan and lag windows.
template <int W>
struct Smem32 {
    static constexpr size_t SETUP = ((2 * sizeof(Setup32) + 15) / 16) * 16;
    static constexpr size_t RED0 = sizeof(float4) * F32_XW * Win<W>::NT * 32;
    static constexpr size_t LB = sizeof(FF) * 32 * Win<W>::NU * 9;
    static constexpr size_t RED = RED0 > LB ? RED0 : LB;
    static constexpr size_t STAGE = ((sizeof(Stage32) + 15) / 16) * 16;
    static constexpr size_t FIXED = SETUP + RED + sizeof(int) * (F32_XW * 32 + 32) + 16 + 2 * STAGE;
    // plus the staged windows, (max_nv 9) x KW FP32 pairs, and two sets of
    // int16 bounds (this chunk's and the next one's)
    static size_t bytes(int KW, int max_nv) {
        const size_t items = (size_t)max_nv * 3 * NLAG;
        return FIXED + items * sizeof(FF) * (KW | 1) + ((4 * items * sizeof(int16_t) + 15) / 16) * 16 +
               2 * items * sizeof(int32_t);
    }
};

// two CTAs per SM (128 registers) for the common window of two cells; wider
// windows hold more slots and run one CTA per SM
template <int W>
__global__ void __launch_bounds__(F32_THREADS_ALL, W == 2 ? 2 : 1)
far32_kernel(const FarArgs A, const __grid_constant__ ChebLag32 C) {
    constexpr int NU = Win<W>::NU;
    constexpr int ITEMS = (32 * NU + F32_THREADS_ALL - 1) / F32_THREADS_ALL;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    unsigned char *p = smem_raw;
    Setup32 *sub = reinterpret_cast<Setup32 *>(p);       // [2]
    p += Smem32<W>::SETUP;
    float4 *red = reinterpret_cast<float4 *>(p);         // [7][NT][32] in P1 / P2
    FF *Lb = reinterpret_cast<FF *>(p);                  // [NU][9][32] in P3
    p += Smem32<W>::RED;
    int *rbase = reinterpret_cast<int *>(p);             // [7][32]
    int *ub = rbase + F32_XW * 32;                       // [32]
    unsigned long long *p3bar = reinterpret_cast<unsigned long long *>(ub + 32);  // P3 completion
    p += sizeof(int) * (F32_XW * 32 + 32) + 16;
    Stage32 *sgs = reinterpret_cast<Stage32 *>(p);       // [2]
    p += 2 * Smem32<W>::STAGE;
    const int nitm = A.max_nv * 3 * NLAG;
    FF *stg = reinterpret_cast<FF *>(p);                 // [max_nv 9][KW | 1]
    int16_t *sw = reinterpret_cast<int16_t *>(stg + (size_t)nitm * kw_stride(A.KW));  // [2][lo, hi][max_nv 9]
    int32_t *srw = reinterpret_cast<int32_t *>(sw + ((4 * nitm + 7) / 8) * 8);          // [2][max_nv 9]
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const bool producer = w == F32_XW;
    const Geo &g = A.g;
    const int64_t nch = A.nchunks;
    const int64_t ntau = A.ncolor > blockIdx.x ? (A.ncolor - 1 - blockIdx.x) / gridDim.x + 1 : 0;
    const int64_t nit = ntau * nch;
    if (nit == 0) return;
    const unsigned mbar = (unsigned)__cvta_generic_to_shared(p3bar);
    if (threadIdx.x == 0) mbar_init(mbar, F32_THREADS_ALL);
    {
        const int64_t t0 = A.color_tris[blockIdx.x];
        if (producer) {
            chunk_setup(A, t0, 0, lane, sub[0]);
            stage_chunk_plan(A, 0, lane, sgs[0]);
        }
        __syncthreads();
        stage_bounds(A, g.F[3 * t0], g.F[3 * t0 + 1], g.F[3 * t0 + 2], sgs[0], sw, sw + nitm, srw);
    }
    __syncthreads();
    int64_t cur_tau = -1;
    float dx0 = 0.f, dx1 = 0.f, dx2 = 0.f;
    for (int64_t it = 0; it < nit; ++it) {
        const int bf = (int)(it & 1);
        const Setup32 &su = sub[bf];
        Stage32 &sg = sgs[bf];
        int16_t *swlo = sw + 2 * nitm * bf, *swhi = swlo + nitm;
        int32_t *srow = srw + nitm * bf;
        if (producer) {
            // the staged windows, this plan's twin and the next setup were read by the previous P3
            if (it > 0) mbar_wait(mbar, (unsigned)((it - 1) & 1), A.status);
            stage_windows(A, lane, sg, srow, stg);
            if (it + 1 < nit) {
                const int64_t t2 = A.color_tris[blockIdx.x + ((it + 1) / nch) * gridDim.x];
                stage_chunk_plan(A, (it + 1) % nch, lane, sgs[bf ^ 1]);
                chunk_setup(A, t2, (it + 1) % nch, lane, sub[bf ^ 1]);
            }
        } else {
            if (su.tau != cur_tau) {
                cur_tau = su.tau;
                dx0 = g.dq32[(cur_tau * 7 + w) * 3 + 0];
                dx1 = g.dq32[(cur_tau * 7 + w) * 3 + 1];
                dx2 = g.dq32[(cur_tau * 7 + w) * 3 + 2];
            }
            quad_thread<W>(A, C, su, w, lane, dx0, dx1, dx2, red, rbase, mbar, it);
        }
        __syncthreads();  // P1 done: red, rbase, staged windows
        if (it + 1 < nit) {  // window bounds of the next chunk (read-only inputs)
            const Setup32 &sn = sub[bf ^ 1];
            int16_t *nlo = sw + 2 * nitm * (bf ^ 1);
            stage_bounds(A, sn.Ft[0], sn.Ft[1], sn.Ft[2], sgs[bf ^ 1], nlo, nlo + nitm, srw + nitm * (bf ^ 1));
        }
        FF L[ITEMS][9];
        int ubv[ITEMS];
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int k = threadIdx.x + r * F32_THREADS_ALL;
            if (k < 32 * NU) reduce_item<W>(A, su, red, rbase, k & 31, k >> 5, L[r], ubv[r]);
        }
        if (producer) asm volatile("cp.async.wait_all;" ::: "memory");  // staged windows landed
        __syncthreads();  // every read of red done: Lb may take its space
#pragma unroll
        for (int r = 0; r < ITEMS; ++r) {
            const int k = threadIdx.x + r * F32_THREADS_ALL;
            if (k < 32 * NU) {
                const int sl = k & 31, ug = k >> 5;
#pragma unroll
                for (int i = 0; i < 9; ++i) Lb[(ug * 9 + i) * 32 + sl] = L[r][i];
                if (ug == 0) ub[sl] = su.base[sl] + ubv[r];
            }
        }
        __syncthreads();  // Lb, ub written
        scatter_chunk32<W>(A, su, sg, stg, swlo, swhi, srow, Lb, ub);
        // P3 done for this thread: the next P1 runs on while others finish;
        // whoever reuses Lb (red), the staging or this setup waits for all
        mbar_arrive(mbar);
    }
}

template <int W>
static void launch32(const FarArgs &a, const ChebLag32 &c32, int grid, cudaStream_t st) {
    const size_t smem = Smem32<W>::bytes(a.KW, a.max_nv);
    cudaFuncSetAttribute(far32_kernel<W>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    far32_kernel<W><<<grid, F32_THREADS_ALL, smem, st>>>(a, c32);
}

int far32_window(double max_dq, double dt) {
    return (int)floor(2.0 * max_dq * 1.0001 / dt + 2e-4) + 2;
}

size_t far32_smem(int W, int KW, int max_nv) {
    if (max_nv > 64) return (size_t)1 << 40;  // the staged vertex list holds 64
    switch (W) {
        case 2: return Smem32<2>::bytes(KW, max_nv);
        case 3: return Smem32<3>::bytes(KW, max_nv);
        case 4: return Smem32<4>::bytes(KW, max_nv);
        default: return Smem32<5>::bytes(KW, max_nv);
    }
}

void launch_far32(const FarArgs &a, const ChebLag32 &c32, int W, int grid, cudaStream_t st) {
    if (W <= 2) launch32<2>(a, c32, grid, st);
    else if (W == 3) launch32<3>(a, c32, (grid + 1) / 2, st);
    else if (W == 4) launch32<4>(a, c32, (grid + 1) / 2, st);
    else launch32<5>(a, c32, (grid + 1) / 2, st);
}

}  // namespace tdbem
