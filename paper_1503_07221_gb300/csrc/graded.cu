// Assembly on a non-equidistant (graded) time grid (paper Sec. 3 with the
// basis of Eq. BasisFunctions on uneven steps; Sec. 3.2 for the cut-off).
// Without the shift invariance of an equidistant grid every nonzero block
// (k, i), i <= k + 1, is assembled from its own psi_{k,i} (Eq. psis), whose
// Chebyshev panels lie between the breakpoints t_{k-a} - t_{i-b}.
//
// Pattern: the kept blocks of a vertex pair (l, j) in trial column i are the
// k with a_{k,i} < Dmax(l,j) and b_{k,i} > Dmin(l,j), where Dmin / Dmax are
// the extreme element-pair bounds over the two vertex stars (both stars are
// connected, so the union of the element-pair distance ranges is one
// interval); a and b grow with k, so this is a contiguous range [K1, K2].
//
// Values are accumulated per batch of trial columns into FP64 windows
// [l][j][k - K1] (far) and [l][neighbour][k - K1] (near) and then gathered
// into per-block CSR. Conflict-free without atomics: a launch covers one
// colour of a vertex-disjoint triangle colouring on the test side (disjoint
// rows), and inside a CTA the trial triangles are taken one colour at a time
// with a barrier in between (disjoint columns).
#include <math.h>

#include "tdbem_internal.h"

namespace tdbem {

// ------------------------------------------------------------ column search
// first k with b_k > x (b nondecreasing in k); k0 + nk if none
__device__ __forceinline__ int g_kfirst(const double *b, int k0, int nk, double x) {
    int L = 0, H = nk;
    while (L < H) {
        const int m = (L + H) >> 1;
        if (b[m] > x) H = m; else L = m + 1;
    }
    return k0 + L;
}
// last k with a_k < x (a nondecreasing in k); k0 - 1 if none
__device__ __forceinline__ int g_klast(const double *a, int k0, int nk, double x) {
    int L = -1, H = nk - 1;
    while (L < H) {
        const int m = (L + H + 1) >> 1;
        if (a[m] < x) L = m; else H = m - 1;
    }
    return k0 + L;
}

// ------------------------------------------------------- packed FP32 pairs
typedef unsigned long long gf2;
__device__ __forceinline__ gf2 gpk(float lo, float hi) {
    gf2 r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void gupk(gf2 v, float &lo, float &hi) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ gf2 gfma2(gf2 a, gf2 b, gf2 c) {
    gf2 d;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
    return d;
}
__device__ __forceinline__ gf2 gsub2(gf2 a, gf2 b) {
    gf2 d;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
    return d;
}

// error-free sum of two floats
__device__ __forceinline__ void g_two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}
// (ah + al) * b as a float pair (h, l)
__device__ __forceinline__ void g_ff_mul(float ah, float al, float b, float &h, float &l) {
    h = __fmul_rn(ah, b);
    l = __fmaf_rn(al, b, __fmaf_rn(ah, b, -h));
}

// -------------------------------------------------- psi tables of a panel
// FP32 (mixed far field): Clenshaw recurrence on (psi, psi~) packed, the
// coefficients as float4 (c_psi[n], c_psi~[n], c_psi[n+1], c_psi~[n+1]),
// n = 0, 2, .., 32 (entry 33 is zero), then the FP32 residuals of c_0..c_3
// (float4 17 and 18) times T_0..T_3: the rounding of the leading
// coefficients would otherwise shift psi by the same amount at every point
// of the panel, an error the quadrature does not average away.
constexpr int GC32 = 19;  // float4 per panel
__device__ __forceinline__ void g_cheb32(const float4 *cf, float x, float &ps, float &pt) {
    const gf2 x2 = gpk(2.f * x, 2.f * x);
    gf2 b1 = 0ull, b2 = 0ull;
    {
        const float4 c = cf[16];
        b1 = gpk(c.x, c.y);  // n = 32
    }
#pragma unroll
    for (int h = 15; h >= 0; --h) {
        const float4 c = cf[h];
        gf2 b0 = gfma2(x2, b1, gsub2(gpk(c.z, c.w), b2));  // n = 2h + 1
        b2 = b1; b1 = b0;
        if (h > 0) {
            b0 = gfma2(x2, b1, gsub2(gpk(c.x, c.y), b2));   // n = 2h
            b2 = b1; b1 = b0;
        } else {
            const gf2 xx = gpk(x, x);
            b0 = gfma2(xx, b1, gsub2(gpk(c.x, c.y), b2));   // f = c_0 + x b_1 - b_2
            const float4 l01 = cf[17], l23 = cf[18];
            const float t2 = fmaf(2.f * x, x, -1.f), t3 = fmaf(2.f * x, t2, -x);
            gf2 cr = gfma2(gpk(t3, t3), gpk(l23.z, l23.w), gpk(l01.x, l01.y));
            cr = gfma2(gpk(t2, t2), gpk(l23.x, l23.y), cr);
            cr = gfma2(xx, gpk(l01.z, l01.w), cr);
            float c0, c1, f0, f1;
            gupk(cr, c0, c1);
            gupk(b0, f0, f1);
            ps = f0 + c0;
            pt = f1 + c1;
        }
    }
}

// FP64: panel p of the block (global index pg), S sub-panels of equal width,
// T_n recurrence with both sums.
__device__ __forceinline__ void g_cheb64(const GradedArgs &A, int pg, int np, double r, double &ps, double &pt) {
    int p = 0;
    while (p + 1 < np && r >= A.pan64[pg + p + 1].x) ++p;
    const GPan64 m = A.pan64[pg + p];  // (start, width, S / width, -)
    double u = (r - m.x) * m.z;
    int sub = (int)floor(u);
    sub = sub < 0 ? 0 : (sub >= A.S64 ? A.S64 - 1 : sub);
    u -= (double)sub;
    const double x = 2.0 * u - 1.0;
    const int set = A.p64[pg + p];
    if (set < 0) {  // no FP64 table for this panel (outside the near range)
        A.status[0] = ST_WINDOW;
        ps = 0.0; pt = 0.0;
        return;
    }
    const double *cf = A.coef64 + ((size_t)set + sub) * (NCHEB * 2);
    double s0 = __ldg(cf) + __ldg(cf + 2) * x, s1 = __ldg(cf + 1) + __ldg(cf + 3) * x;
    double tm = 1.0, t = x;
    const double x2 = x + x;
#pragma unroll 4
    for (int n = 2; n < NCHEB; ++n) {
        const double tn = x2 * t - tm;
        tm = t; t = tn;
        s0 += __ldg(cf + 2 * n) * tn;
        s1 += __ldg(cf + 2 * n + 1) * tn;
    }
    ps = s0; pt = s1;
}

// FP32 evaluation of NC panels at once (independent chains, interleaved so
// the dependent FMA sequences of one lane overlap). T_n by the three-term
// recurrence; the terms n >= 8 (a few 1e-3 of the panel maximum at most) are
// summed as the recurrence runs, then the FP32 residuals of c_0..c_3 and the
// terms n = 7..3 are added, and the three largest terms n = 2, 1, 0 last
// with exact products and a compensated (two-sum) accumulation. Relative to
// a plain FP32 Clenshaw sum this lowers the evaluation error about six-fold
// (CPU emulation at the torus grid: 1e-7 -> 1.5e-8 of the panel maximum).
template <int NC>
__device__ __forceinline__ void g_eval32(const float4 *const (&cf)[NC], const float (&x)[NC], float (&ps)[NC],
                                         float (&pt)[NC]) {
    float T[NC][8], tm[NC], tc[NC];
    gf2 hi[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        T[c][0] = 1.f;
        T[c][1] = x[c];
#pragma unroll
        for (int n = 2; n < 8; ++n) T[c][n] = fmaf(2.f * x[c], T[c][n - 1], -T[c][n - 2]);
        tm[c] = T[c][6];
        tc[c] = T[c][7];
        hi[c] = 0ull;
    }
#pragma unroll
    for (int h = 4; h <= 16; ++h) {
#pragma unroll
        for (int c = 0; c < NC; ++c) {
            const float4 q = cf[c][h];
            float t = fmaf(2.f * x[c], tc[c], -tm[c]);
            tm[c] = tc[c]; tc[c] = t;
            hi[c] = gfma2(gpk(t, t), gpk(q.x, q.y), hi[c]);  // n = 2h
            if (2 * h + 1 <= 32) {
                t = fmaf(2.f * x[c], tc[c], -tm[c]);
                tm[c] = tc[c]; tc[c] = t;
                hi[c] = gfma2(gpk(t, t), gpk(q.z, q.w), hi[c]);  // n = 2h + 1
            }
        }
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float4 l01 = cf[c][17], l23 = cf[c][18];
        gf2 a = hi[c];
        a = gfma2(gpk(T[c][3], T[c][3]), gpk(l23.z, l23.w), a);
        a = gfma2(gpk(T[c][2], T[c][2]), gpk(l23.x, l23.y), a);
        a = gfma2(gpk(T[c][1], T[c][1]), gpk(l01.z, l01.w), a);
        a = gfma2(gpk(1.f, 1.f), gpk(l01.x, l01.y), a);
        const float4 q3 = cf[c][3], q2 = cf[c][2], q1 = cf[c][1], q0 = cf[c][0];
        a = gfma2(gpk(T[c][7], T[c][7]), gpk(q3.z, q3.w), a);
        a = gfma2(gpk(T[c][6], T[c][6]), gpk(q3.x, q3.y), a);
        a = gfma2(gpk(T[c][5], T[c][5]), gpk(q2.z, q2.w), a);
        a = gfma2(gpk(T[c][4], T[c][4]), gpk(q2.x, q2.y), a);
        a = gfma2(gpk(T[c][3], T[c][3]), gpk(q1.z, q1.w), a);
        float s0, s1;
        gupk(a, s0, s1);
        float k0 = 0.f, k1 = 0.f;
        const float cc0[3] = {q1.x, q0.z, q0.x}, cc1[3] = {q1.y, q0.w, q0.y};
        const float tt[3] = {T[c][2], T[c][1], 1.f};
#pragma unroll
        for (int m = 0; m < 3; ++m) {
            float p = __fmul_rn(cc0[m], tt[m]), pe = __fmaf_rn(cc0[m], tt[m], -p), sn, e;
            g_two_sum(s0, p, sn, e);
            s0 = sn;
            k0 = __fadd_rn(k0, __fadd_rn(e, pe));
            p = __fmul_rn(cc1[m], tt[m]);
            pe = __fmaf_rn(cc1[m], tt[m], -p);
            g_two_sum(s1, p, sn, e);
            s1 = sn;
            k1 = __fadd_rn(k1, __fadd_rn(e, pe));
        }
        ps[c] = __fadd_rn(s0, k0);
        pt[c] = __fadd_rn(s1, k1);
    }
}

// Trial points y0 .. y0 + NC - 1 of one lane's (test point, block): distance
// from the FP64-anchored element-pair geometry, panel, argument, psi and psi~
// (g_eval32), and the weighted sums t_b += w_y lambda_b(y) psi / r, s~ +=
// w_y psi~ / r (weights as FP32 pairs). Points outside the block's support
// contribute zero.
// (h, l) += (gh + gl) v: exact product error and a two-sum into h
__device__ __forceinline__ void g_ff_acc(float &h, float &l, float gh, float gl, float v) {
    const float p = __fmul_rn(gh, v);
    const float pe = __fmaf_rn(gl, v, __fmaf_rn(gh, v, -p));
    float s, e;
    g_two_sum(h, p, s, e);
    h = s;
    l = __fadd_rn(l, __fadd_rn(e, pe));
}

// r - R0h of the point pair (x, y) of one element pair as (u, sl), u the
// leading part: D^.e with D^ = (c_tau - c_sigma)/|D| and e the difference of
// the FP32 offsets from the centroids, both as float pairs; sl = R0l + the
// small terms, with r - R0 = u + |e_perp|^2 / ((R0 + u) + r)
__device__ __forceinline__ float2 g_dist(const float *qx, const float *qy, const float (&Dn)[3], const float (&Dnl)[3],
                                         float R0h, float R0l) {
    float e0, e1, e2, l0, l1, l2;
    g_two_sum(qx[0], -qy[0], e0, l0);
    g_two_sum(qx[1], -qy[1], e1, l1);
    g_two_sum(qx[2], -qy[2], e2, l2);
    const float u = fmaf(Dn[0], e0, fmaf(Dn[1], e1, Dn[2] * e2));
    const float ul = fmaf(Dn[0], l0, fmaf(Dn[1], l1, fmaf(Dn[2], l2, fmaf(Dnl[0], e0, fmaf(Dnl[1], e1, Dnl[2] * e2)))));
    const float ee = fmaf(e0, e0, fmaf(e1, e1, e2 * e2));
    const float ep = fmaxf(fmaf(-u, u, ee), 0.f);
    const float r1 = sqrtf(fmaf(R0h, R0h, fmaf(2.f * R0h, u, ee)));
    const float q2 = ep / ((R0h + u) + r1);
    return make_float2(u, R0l + ul + q2);
}

template <int NC>
__device__ __forceinline__ void g_far_group(const GradedArgs &A, const float4 *scoef, const float4 *smeta,
                                            const float2 *dist, int y0, float R0h, float fa, float fb, int pb, int pe,
                                            float (&acc)[8]) {
    float x[NC], ir[NC], ps[NC], pt[NC];
    bool in[NC];
    const float4 *cf[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const float2 du = dist[y0 + c];
        const float u = du.x, sl = du.y;
        const float s = u + sl;
        const float rr = R0h + s;
        in[c] = rr > fa && rr < fb;
        int p = pb;
        if (in[c])
            while (p + 1 < pe && rr >= smeta[p + 1].x) ++p;
        const float4 mt = smeta[p];  // (start, mid_h, mid_l, 2 / width)
        x[c] = in[c] ? fminf(fmaxf(((R0h - mt.y) + u + (sl - mt.z)) * mt.w, -1.f), 1.f) : 0.f;
        ir[c] = __frcp_rn(rr);
        cf[c] = scoef + (size_t)p * GC32;
    }
    g_eval32<NC>(cf, x, ps, pt);
#pragma unroll
    for (int c = 0; c < NC; ++c) {
        const int y = y0 + c;
        const float v = in[c] ? ps[c] * ir[c] : 0.f, vt = in[c] ? pt[c] * ir[c] : 0.f;
        g_ff_acc(acc[0], acc[1], A.gwh[3 * y], A.gwl[3 * y], v);
        g_ff_acc(acc[2], acc[3], A.gwh[3 * y + 1], A.gwl[3 * y + 1], v);
        g_ff_acc(acc[4], acc[5], A.gwh[3 * y + 2], A.gwl[3 * y + 2], v);
        g_ff_acc(acc[6], acc[7], A.wwh[y], A.wwl[y], vt);
    }
}

// ---------------------------------------------------------------- far field
// CTA = GF_WARPS warps over the test triangles of one colour; per trial
// column of the batch the column's panel tables are staged in shared memory
// (FP32 path). A warp takes one far element pair at a time: lane = (block
// slot ks, test point x) = 8 ks + x, x < 7, four blocks of the element pair's
// kept range per round, each lane summing over the 7 trial points; the sums
// over the test points are shuffle reductions inside the 8-lane groups.
size_t gfar_smem(int maxpan, bool fp64) {
    size_t s = 2 * GP_MAXK * sizeof(double) + (GP_MAXK + 4) * sizeof(int);
    if (!fp64) s += (size_t)maxpan * sizeof(float4) * (1 + GC32);
    return s;
}

constexpr int GF_LIST = 1024;  // trial triangles compacted per pass

template <bool FP64>
__global__ void __launch_bounds__(GF_WARPS * 32, 1) gfar_kernel(const GradedArgs A) {
    extern __shared__ __align__(16) unsigned char g_sm[];
    double *sa = reinterpret_cast<double *>(g_sm);
    double *sb = sa + GP_MAXK;
    int *sp0 = reinterpret_cast<int *>(sb + GP_MAXK);
    float4 *smeta = reinterpret_cast<float4 *>(sp0 + GP_MAXK + 4);
    float4 *scoef = smeta + A.maxpan;
    __shared__ int2 s_list[GF_LIST];  // kept far pairs: (sigma, K1 << 16 | K2)
    __shared__ int s_cnt, s_next;
    __shared__ float2 s_dist[GF_WARPS][56];  // per warp: (u, sl) of the 49 point pairs, index 7 x + y
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int xs = lane & 7, ks = lane >> 3;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E;
    for (int ci = A.i0; ci < A.i1; ++ci) {
        const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
        if (nk <= 0) continue;
        const int pbase = A.pan0[cb0], npan = A.pan0[cb0 + nk] - pbase;
        __syncthreads();
        for (int t = threadIdx.x; t < nk; t += blockDim.x) {
            sa[t] = A.ga[cb0 + t];
            sb[t] = A.gb[cb0 + t];
            sp0[t] = A.pan0[cb0 + t] - pbase;
        }
        if (threadIdx.x == 0) sp0[nk] = npan;
        if constexpr (!FP64) {
            for (int t = threadIdx.x; t < npan; t += blockDim.x) smeta[t] = A.pan32[pbase + t];
            const float4 *src = reinterpret_cast<const float4 *>(A.coef32) + (size_t)pbase * GC32;
            for (int t = threadIdx.x; t < npan * GC32; t += blockDim.x) scoef[t] = src[t];
        }
        __syncthreads();
        const int KW = A.kw[ci];
        double *dense = A.dense + A.doff[ci - A.i0];
        for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
            const int64_t tau = A.color_tris[ti];
            const int Ft0 = g.F[3 * tau], Ft1 = g.F[3 * tau + 1], Ft2 = g.F[3 * tau + 2];
            // this lane's test point (offset from the centroid)
            float ex[3] = {0.f, 0.f, 0.f};
            double exd[3] = {0.0, 0.0, 0.0};
            if (xs < 7)
                for (int d = 0; d < 3; ++d) {
                    if constexpr (FP64) exd[d] = g.dq[(tau * 7 + xs) * 3 + d];
                    else ex[d] = g.dq32[(tau * 7 + xs) * 3 + d];
                }
            for (int c2 = 0; c2 < A.ncol; ++c2) {
                // the colour's trial triangles GF_LIST at a time: (1) each lane decides
                // one (far pair, kept range) and the kept pairs are compacted into a
                // shared list; (2) warps take list entries one at a time from a shared
                // counter (balanced; entries of one trial colour share no vertex, so
                // the order does not change any sum)
                const int64_t cend = A.col_off[c2 + 1];
                for (int64_t pbeg = A.col_off[c2]; pbeg < cend; pbeg += GF_LIST) {
                  const int64_t pend = min(cend, pbeg + (int64_t)GF_LIST);
                  if (threadIdx.x == 0) { s_cnt = 0; s_next = 0; }
                  __syncthreads();
                  for (int64_t sb0 = pbeg + 32 * w; sb0 < pend; sb0 += 32 * GF_WARPS) {
                      int K1l = 1, K2l = 0;
                      int sgl = 0;
                      if (sb0 + lane < pend) {
                          sgl = A.all_tris[sb0 + lane];
                          const int q0 = g.F[3 * (int64_t)sgl], q1 = g.F[3 * (int64_t)sgl + 1], q2 = g.F[3 * (int64_t)sgl + 2];
                          const bool adj = Ft0 == q0 || Ft0 == q1 || Ft0 == q2 || Ft1 == q0 || Ft1 == q1 ||
                                           Ft1 == q2 || Ft2 == q0 || Ft2 == q1 || Ft2 == q2;
                          if (!adj) {
                              const double2 bd = A.pair[tau * E + sgl];
                              K1l = g_kfirst(sb, k0, nk, bd.x + A.tie);
                              K2l = g_klast(sa, k0, nk, bd.y - A.tie);
                          }
                      }
                      const bool keep = K1l <= K2l;
                      const unsigned bal = __ballot_sync(0xffffffffu, keep);
                      int base = 0;
                      if (lane == 0 && bal) base = atomicAdd(&s_cnt, __popc(bal));
                      base = __shfl_sync(0xffffffffu, base, 0);
                      if (keep) s_list[base + __popc(bal & ((1u << lane) - 1u))] = make_int2(sgl, (K1l << 16) | K2l);
                  }
                  __syncthreads();
                  const int nlist = s_cnt;
                  for (;;) {
                    int it = 0;
                    if (lane == 0) it = atomicAdd(&s_next, 1);
                    it = __shfl_sync(0xffffffffu, it, 0);
                    if (it >= nlist) break;
                    const int2 ent = s_list[it];
                    const int64_t sg = ent.x;
                    const int K1 = ent.y >> 16, K2 = ent.y & 0xffff;
                    const int Fs0 = g.F[3 * sg], Fs1 = g.F[3 * sg + 1], Fs2 = g.F[3 * sg + 2];
                    // window starts of the nine vertex pairs (lane e = 3a + b)
                    int K1e = 0;
                    if (lane < 9) {
                        const int a = lane / 3, b = lane % 3;
                        const int64_t l = a == 0 ? Ft0 : (a == 1 ? Ft1 : Ft2);
                        const int64_t j = b == 0 ? Fs0 : (b == 1 ? Fs1 : Fs2);
                        K1e = g_kfirst(sb, k0, nk, A.vmin[l * M + j] + A.tie);
                    }
                    // element-pair geometry
                    float R0h = 0.f, R0l = 0.f, Dn[3] = {0.f, 0.f, 0.f}, Dnl[3] = {0.f, 0.f, 0.f};
                    double cd[3] = {0.0, 0.0, 0.0};
                    if constexpr (FP64) {
                        for (int d = 0; d < 3; ++d) cd[d] = g.cen[3 * tau + d] - g.cen[3 * sg + d];
                    } else {
                        // D = c_tau - c_sigma from the centroid pairs, |D| as a float pair
                        float Dh[3], Dl[3];
                        for (int d = 0; d < 3; ++d) {
                            float s, e;
                            g_two_sum(A.cenh[3 * tau + d], -A.cenh[3 * sg + d], s, e);
                            e = __fadd_rn(e, __fsub_rn(A.cenl[3 * tau + d], A.cenl[3 * sg + d]));
                            Dh[d] = __fadd_rn(s, e);
                            Dl[d] = __fsub_rn(e, __fsub_rn(Dh[d], s));
                        }
                        float Sh = 0.f, Sl = 0.f;
                        for (int d = 0; d < 3; ++d) {
                            const float p = __fmul_rn(Dh[d], Dh[d]);
                            const float pe = __fmaf_rn(Dh[d], Dh[d], -p);
                            float s, e;
                            g_two_sum(Sh, p, s, e);
                            Sh = s;
                            Sl = __fadd_rn(Sl, __fadd_rn(e, __fmaf_rn(2.f * Dh[d], Dl[d], pe)));
                        }
                        R0h = sqrtf(Sh);
                        R0l = __fdiv_rn(__fadd_rn(__fmaf_rn(-R0h, R0h, Sh), Sl), 2.f * R0h);
                        const float inv = __frcp_rn(R0h);
                        // unit vector D / |D| as a float pair (hi, lo)
                        for (int d = 0; d < 3; ++d) {
                            Dn[d] = __fmul_rn(__fadd_rn(Dh[d], Dl[d]), inv);
                            const float res = __fsub_rn(__fadd_rn(__fmaf_rn(-Dn[d], R0h, Dh[d]), Dl[d]), __fmul_rn(Dn[d], R0l));
                            Dnl[d] = __fmul_rn(res, inv);
                        }
                        // the 49 point-pair distances, once per element pair (every block
                        // round of the warp reads them)
                        __syncwarp();
                        for (int it = lane; it < 49; it += 32) {
                            const int px = it / 7, py = it % 7;
                            s_dist[w][it] = g_dist(g.dq32 + (tau * 7 + px) * 3, g.dq32 + (sg * 7 + py) * 3, Dn, Dnl,
                                                   R0h, R0l);
                        }
                        __syncwarp();
                    }
                    for (int base = K1; base <= K2; base += GP_KSLOT) {
                        const int k = base + ks;
                        const bool act = xs < 7 && k <= K2;
                        const int cbl = act ? k - k0 : 0;
                        const int pb = sp0[cbl], pe = sp0[cbl + 1];
                        // sums over the trial points: t_b = sum_y w_y lambda_b(y) psi / r, s~ = sum_y w_y psi~ / r
                        double t0 = 0.0, t1 = 0.0, t2 = 0.0, ts = 0.0;
                        float f0 = 0.f, f1 = 0.f, f2 = 0.f, fs = 0.f;   // float pairs (f, fl)
                        float f0l = 0.f, f1l = 0.f, f2l = 0.f, fsl = 0.f;
                        if (act) {
                            if constexpr (FP64) {
                                const double ba = sa[cbl], bb = sb[cbl];
                                for (int y = 0; y < 7; ++y) {
                                    double r2 = 0.0;
                                    for (int d = 0; d < 3; ++d) {
                                        const double v = cd[d] + (exd[d] - g.dq[(sg * 7 + y) * 3 + d]);
                                        r2 += v * v;
                                    }
                                    const double r = sqrt(r2);
                                    if (!(r > ba && r < bb)) continue;
                                    double ps, pt;
                                    g_cheb64(A, A.pan0[cb0] + pb, pe - pb, r, ps, pt);
                                    const double v = ps / r, vt = pt / r;
                                    t0 += A.rule_w64[y] * A.rule_l64[3 * y] * v;
                                    t1 += A.rule_w64[y] * A.rule_l64[3 * y + 1] * v;
                                    t2 += A.rule_w64[y] * A.rule_l64[3 * y + 2] * v;
                                    ts += A.rule_w64[y] * vt;
                                }
                            } else {
                                const float fa = (float)sa[cbl], fb = (float)sb[cbl];
                                const float4 *scf = scoef;
                                const float4 *smt = smeta;
                                float acc[8] = {f0, f0l, f1, f1l, f2, f2l, fs, fsl};
                                const float2 *dist = &s_dist[w][7 * xs];
                                g_far_group<4>(A, scf, smt, dist, 0, R0h, fa, fb, pb, pe, acc);
                                g_far_group<3>(A, scf, smt, dist, 4, R0h, fa, fb, pb, pe, acc);
                                f0 = acc[0]; f0l = acc[1]; f1 = acc[2]; f1l = acc[3];
                                f2 = acc[4]; f2l = acc[5]; fs = acc[6]; fsl = acc[7];
                            }
                        }
                        // weighted by the test point: S_ab = sum_x w_x lambda_a(x) t_b, S~ = sum_x w_x s~
                        if constexpr (FP64) {
                            double S[10];
                            const int xx = xs < 7 ? xs : 0;
                            const double wx = xs < 7 ? A.rule_w64[xx] : 0.0;
                            for (int a = 0; a < 3; ++a) {
                                const double gxa = wx * A.rule_l64[3 * xx + a];
                                S[3 * a] = gxa * t0; S[3 * a + 1] = gxa * t1; S[3 * a + 2] = gxa * t2;
                            }
                            S[9] = wx * ts;
#pragma unroll
                            for (int o = 1; o < 8; o <<= 1)
                                for (int q = 0; q < 10; ++q) S[q] += __shfl_xor_sync(0xffffffffu, S[q], o);
                            const double nn = g.geo64[16 * tau] * g.geo64[16 * sg] +
                                              g.geo64[16 * tau + 1] * g.geo64[16 * sg + 1] +
                                              g.geo64[16 * tau + 2] * g.geo64[16 * sg + 2];
                            const double sc = g.geo64[16 * tau + 3] * g.geo64[16 * sg + 3] * 0.07957747154594767;
                            for (int rep = 0; rep < 2; ++rep) {
                                const int e = xs + 8 * rep;
                                const int Ke = __shfl_sync(0xffffffffu, K1e, e < 9 ? e : 0);
                                if (e >= 9 || k > K2) continue;
                                const int a = e / 3, b = e % 3;
                                const double *ct = g.geo64 + 16 * tau + 4 + 3 * a, *cs = g.geo64 + 16 * sg + 4 + 3 * b;
                                const double cc = ct[0] * cs[0] + ct[1] * cs[1] + ct[2] * cs[2];
                                const double L = sc * (nn * S[e] + cc * S[9]);
                                const int slot = k - Ke;
                                if (slot < 0 || slot >= KW) { A.status[0] = ST_WINDOW; continue; }
                                const int64_t l = a == 0 ? Ft0 : (a == 1 ? Ft1 : Ft2);
                                const int64_t j = b == 0 ? Fs0 : (b == 1 ? Fs1 : Fs2);
                                dense[(l * M + j) * KW + slot] += L;
                            }
                        } else {
                            // S_ab = sum_x (w_x lambda_a(x)) t_b(x) and S~ in float pairs: products of
                            // the (hi, lo) weights and the (hi, lo) trial sums, then a two-sum
                            // reduction over the 8 lanes of the group
                            float S[10], SL[10];
                            const int xx = xs < 7 ? xs : 0;
                            const float th[3] = {f0, f1, f2}, tlo[3] = {f0l, f1l, f2l};
                            for (int a = 0; a < 3; ++a) {
                                const float gh = xs < 7 ? A.gwh[3 * xx + a] : 0.f, gl = xs < 7 ? A.gwl[3 * xx + a] : 0.f;
                                for (int b = 0; b < 3; ++b) {
                                    S[3 * a + b] = __fmul_rn(gh, th[b]);
                                    SL[3 * a + b] = __fmaf_rn(gh, tlo[b], __fmaf_rn(gl, th[b], __fmaf_rn(gh, th[b], -S[3 * a + b])));
                                }
                            }
                            {
                                const float gh = xs < 7 ? A.wwh[xx] : 0.f, gl = xs < 7 ? A.wwl[xx] : 0.f;
                                S[9] = __fmul_rn(gh, fs);
                                SL[9] = __fmaf_rn(gh, fsl, __fmaf_rn(gl, fs, __fmaf_rn(gh, fs, -S[9])));
                            }
#pragma unroll
                            for (int o = 1; o < 8; o <<= 1)
                                for (int q = 0; q < 10; ++q) {
                                    const float oh = __shfl_xor_sync(0xffffffffu, S[q], o);
                                    const float ol = __shfl_xor_sync(0xffffffffu, SL[q], o);
                                    float sh, se;
                                    g_two_sum(S[q], oh, sh, se);
                                    S[q] = sh;
                                    SL[q] = __fadd_rn(__fadd_rn(SL[q], ol), se);
                                }
                            // combination L_ab = |tau||sigma|/(4 pi) (n.n S_ab + curl_a.curl_b S~) in
                            // float-pair arithmetic from the FP32-pair geometry of both triangles
                            const float *gt = A.geoh + 16 * tau, *gs = A.geoh + 16 * sg;
                            const float *lt = A.geol + 16 * tau, *ls = A.geol + 16 * sg;
                            float nnh = 0.f, nnl = 0.f;
                            for (int d = 0; d < 3; ++d) {
                                const float p = __fmul_rn(gt[d], gs[d]);
                                const float pe = __fmaf_rn(gt[d], gs[d], -p);
                                float s, e;
                                g_two_sum(nnh, p, s, e);
                                nnh = s;
                                nnl = __fadd_rn(nnl, __fadd_rn(e, __fmaf_rn(gt[d], ls[d], __fmaf_rn(lt[d], gs[d], pe))));
                            }
                            float sch, scl;
                            {
                                const float p = __fmul_rn(gt[3], gs[3]);
                                const float pe = __fmaf_rn(gt[3], gs[3], -p);
                                const float pl = __fmaf_rn(gt[3], ls[3], __fmaf_rn(lt[3], gs[3], pe));
                                // times 1/(4 pi) as a float pair
                                const float ch = 0.07957746833562851f, cl = 3.2103191632826267e-09f;
                                sch = __fmul_rn(p, ch);
                                scl = __fmaf_rn(p, cl, __fmaf_rn(pl, ch, __fmaf_rn(p, ch, -sch)));
                            }
                            for (int rep = 0; rep < 2; ++rep) {
                                const int e = xs + 8 * rep;
                                const int Ke = __shfl_sync(0xffffffffu, K1e, e < 9 ? e : 0);
                                if (e >= 9 || k > K2) continue;
                                const int a = e / 3, b = e % 3;
                                float cch = 0.f, ccl = 0.f;
                                for (int d = 0; d < 3; ++d) {
                                    const float ta = gt[4 + 3 * a + d], sbv = gs[4 + 3 * b + d];
                                    const float p = __fmul_rn(ta, sbv);
                                    const float pe = __fmaf_rn(ta, sbv, -p);
                                    float s, ee;
                                    g_two_sum(cch, p, s, ee);
                                    cch = s;
                                    ccl = __fadd_rn(ccl, __fadd_rn(ee, __fmaf_rn(ta, ls[4 + 3 * b + d],
                                                                              __fmaf_rn(lt[4 + 3 * a + d], sbv, pe))));
                                }
                                float ah, al, bh, bl, s, ee;
                                g_ff_mul(nnh, nnl, S[e], ah, al);
                                g_ff_mul(cch, ccl, S[9], bh, bl);
                                al = __fmaf_rn(nnh, SL[e], al);
                                bl = __fmaf_rn(cch, SL[9], bl);
                                g_two_sum(ah, bh, s, ee);
                                const float sl = __fadd_rn(ee, __fadd_rn(al, bl));
                                const float Lh = __fmul_rn(sch, s);
                                const float Ll = __fmaf_rn(sch, sl, __fmaf_rn(scl, s, __fmaf_rn(sch, s, -Lh)));
                                const int slot = k - Ke;
                                if (slot < 0 || slot >= KW) { A.status[0] = ST_WINDOW; continue; }
                                const int64_t l = a == 0 ? Ft0 : (a == 1 ? Ft1 : Ft2);
                                const int64_t j = b == 0 ? Fs0 : (b == 1 ? Fs1 : Fs2);
                                dense[(l * M + j) * KW + slot] += (double)Lh + (double)Ll;
                            }
                        }
                    }
                  }
                  __syncthreads();
                }
            }
        }
    }
}

void launch_gfar(const GradedArgs &a, bool fp64, int grid, size_t smem, cudaStream_t st) {
    if (grid <= 0) return;
    if (fp64) {
        cudaFuncSetAttribute(gfar_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        gfar_kernel<true><<<grid, GF_WARPS * 32, smem, st>>>(a);
    } else {
        cudaFuncSetAttribute(gfar_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        gfar_kernel<false><<<grid, GF_WARPS * 32, smem, st>>>(a);
    }
}

// --------------------------------------------------------------- near field
// CTA per test triangle of the colour; its adjacent trial triangles one after
// another (they share vertices among themselves). Point pairs of the
// Sauter-Schwab rule are staged GN_TILE at a time (FP64 r, weight / r and the
// barycentrics); the kept blocks of every batch column are the items, one
// warp per item, lanes over the staged point pairs. FP64 path: FP64 tables
// throughout. F32 (mixed path): per point pair r as an FP32 pair and the
// weight w / r as an FP32 pair; per (point pair, block) the panel found in
// FP32, its argument from the FP32-pair distance against the panel's midpoint
// pair, psi and psi~ from the panel's FP32 expansion with the residuals of
// its leading coefficients (g_cheb32), and the nine sums S_ab and S~ as FP32
// pairs (two-sum), added across the warp in FP64.
__device__ static inline double g_dsum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int GN_ITEMS = 256;

__device__ __forceinline__ void gn_two_sum_add(float &h, float &l, float v) {
    const float s = h + v;
    const float bb = s - h;
    l += (h - (s - bb)) + (v - bb);
    h = s;
}

template <bool F32>
__global__ void __launch_bounds__(GN_WARPS * 32) gnear_kernel(const GradedArgs A) {
    __shared__ double q[GN_TILE * 6];
    __shared__ float qf[F32 ? GN_TILE * 8 : 1];  // rh, rl, wh, wl, lx0, lx1, ly0, ly1
    __shared__ double acc[GN_ITEMS * 10];
    __shared__ int items[GN_ITEMS];  // (batch column << 16) | (k - k0 of that column)
    __shared__ int nitems, ntotal;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E;
    for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
        const int64_t tau = A.color_tris[ti];
        for (int64_t pi = A.adj_ptr[tau]; pi < A.adj_ptr[tau + 1]; ++pi) {
            const int64_t sg = A.adj_tri[pi];
            const int8_t *pm = A.adj_perm + 8 * pi;
            const int kase = pm[0];
            const int pa[3] = {pm[1], pm[2], pm[3]}, pb[3] = {pm[4], pm[5], pm[6]};
            const int npp = A.ss_npp[kase];
            const double *rule = A.ss_xy[kase];
            const double dmax = A.pair[tau * E + sg].y;
            double X[3][3], Y[3][3];
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) {
                    X[k][d] = g.V[3 * g.F[3 * tau + pa[k]] + d];
                    Y[k][d] = g.V[3 * g.F[3 * sg + pb[k]] + d];
                }
            const double at = g.geo64[16 * tau + 3], as = g.geo64[16 * sg + 3];
            const double scale = 4.0 * at * as * 0.07957747154594767;  // |J| = 2|T| on both sides, 1/(4 pi)
            const double nn = g.geo64[16 * tau] * g.geo64[16 * sg] + g.geo64[16 * tau + 1] * g.geo64[16 * sg + 1] +
                              g.geo64[16 * tau + 2] * g.geo64[16 * sg + 2];
            // items: kept blocks of every batch column for this element pair (dmin = 0)
            if (threadIdx.x == 0) {
                int n = 0;
                for (int ci = A.i0; ci < A.i1; ++ci) {
                    const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
                    if (nk <= 0) continue;
                    const int K1 = g_kfirst(A.gb + cb0, k0, nk, 0.0 + A.tie);
                    const int K2 = g_klast(A.ga + cb0, k0, nk, dmax - A.tie);
                    for (int k = K1; k <= K2; ++k) {
                        if (n < GN_ITEMS) items[n] = ((ci - A.i0) << 16) | (k - k0);
                        ++n;
                    }
                }
                ntotal = n;
            }
            __syncthreads();
            const int nt = ntotal;
            for (int ib = 0; ib < nt; ib += GN_ITEMS) {
                if (ib > 0) {
                    // items beyond the first GN_ITEMS: rebuild the list for this chunk
                    __syncthreads();
                    if (threadIdx.x == 0) {
                        int n = 0;
                        for (int ci = A.i0; ci < A.i1; ++ci) {
                            const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
                            if (nk <= 0) continue;
                            const int K1 = g_kfirst(A.gb + cb0, k0, nk, 0.0 + A.tie);
                            const int K2 = g_klast(A.ga + cb0, k0, nk, dmax - A.tie);
                            for (int k = K1; k <= K2; ++k) {
                                if (n >= ib && n < ib + GN_ITEMS) items[n - ib] = ((ci - A.i0) << 16) | (k - k0);
                                ++n;
                            }
                        }
                    }
                }
                if (threadIdx.x == 0) nitems = min(GN_ITEMS, nt - ib);
                for (int t = threadIdx.x; t < GN_ITEMS * 10; t += blockDim.x) acc[t] = 0.0;
                __syncthreads();
                const int ni = nitems;
                for (int p0 = 0; p0 < npp; p0 += GN_TILE) {
                    const int np = min(GN_TILE, npp - p0);
                    __syncthreads();
                    for (int p = threadIdx.x; p < np; p += blockDim.x) {
                        const double *rr = rule + 5 * (p0 + p);
                        const double xh0 = rr[0], xh1 = rr[1], yh0 = rr[2], yh1 = rr[3];
                        double r2 = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            const double xd = X[0][d] + xh0 * (X[1][d] - X[0][d]) + xh1 * (X[2][d] - X[1][d]);
                            const double yd = Y[0][d] + yh0 * (Y[1][d] - Y[0][d]) + yh1 * (Y[2][d] - Y[1][d]);
                            r2 += (xd - yd) * (xd - yd);
                        }
                        const double r = sqrt(r2);
                        if constexpr (F32) {
                            float *qq = qf + 8 * p;
                            const double wr = rr[4] * scale / r;
                            qq[0] = (float)r; qq[1] = (float)(r - (double)qq[0]);
                            qq[2] = (float)wr; qq[3] = (float)(wr - (double)qq[2]);
                            qq[4] = (float)(1.0 - xh0); qq[5] = (float)(xh0 - xh1);
                            qq[6] = (float)(1.0 - yh0); qq[7] = (float)(yh0 - yh1);
                        } else {
                            double *qq = q + 6 * p;
                            qq[0] = r;
                            qq[1] = rr[4] * scale / r;
                            qq[2] = 1.0 - xh0; qq[3] = xh0 - xh1;
                            qq[4] = 1.0 - yh0; qq[5] = yh0 - yh1;
                        }
                    }
                    __syncthreads();
                    for (int it = w; it < ni; it += GN_WARPS) {
                        const int ci = A.i0 + (items[it] >> 16), kl = items[it] & 0xffff;
                        const int cb = A.colblk[ci] + kl;
                        const double ba = A.ga[cb], bb = A.gb[cb];
                        const int pg = A.pan0[cb], npn = A.pan0[cb + 1] - pg;
                        double Sab[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, St = 0.0;
                        if constexpr (F32) {
                            const float ba32 = (float)ba, bb32 = (float)bb;
                            float Sh[9], Sl[9], Th = 0.f, Tl = 0.f;
#pragma unroll
                            for (int e = 0; e < 9; ++e) Sh[e] = Sl[e] = 0.f;
                            for (int p = lane; p < np; p += 32) {
                                const float *qq = qf + 8 * p;
                                const float rh = qq[0], rl = qq[1];
                                if (!(rh > ba32 && rh < bb32)) continue;
                                int pp = 0;
                                while (pp + 1 < npn && rh >= A.pan32[pg + pp + 1].x) ++pp;
                                const float4 mt = A.pan32[pg + pp];  // (start_h, mid_h, mid_l, 2 / width)
                                const float x = ((rh - mt.y) + (rl - mt.z)) * mt.w;
                                float ps, pt;
                                g_cheb32(reinterpret_cast<const float4 *>(A.coef32) + (size_t)(pg + pp) * GC32, x, ps,
                                         pt);
                                const float wp = fmaf(qq[3], ps, qq[2] * ps), wt = fmaf(qq[3], pt, qq[2] * pt);
                                const float lx[3] = {qq[4], qq[5], 1.f - qq[4] - qq[5]};
                                const float ly[3] = {qq[6], qq[7], 1.f - qq[6] - qq[7]};
#pragma unroll
                                for (int a = 0; a < 3; ++a) {
                                    const float wa = wp * lx[a];
#pragma unroll
                                    for (int b = 0; b < 3; ++b) gn_two_sum_add(Sh[3 * a + b], Sl[3 * a + b], wa * ly[b]);
                                }
                                gn_two_sum_add(Th, Tl, wt);
                            }
#pragma unroll
                            for (int e = 0; e < 9; ++e) Sab[e] = (double)Sh[e] + (double)Sl[e];
                            St = (double)Th + (double)Tl;
                        }
                        for (int p = lane; !F32 && p < np; p += 32) {
                            const double *qq = q + 6 * p;
                            const double r = qq[0];
                            if (!(r > ba && r < bb)) continue;
                            double ps, pt;
                            g_cheb64(A, pg, npn, r, ps, pt);
                            const double lx[3] = {qq[2], qq[3], 1.0 - qq[2] - qq[3]};
                            const double ly[3] = {qq[4], qq[5], 1.0 - qq[4] - qq[5]};
                            const double wp = qq[1] * ps;
                            for (int a = 0; a < 3; ++a)
                                for (int b = 0; b < 3; ++b) Sab[3 * a + b] += wp * lx[a] * ly[b];
                            St += qq[1] * pt;
                        }
                        for (int e = 0; e < 9; ++e) Sab[e] = g_dsum(Sab[e]);
                        St = g_dsum(St);
                        if (lane < 9) acc[it * 10 + lane] += Sab[lane];
                        if (lane == 9) acc[it * 10 + 9] += St;
                    }
                }
                __syncthreads();
                // add the 3x3 results into the near windows
                for (int t = threadIdx.x; t < ni * 9; t += blockDim.x) {
                    const int it = t / 9, e = t % 9;
                    const int ci = A.i0 + (items[it] >> 16), kl = items[it] & 0xffff;
                    const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
                    const int k = k0 + kl;
                    const int a = e / 3, b = e % 3;
                    const int ca = pa[a], cbn = pb[b];
                    const double *ct = g.geo64 + 16 * tau + 4 + 3 * ca, *cs = g.geo64 + 16 * sg + 4 + 3 * cbn;
                    const double cc = ct[0] * cs[0] + ct[1] * cs[1] + ct[2] * cs[2];
                    const double L = nn * acc[it * 10 + e] + cc * acc[it * 10 + 9];
                    const int64_t l = g.F[3 * tau + ca], j = g.F[3 * sg + cbn];
                    const int nbi = A.adj_nbr[9 * pi + 3 * a + b];
                    if (nbi < 0) { A.status[0] = ST_NBR; continue; }
                    const int K1 = g_kfirst(A.gb + cb0, k0, nk, A.vmin[l * M + j] + A.tie);
                    const int KW = A.kw[ci];
                    const int slot = k - K1;
                    if (slot < 0 || slot >= KW) { A.status[0] = ST_WINDOW; continue; }
                    A.ndense[A.ndoff[ci - A.i0] + ((l * A.NB + nbi) * KW + slot)] += L;
                }
                __syncthreads();
            }
        }
    }
}

void launch_gnear(const GradedArgs &a, bool f32, int grid, cudaStream_t st) {
    if (grid <= 0) return;
    if (f32) gnear_kernel<true><<<grid, GN_WARPS * 32, 0, st>>>(a);
    else gnear_kernel<false><<<grid, GN_WARPS * 32, 0, st>>>(a);
}

// ----------------------------------------------------------- vertex bounds
// Dmin / Dmax of every vertex pair over the element pairs of the two stars;
// per-CTA maxima of Dmax - Dmin (the window length bound) in partial.
__global__ void gvertex_kernel(const GradedArgs A, double *vmin, double *vmax, double *partial) {
    __shared__ double red[256];
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, n = M * M;
    double spread = 0.0;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n; id += (int64_t)gridDim.x * blockDim.x) {
        const int64_t l = id / M, j = id % M;
        double mn = 1e300, mx = 0.0;
        for (int64_t x = g.vt_ptr[l]; x < g.vt_ptr[l + 1]; ++x) {
            const int64_t tau = g.vt_tri[x];
            for (int64_t y = g.vt_ptr[j]; y < g.vt_ptr[j + 1]; ++y) {
                const double2 b = A.pair[tau * E + g.vt_tri[y]];
                mn = fmin(mn, b.x);
                mx = fmax(mx, b.y);
            }
        }
        vmin[id] = mn;
        vmax[id] = mx;
        spread = fmax(spread, mx - mn);
    }
    red[threadIdx.x] = spread;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] = fmax(red[threadIdx.x], red[threadIdx.x + s]);
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

void launch_gvertex(const GradedArgs &a, double *vmin, double *vmax, double *partial, int nblocks, cudaStream_t st) {
    gvertex_kernel<<<nblocks, 256, 0, st>>>(a, vmin, vmax, partial);
}

// ------------------------------------------------------------- row counts
// One warp per (row l, column i): window [K1, K2] of every column j (far) and
// of the row's near neighbours (near), histogrammed per block in shared
// memory; written per block in the caller's (k-major) numbering.
constexpr int GC_WARPS = 8;

__global__ void gcount_kernel(const GradedArgs A, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                              int64_t *cnt_far, int64_t *cnt_near) {
    __shared__ int hist[GC_WARPS][2][GP_MAXK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t M = A.g.M;
    const int64_t item = blockIdx.x * (int64_t)GC_WARPS + w;
    if (item >= M * A.N) return;
    const int ci = (int)(item / M);
    const int64_t l = item % M;
    const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
    if (nk <= 0) return;
    for (int x = lane; x < nk; x += 32) { hist[w][0][x] = 0; hist[w][1][x] = 0; }
    __syncwarp();
    const double *ca = A.ga + cb0, *cbv = A.gb + cb0;
    for (int side = 0; side < 2; ++side) {
        const int64_t j0 = side ? nbr_ptr[l] : 0, j1 = side ? nbr_ptr[l + 1] : M;
        for (int64_t x = j0 + lane; x < j1; x += 32) {
            const int64_t j = side ? nbr[x] : x;
            const int K1 = g_kfirst(cbv, k0, nk, A.vmin[l * M + j] + A.tie);
            const int K2 = g_klast(ca, k0, nk, A.vmax[l * M + j] - A.tie);
            for (int k = K1; k <= K2; ++k) atomicAdd(&hist[w][side][k - k0], 1);
        }
    }
    __syncwarp();
    for (int x = lane; x < nk; x += 32) {
        const int64_t b = cb2api[cb0 + x];
        cnt_far[b * M + l] = hist[w][0][x];
        cnt_near[b * M + l] = hist[w][1][x];
    }
}

void launch_gcount(const GradedArgs &a, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                   int64_t *cnt_far, int64_t *cnt_near, cudaStream_t st) {
    const int64_t items = a.g.M * a.N;
    gcount_kernel<<<(unsigned)((items + GC_WARPS - 1) / GC_WARPS), GC_WARPS * 32, 0, st>>>(a, cb2api, nbr_ptr, nbr,
                                                                                      cnt_far, cnt_near);
}

// ------------------------------------------------- quadrature point pairs
__global__ void gcount_quad_kernel(const GradedArgs A, int npp0, int npp1, int npp2, int npp3, int64_t *partial) {
    __shared__ int64_t red[256], redf[256];
    const Geo &g = A.g;
    const int64_t E = g.E, n = E * E;
    int64_t acc = 0, accf = 0;
    for (int64_t id = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; id < n; id += (int64_t)gridDim.x * blockDim.x) {
        const int64_t q = id / E, s = id % E;
        int shared = 0;
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) shared += g.F[3 * q + a] == g.F[3 * s + b];
        const double2 bd = A.pair[id];
        int64_t kept = 0;
        for (int ci = 0; ci < A.N; ++ci) {
            const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
            if (nk <= 0) continue;
            const int K1 = g_kfirst(A.gb + cb0, k0, nk, bd.x + A.tie);
            const int K2 = g_klast(A.ga + cb0, k0, nk, bd.y - A.tie);
            if (K2 >= K1) kept += K2 - K1 + 1;
        }
        const int npp = shared == 0 ? npp0 : (shared == 1 ? npp1 : (shared == 2 ? npp2 : npp3));
        acc += kept * npp;
        if (shared == 0) accf += kept * npp;
    }
    red[threadIdx.x] = acc;
    redf[threadIdx.x] = accf;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) { red[threadIdx.x] += red[threadIdx.x + s]; redf[threadIdx.x] += redf[threadIdx.x + s]; }
        __syncthreads();
    }
    if (threadIdx.x == 0) { partial[blockIdx.x] = red[0]; partial[gridDim.x + blockIdx.x] = redf[0]; }
}

void launch_gcount_quad(const GradedArgs &a, int npp_far, const int *npp_near, int64_t *partial, int nblocks,
                        cudaStream_t st) {
    gcount_quad_kernel<<<nblocks, 256, 0, st>>>(a, npp_far, npp_near[1], npp_near[2], npp_near[3], partial);
}

// ----------------------------------------------------------------- CSR fill
// One warp per (row l, batch column); columns j in increasing order in chunks
// of 32, a ballot per block present in the chunk (rows come out sorted).
template <typename T>
__global__ void gfill_kernel(const GradedArgs A, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                             const int64_t *rp_far, const int64_t *off_far, int32_t *col_far, T *val_far,
                             const int64_t *rp_near, const int64_t *off_near, int32_t *col_near,
                             double *val_near) {
    __shared__ int cur[GC_WARPS][GP_MAXK];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t M = A.g.M;
    const int nb = A.i1 - A.i0;
    const int64_t item = blockIdx.x * (int64_t)GC_WARPS + w;
    if (item >= M * nb) return;
    const int ci = A.i0 + (int)(item / M);
    const int64_t l = item % M;
    const int cb0 = A.colblk[ci], nk = A.colblk[ci + 1] - cb0, k0 = A.colk0[ci];
    if (nk <= 0) return;
    const double *ca = A.ga + cb0, *cbv = A.gb + cb0;
    const int KW = A.kw[ci];
    const unsigned ltm = (1u << lane) - 1u;
    for (int side = 0; side < 2; ++side) {
        for (int x = lane; x < nk; x += 32) cur[w][x] = 0;
        __syncwarp();
        const int64_t j0 = side ? nbr_ptr[l] : 0, j1 = side ? nbr_ptr[l + 1] : M;
        for (int64_t xb = j0; xb < j1; xb += 32) {
            const int64_t x = xb + lane;
            const bool ok = x < j1;
            const int64_t j = ok ? (side ? nbr[x] : x) : 0;
            int K1 = 1 << 30, K2 = -(1 << 30);
            if (ok) {
                K1 = g_kfirst(cbv, k0, nk, A.vmin[l * M + j] + A.tie);
                K2 = g_klast(ca, k0, nk, A.vmax[l * M + j] - A.tie);
            }
            int lo = K1, hi = K2;
            for (int o = 16; o > 0; o >>= 1) {
                lo = min(lo, __shfl_xor_sync(0xffffffffu, lo, o));
                hi = max(hi, __shfl_xor_sync(0xffffffffu, hi, o));
            }
            for (int k = lo; k <= hi; ++k) {
                const bool in = K1 <= k && k <= K2;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (!bal) continue;
                const int kl = k - k0;
                if (in && k - K1 >= KW) {
                    A.status[0] = ST_WINDOW;
                } else if (in) {
                    const int64_t b = cb2api[cb0 + kl];
                    if (side == 0) {
                        const int64_t pos = off_far[b] + rp_far[b * (M + 1) + l] + cur[w][kl] + __popc(bal & ltm);
                        col_far[pos] = (int32_t)j;
                        val_far[pos] = (T)A.dense[A.doff[ci - A.i0] + (l * M + j) * KW + (k - K1)];
                    } else {
                        const int64_t pos = off_near[b] + rp_near[b * (M + 1) + l] + cur[w][kl] + __popc(bal & ltm);
                        col_near[pos] = (int32_t)j;
                        val_near[pos] = A.ndense[A.ndoff[ci - A.i0] + ((l * A.NB + (x - j0)) * KW + (k - K1))];
                    }
                }
                __syncwarp();
                if (lane == 0) cur[w][kl] += __popc(bal);
                __syncwarp();
            }
        }
        __syncwarp();
    }
}

void launch_gfill(const GradedArgs &a, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                  const int64_t *rp_far, const int64_t *off_far, int32_t *col_far, void *val_far, bool fp64,
                  const int64_t *rp_near, const int64_t *off_near, int32_t *col_near, double *val_near,
                  cudaStream_t st) {
    const int64_t items = a.g.M * (a.i1 - a.i0);
    if (items <= 0) return;
    const unsigned grid = (unsigned)((items + GC_WARPS - 1) / GC_WARPS);
    if (fp64)
        gfill_kernel<double><<<grid, GC_WARPS * 32, 0, st>>>(a, cb2api, nbr_ptr, nbr, rp_far, off_far, col_far,
                                                             (double *)val_far, rp_near, off_near, col_near, val_near);
    else
        gfill_kernel<float><<<grid, GC_WARPS * 32, 0, st>>>(a, cb2api, nbr_ptr, nbr, rp_far, off_far, col_far,
                                                            (float *)val_far, rp_near, off_near, col_near, val_near);
}

// FP32 coefficient layout of the far kernel: per panel GC32 float4 = 17 x
// (psi_n, psi~_n, psi_{n+1}, psi~_{n+1}), n = 0, 2, .., 32 (entry 33 zero),
// then (lo_0, lo~_0, lo_1, lo~_1), (lo_2, lo~_2, lo_3, lo~_3) with
// lo_n = c_n - (double)(float)c_n.
__global__ void gcoef32_kernel(const double *coef, int npan, float *out) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= npan * 38) return;
    const int p = id / 38, n = id % 38;
    float a = 0.f, b = 0.f;
    if (n < NCHEB) {
        a = (float)coef[((size_t)p * NCHEB + n) * 2];
        b = (float)coef[((size_t)p * NCHEB + n) * 2 + 1];
    } else if (n >= 34) {
        const double ca = coef[((size_t)p * NCHEB + (n - 34)) * 2], cb = coef[((size_t)p * NCHEB + (n - 34)) * 2 + 1];
        a = (float)(ca - (double)(float)ca);
        b = (float)(cb - (double)(float)cb);
    }
    out[(size_t)p * 4 * GC32 + 2 * n] = a;
    out[(size_t)p * 4 * GC32 + 2 * n + 1] = b;
}

void launch_gcoef32(const double *coef, int npan, float *out, cudaStream_t st) {
    if (npan <= 0) return;
    gcoef32_kernel<<<(npan * 38 + 255) / 256, 256, 0, st>>>(coef, npan, out);
}

}  // namespace tdbem
