// Near-field quadrature of the mixed path (element pairs sharing a vertex,
// an edge or the whole triangle; Eq. MatrixEntries with the Sauter-Schwab
// regularising maps of [0,1]^4, Sauter & Schwab, Boundary Element Methods,
// Sec. 5.2): the structure of near_kernel (one CTA per test triangle of the
// current colour, its adjacent trial triangles in turn, point pairs sorted
// by lag cell, one warp per (block, pair) over the point pairs in that
// block's support), with psi and psi~ evaluated in FP32.
//
// Per point pair, in FP64: the distance r and the retarded argument
// q = r / dt, kept as its cell floor(q) and the Chebyshev argument
// x = 2 frac(q) - 1 rounded to FP32. With one panel per unit of q every lag
// class has its breakpoints at integer q (Sec. 3.1, Eq. psiTildeRed), so
// every block sees the same x at a point pair and only the panel, cell - lag,
// depends on the block. Per (point pair, block), in FP32: the T_n recurrence
// and the degree-32 sums of (psi, psi~) from the one-panel-per-unit FP32
// tables in shared memory, whose four leading coefficients carry their FP32
// residuals (a rounding shared by every point pair would not average out);
// the weight w / r as an FP32 pair; the nine sums S_ab and S~ accumulated as
// FP32 pairs with an error-free two-sum (the n.n and curl.curl parts of a
// block cancel to a small fraction of either part, so their summation error
// is amplified), added across the warp in FP64; the combination and the
// read-modify-write of the FP64 near windows as in near_kernel.
#include <math.h>

#include "tdbem_internal.h"

namespace tdbem {

constexpr int N32_WARPS = 8;
constexpr int N32_THREADS = N32_WARPS * 32;
constexpr int N32_CELLS = 16;  // lag cells floor(q) a near point pair can occupy
// point chunks of N32_THREADS in the sort: 4096 point pairs, above the largest
// rule (near_order <= 5: 6 x 5^4 = 3750 for identical triangles)
constexpr int N32_MAXCHK = 16;

// one point pair: Chebyshev argument, weight w / r as an FP32 pair, the two
// free barycentrics of each side, and the cell floor(q)
struct alignas(16) NearPt32 {
    float x, wh, wl, lx0, lx1, ly0, ly1;
    int cell;
};

__device__ __forceinline__ void n32_two_sum(float &h, float &l, float v) {
    const float s = h + v;
    const float bb = s - h;
    l += (h - (s - bb)) + (v - bb);
    h = s;
}

__device__ static inline double n32_dsum_warp(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

__global__ void __launch_bounds__(N32_THREADS, 3) near32_kernel(const NearArgs A, const ChebF32 C, int npp_max) {
    extern __shared__ __align__(16) unsigned char n32_raw[];
    NearPt32 *pts = reinterpret_cast<NearPt32 *>(n32_raw);
    int16_t *order = reinterpret_cast<int16_t *>(pts + npp_max);
    __shared__ float2 cs[TOTAL_PANELS][NCHEB];     // (psi, psi~) per term
    __shared__ float2 clo[TOTAL_PANELS][NCHEB_LO]; // residuals of the leading terms
    __shared__ int items[64];
    __shared__ int nitems;
    __shared__ int bstart[N32_CELLS + 1];
    __shared__ int scnt[N32_CELLS * N32_MAXCHK * N32_WARPS];  // per (cell, chunk, warp): count, then offset
    __shared__ int ctot[N32_CELLS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, MM = M * M;
    const double inv_dt = A.lt.inv_dt;
    for (int i = threadIdx.x; i < TOTAL_PANELS * NCHEB; i += N32_THREADS) {
        const int p = i / NCHEB, n = i % NCHEB;
        cs[p][n] = make_float2(C.c[p][n][0], C.c[p][n][1]);
    }
    for (int i = threadIdx.x; i < TOTAL_PANELS * NCHEB_LO; i += N32_THREADS) {
        const int p = i / NCHEB_LO, n = i % NCHEB_LO;
        clo[p][n] = make_float2(C.lo[p][n][0], C.lo[p][n][1]);
    }
    __syncthreads();

    for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
        const int64_t tau = A.color_tris[ti];
        for (int64_t pi = A.adj_ptr[tau]; pi < A.adj_ptr[tau + 1]; ++pi) {
            const int64_t sg = A.adj_tri[pi];
            const int8_t *pm = A.adj_perm + 8 * pi;
            const int kase = pm[0];
            const int pa[3] = {pm[1], pm[2], pm[3]}, pb[3] = {pm[4], pm[5], pm[6]};
            const int npp = A.ss_npp[kase];
            const double *rule = A.ss_xy[kase];
            double X[3][3], Y[3][3];
            for (int k = 0; k < 3; ++k)
                for (int d = 0; d < 3; ++d) {
                    X[k][d] = g.V[3 * g.F[3 * tau + pa[k]] + d];
                    Y[k][d] = g.V[3 * g.F[3 * sg + pb[k]] + d];
                }
            const double at = g.geo64[16 * tau + 3], as = g.geo64[16 * sg + 3];
            // reference triangle of area 1/2 on both sides: |J| = 2|T|
            const double scale = 4.0 * at * as * 0.07957747154594767;
            for (int p = threadIdx.x; p < npp; p += N32_THREADS) {
                const double xh0 = rule[5 * p], xh1 = rule[5 * p + 1];
                const double yh0 = rule[5 * p + 2], yh1 = rule[5 * p + 3];
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double xd = X[0][d] + xh0 * (X[1][d] - X[0][d]) + xh1 * (X[2][d] - X[1][d]);
                    const double yd = Y[0][d] + yh0 * (Y[1][d] - Y[0][d]) + yh1 * (Y[2][d] - Y[1][d]);
                    r2 += (xd - yd) * (xd - yd);
                }
                // 1 / r once (CUDA's FP64 rsqrt, within 1 ulp): r and the weight w / r
                const double ir = rsqrt(r2);
                const double q = (r2 * ir) * inv_dt;
                const double cf = floor(q);
                const double wgt = rule[5 * p + 4] * scale * ir;
                NearPt32 t;
                t.x = (float)(2.0 * (q - cf) - 1.0);
                t.wh = (float)wgt;
                t.wl = (float)(wgt - (double)t.wh);
                t.lx0 = (float)(1.0 - xh0);
                t.lx1 = (float)(xh0 - xh1);
                t.ly0 = (float)(1.0 - yh0);
                t.ly1 = (float)(yh0 - yh1);
                t.cell = (int)min(cf, 1e6);
                pts[p] = t;
            }
            __syncthreads();
            // stable counting sort of the point pairs by lag cell: a block's
            // support is then one contiguous run of the order (no idle lanes).
            // Counts per (point chunk k, warp, cell) by ballots, offsets in
            // the order (cell, k, warp, lane) = (cell, point index), scatter.
            {
                const int nchk = (npp + N32_THREADS - 1) / N32_THREADS;
                for (int k = 0; k < nchk; ++k) {
                    const int p = k * N32_THREADS + threadIdx.x;
                    const int cl = p < npp ? min(pts[p].cell, N32_CELLS - 1) : N32_CELLS;
                    for (int cb = 0; cb < N32_CELLS; ++cb) {
                        const unsigned bal = __ballot_sync(0xffffffffu, cl == cb);
                        if (lane == 0) scnt[(cb * N32_MAXCHK + k) * N32_WARPS + w] = __popc(bal);
                    }
                }
                __syncthreads();
                if (threadIdx.x < N32_CELLS) {
                    int tot = 0;
                    for (int i = 0; i < nchk * N32_WARPS; ++i) tot += scnt[threadIdx.x * N32_MAXCHK * N32_WARPS + i];
                    ctot[threadIdx.x] = tot;
                }
                __syncthreads();
                if (threadIdx.x < N32_CELLS) {
                    int base = 0;
                    for (int cb = 0; cb < (int)threadIdx.x; ++cb) base += ctot[cb];
                    bstart[threadIdx.x] = base;
                    if (threadIdx.x == N32_CELLS - 1) bstart[N32_CELLS] = base + ctot[threadIdx.x];
                    int *c = scnt + threadIdx.x * N32_MAXCHK * N32_WARPS;
                    for (int i = 0; i < nchk * N32_WARPS; ++i) {  // counts -> offsets in place
                        const int v = c[i];
                        c[i] = base;
                        base += v;
                    }
                }
                __syncthreads();
                for (int k = 0; k < nchk; ++k) {
                    const int p = k * N32_THREADS + threadIdx.x;
                    const int cl = p < npp ? min(pts[p].cell, N32_CELLS - 1) : N32_CELLS;
                    for (int cb = 0; cb < N32_CELLS; ++cb) {
                        const unsigned bal = __ballot_sync(0xffffffffu, cl == cb);
                        if (cl == cb)
                            order[scnt[(cb * N32_MAXCHK + k) * N32_WARPS + w] + __popc(bal & ((1u << lane) - 1u))] =
                                (int16_t)p;
                    }
                }
            }
            if (threadIdx.x == 0) {
                const PairRec rc = A.rec[tau * E + sg];
                int n = 0;
                for (int c = 0; c < NLAG; ++c)
                    for (int k = 0; k < rc.cnt[c] && n < 64; ++k) items[n++] = (c << 16) | ((rc.lo[c] + k) & 0xffff);
                for (int s = 0; s < NSPEC; ++s)
                    if (((rc.smask >> s) & 1u) && n < 64) items[n++] = ((NLAG + s) << 16);
                if (rc.cnt[0] + rc.cnt[1] + rc.cnt[2] + __popc(rc.smask) > 64) A.status[0] = ST_WINDOW;
                nitems = n;
            }
            __syncthreads();
            const double nn = g.geo64[16 * tau] * g.geo64[16 * sg] + g.geo64[16 * tau + 1] * g.geo64[16 * sg + 1] +
                              g.geo64[16 * tau + 2] * g.geo64[16 * sg + 2];
            for (int it = w; it < nitems; it += N32_WARPS) {
                const int c = items[it] >> 16;
                const int d = (int16_t)(items[it] & 0xffff);
                const int P = A.lt.P[c], rho = A.lt.rho[c];
                int p0 = 0;
                for (int x = 0; x < c; ++x) p0 += A.lt.P[x];
                float Sh[3][3], Sl[3][3], Th = 0.f, Tl = 0.f;
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) Sh[a][b] = Sl[a][b] = 0.f;
                // cells d + rho .. d + rho + P - 1 hold this block's support
                const int c0 = max(d + rho, 0), c1 = min(d + rho + P, N32_CELLS);
                const int k0 = c0 < c1 ? bstart[c0] : 0, k1 = c0 < c1 ? bstart[c1] : 0;
                for (int kk = k0 + lane; kk < k1; kk += 32) {
                    const NearPt32 t = pts[order[kk]];
                    const int j = t.cell - d - rho;
                    if (j < 0 || j >= P) continue;
                    const float2 *cf = cs[p0 + j];
                    const float2 *lo = clo[p0 + j];
                    const float x = t.x, x2 = x + x;
                    float ps = fmaf(cf[1].x, x, cf[0].x), pt = fmaf(cf[1].y, x, cf[0].y);
                    float tm = 1.f, tc = x, t2 = 0.f, t3 = 0.f;
#pragma unroll
                    for (int n = 2; n < NCHEB; ++n) {
                        const float tn = fmaf(x2, tc, -tm);
                        tm = tc;
                        tc = tn;
                        if (n == 2) t2 = tn;
                        if (n == 3) t3 = tn;
                        ps = fmaf(cf[n].x, tn, ps);
                        pt = fmaf(cf[n].y, tn, pt);
                    }
                    ps += fmaf(lo[3].x, t3, fmaf(lo[2].x, t2, fmaf(lo[1].x, x, lo[0].x)));
                    pt += fmaf(lo[3].y, t3, fmaf(lo[2].y, t2, fmaf(lo[1].y, x, lo[0].y)));
                    const float wp = fmaf(t.wl, ps, t.wh * ps);
                    const float wt = fmaf(t.wl, pt, t.wh * pt);
                    const float lx[3] = {t.lx0, t.lx1, 1.f - t.lx0 - t.lx1};
                    const float ly[3] = {t.ly0, t.ly1, 1.f - t.ly0 - t.ly1};
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const float wa = wp * lx[a];
#pragma unroll
                        for (int b = 0; b < 3; ++b) n32_two_sum(Sh[a][b], Sl[a][b], wa * ly[b]);
                    }
                    n32_two_sum(Th, Tl, wt);
                }
                double Sab[3][3];
#pragma unroll
                for (int a = 0; a < 3; ++a)
#pragma unroll
                    for (int b = 0; b < 3; ++b) Sab[a][b] = n32_dsum_warp((double)Sh[a][b] + (double)Sl[a][b]);
                const double St = n32_dsum_warp((double)Th + (double)Tl);
                if (lane < 9) {
                    const int a = lane / 3, b = lane % 3;
                    const int ca = pa[a], cb = pb[b];
                    const double *ct = g.geo64 + 16 * tau + 4 + 3 * ca, *cs2 = g.geo64 + 16 * sg + 4 + 3 * cb;
                    const double cc = ct[0] * cs2[0] + ct[1] * cs2[1] + ct[2] * cs2[2];
                    const double L = nn * Sab[a][b] + cc * St;
                    const int64_t l = g.F[3 * tau + ca], jj = g.F[3 * sg + cb];
                    const int k = A.adj_nbr[9 * pi + 3 * a + b];
                    if (k < 0) { A.status[0] = ST_NBR; continue; }
                    if (c < NLAG) {
                        const int wlo = A.dlo[c * MM + l * M + jj], whi = A.dhi[c * MM + l * M + jj];
                        if (d < wlo || d > whi || d - wlo >= A.KW) { A.status[0] = ST_WINDOW; continue; }
                        A.ndense[((c * M + l) * A.NB + k) * A.KW + (d - wlo)] += L;
                    } else {
                        A.ndense_spec[((c - NLAG) * M + l) * A.NB + k] += L;
                    }
                }
            }
            __syncthreads();
        }
    }
}

// Far element pairs (no shared vertex) that reach a special block, with the
// 7-point rule on both triangles, in the precision scheme of this file:
// per point pair the distance r, q = r / dt and the factor
// |tau||sigma| / (4 pi r) in FP64, once for every special block; per
// (point pair, special block) psi and psi~ from the FP32 tables with the
// residuals of the leading coefficients; the rule products
// w_x w_y lambda_a(x) lambda_b(y) and w_x w_y are FP32 pairs (their
// rounding would otherwise be one bias shared by every element pair), the
// nine S_ab and S~ are accumulated as FP32 pairs and added across the warp in
// FP64. One CTA per test triangle of the current colour. Its four warps scan
// the pair records of one quarter of the trial triangles each, in trial
// order, into their own lists (no CTA barrier while scanning; a round ends
// when a list could overflow, or at the end of the row). The concatenated
// lists are then taken four entries at a time, one per warp (lanes over the
// 49 point pairs), and warp 0 adds their values into the far special-block
// windows in list order: the order depends on the data only, so the sums
// repeat exactly.
constexpr int FS32_WARPS = 4;
constexpr int FS32_THREADS = FS32_WARPS * 32;
constexpr int FS32_LIST = 128;
__global__ void __launch_bounds__(FS32_THREADS) farspec32_kernel(const NearArgs A, const ChebF32 C) {
    __shared__ float2 cs[TOTAL_PANELS][NCHEB];
    __shared__ float2 clo[TOTAL_PANELS][NCHEB_LO];
    __shared__ float2 gw[49][10];  // (hi, lo) of w_x w_y lambda_a lambda_b, (a, b) row-major, then w_x w_y
    __shared__ int list[FS32_WARPS][FS32_LIST];
    __shared__ int wcount[FS32_WARPS];
    __shared__ double fs_val[FS32_WARPS][NSPEC][9];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, MM = M * M;
    const double inv_dt = A.lt.inv_dt;
    for (int i = threadIdx.x; i < TOTAL_PANELS * NCHEB; i += FS32_THREADS) {
        const int p = i / NCHEB, n = i % NCHEB;
        cs[p][n] = make_float2(C.c[p][n][0], C.c[p][n][1]);
    }
    for (int i = threadIdx.x; i < TOTAL_PANELS * NCHEB_LO; i += FS32_THREADS) {
        const int p = i / NCHEB_LO, n = i % NCHEB_LO;
        clo[p][n] = make_float2(C.lo[p][n][0], C.lo[p][n][1]);
    }
    for (int i = threadIdx.x; i < 49 * 10; i += FS32_THREADS) {
        const int pp = i / 10, k = i % 10, ix = pp / 7, iy = pp % 7;
        double v = A.rule_w64[ix] * A.rule_w64[iy];
        if (k < 9) v *= A.rule_l64[3 * ix + k / 3] * A.rule_l64[3 * iy + k % 3];
        const float hi = (float)v;
        gw[pp][k] = make_float2(hi, (float)(v - (double)hi));
    }
    __syncthreads();
    const unsigned lt_mask = (1u << lane) - 1u;
    const int64_t qlen = (E + FS32_WARPS - 1) / FS32_WARPS;
    const int64_t lo_w = min(E, w * qlen), hi_w = min(E, lo_w + qlen);
    for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
        const int64_t tau = A.color_tris[ti];
        int64_t pos = lo_w;
        while (__syncthreads_or(pos < hi_w)) {
            int n = 0;
            while (pos < hi_w && n + 32 <= FS32_LIST) {
                const int64_t sg = pos + lane;
                bool need = false;
                if (sg < hi_w) {
                    const PairRec rc = A.rec[tau * E + sg];
                    need = rc.adj == 0 && rc.smask != 0;
                }
                const unsigned bal = __ballot_sync(0xffffffffu, need);
                if (need) list[w][n + __popc(bal & lt_mask)] = (int)sg;
                n += __popc(bal);
                pos += 32;
            }
            if (lane == 0) wcount[w] = n;
            __syncthreads();
            int nlist = 0;
            for (int k = 0; k < FS32_WARPS; ++k) nlist += wcount[k];
            auto entry = [&](int q) {
                int k = 0;
                while (q >= wcount[k]) q -= wcount[k++];
                return list[k][q];
            };
            for (int q0 = 0; q0 < nlist; q0 += FS32_WARPS) {
                const int q = q0 + w;
                if (q < nlist) {
                    const int64_t s2 = entry(q);
                    const PairRec r2 = A.rec[tau * E + s2];
                    double nn = 0.0;
                    for (int d = 0; d < 3; ++d) nn += g.geo64[16 * tau + d] * g.geo64[16 * s2 + d];
                    const double scale = g.geo64[16 * tau + 3] * g.geo64[16 * s2 + 3] * 0.07957747154594767;
                    // the lane's point pairs pp = lane, lane + 32: q and |tau||sigma| / (4 pi r)
                    double qv[2] = {-1.0, -1.0};
                    float sw[2] = {0.f, 0.f};
#pragma unroll
                    for (int h = 0; h < 2; ++h) {
                        const int pp = lane + 32 * h;
                        if (pp >= 49) continue;
                        const int ix = pp / 7, iy = pp % 7;
                        double r2s = 0.0;
                        for (int d = 0; d < 3; ++d) {
                            const double xd = g.cen[3 * tau + d] + g.dq[(tau * 7 + ix) * 3 + d];
                            const double yd = g.cen[3 * s2 + d] + g.dq[(s2 * 7 + iy) * 3 + d];
                            r2s += (xd - yd) * (xd - yd);
                        }
                        const double ir = rsqrt(r2s);  // 1 / r within 1 ulp: r and the weight factor
                        qv[h] = (r2s * ir) * inv_dt;
                        sw[h] = (float)(scale * ir);
                    }
                    for (int sb = 0; sb < NSPEC; ++sb) {
                        if (!((r2.smask >> sb) & 1u)) continue;
                        const int c = NLAG + sb;
                        const int P = A.lt.P[c], rho = A.lt.rho[c];
                        int p0 = 0;
                        for (int x = 0; x < c; ++x) p0 += A.lt.P[x];
                        float Sh[9], Sl[9], Th = 0.f, Tl = 0.f;
#pragma unroll
                        for (int k = 0; k < 9; ++k) Sh[k] = Sl[k] = 0.f;
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int pp = lane + 32 * h;
                            if (pp >= 49) continue;
                            const double v = qv[h] - (double)rho;
                            if (!(v >= 0.0 && v < (double)P)) continue;
                            const double jf = floor(v);
                            const int j = (int)jf;
                            const float x = (float)(2.0 * (v - jf) - 1.0), x2 = x + x;
                            const float2 *cf = cs[p0 + j];
                            const float2 *lo = clo[p0 + j];
                            float ps = fmaf(cf[1].x, x, cf[0].x), pt = fmaf(cf[1].y, x, cf[0].y);
                            float tm = 1.f, tc = x, t2 = 0.f, t3 = 0.f;
#pragma unroll
                            for (int nn2 = 2; nn2 < NCHEB; ++nn2) {
                                const float tn = fmaf(x2, tc, -tm);
                                tm = tc;
                                tc = tn;
                                if (nn2 == 2) t2 = tn;
                                if (nn2 == 3) t3 = tn;
                                ps = fmaf(cf[nn2].x, tn, ps);
                                pt = fmaf(cf[nn2].y, tn, pt);
                            }
                            ps += fmaf(lo[3].x, t3, fmaf(lo[2].x, t2, fmaf(lo[1].x, x, lo[0].x)));
                            pt += fmaf(lo[3].y, t3, fmaf(lo[2].y, t2, fmaf(lo[1].y, x, lo[0].y)));
                            const float s = sw[h];
#pragma unroll
                            for (int k = 0; k < 9; ++k) {
                                const float2 gk = gw[pp][k];
                                n32_two_sum(Sh[k], Sl[k], ps * fmaf(s, gk.y, s * gk.x));
                            }
                            const float2 gt = gw[pp][9];
                            n32_two_sum(Th, Tl, pt * fmaf(s, gt.y, s * gt.x));
                        }
                        double Sab[9];
#pragma unroll
                        for (int k = 0; k < 9; ++k) Sab[k] = n32_dsum_warp((double)Sh[k] + (double)Sl[k]);
                        const double St = n32_dsum_warp((double)Th + (double)Tl);
                        if (lane < 9) {
                            const int a = lane / 3, b = lane % 3;
                            const double *ct = g.geo64 + 16 * tau + 4 + 3 * a, *cs2 = g.geo64 + 16 * s2 + 4 + 3 * b;
                            const double cc = ct[0] * cs2[0] + ct[1] * cs2[1] + ct[2] * cs2[2];
                            double Sl9 = Sab[0];
#pragma unroll
                            for (int k = 1; k < 9; ++k) Sl9 = lane == k ? Sab[k] : Sl9;
                            fs_val[w][sb][lane] = nn * Sl9 + cc * St;
                        }
                    }
                }
                __syncthreads();
                if (w == 0 && lane < 9)
                    for (int k = 0; k < FS32_WARPS && q0 + k < nlist; ++k) {
                        const int64_t s2 = entry(q0 + k);
                        const PairRec r2 = A.rec[tau * E + s2];
                        const int a = lane / 3, b = lane % 3;
                        const int64_t l = g.F[3 * tau + a], j = g.F[3 * s2 + b];
                        for (int sb = 0; sb < NSPEC; ++sb)
                            if (((r2.smask >> sb) & 1u) && ((A.smask[l * M + j] >> sb) & 1u))
                                A.far_spec[sb * MM + l * M + j] += fs_val[k][sb][lane];
                    }
                __syncthreads();
            }
        }
    }
}

void launch_farspec32(const NearArgs &a, const ChebF32 &c32, int grid, cudaStream_t st) {
    farspec32_kernel<<<grid, FS32_THREADS, 0, st>>>(a, c32);
}

void launch_near32(const NearArgs &a, const ChebF32 &c32, int grid, cudaStream_t st) {
    int mx = 0;
    for (int k = 1; k <= 3; ++k) mx = a.ss_npp[k] > mx ? a.ss_npp[k] : mx;

    const size_t smem = (size_t)mx * sizeof(NearPt32) + ((size_t)mx * sizeof(int16_t) + 15) / 16 * 16;
    cudaFuncSetAttribute(near32_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    near32_kernel<<<grid, N32_THREADS, smem, st>>>(a, c32, mx);
}

}  // namespace tdbem
