// Near-field quadrature (element pairs sharing a vertex, an edge or the
// whole triangle) of Eq. MatrixEntries in FP64 with Sauter-Schwab
// regularising maps of [0,1]^4 (Sauter & Schwab, Boundary Element Methods,
// Sec. 5.2) and Gauss-Legendre points per direction; psi, psi~ come from the
// FP64 Chebyshev tables. One CTA per test triangle of the current colour;
// its adjacent trial triangles are processed one after another, each
// (block, pair) by one warp with a shuffle reduction, and the 3x3 result is
// added into the near lag windows of the test triangle's rows.
#include <math.h>

#include "tdbem_internal.h"

namespace tdbem {

constexpr int NEAR_WARPS = 8;
constexpr int NEAR_THREADS = NEAR_WARPS * 32;

__device__ static inline double dsum_warp(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

constexpr int NEAR_CELLS = 16;  // lag cells floor(r/dt) a near point pair can occupy

__global__ void __launch_bounds__(NEAR_THREADS)
near_kernel(const NearArgs A) {
    extern __shared__ __align__(16) double sm[];  // npp x 6: r, w/r, lx0, lx1, ly0, ly1; then npp x int16 order
    __shared__ int items[64];
    __shared__ int nitems;
    __shared__ int bstart[NEAR_CELLS + 1];
    __shared__ int wcnt[NEAR_WARPS];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, MM = M * M;
    const double inv_dt = A.lt.inv_dt;
    const int S = A.S;

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
            for (int p = threadIdx.x; p < npp; p += NEAR_THREADS) {
                const double xh0 = rule[5 * p], xh1 = rule[5 * p + 1];
                const double yh0 = rule[5 * p + 2], yh1 = rule[5 * p + 3];
                double r2 = 0.0;
                for (int d = 0; d < 3; ++d) {
                    const double xd = X[0][d] + xh0 * (X[1][d] - X[0][d]) + xh1 * (X[2][d] - X[1][d]);
                    const double yd = Y[0][d] + yh0 * (Y[1][d] - Y[0][d]) + yh1 * (Y[2][d] - Y[1][d]);
                    r2 += (xd - yd) * (xd - yd);
                }
                const double r = sqrt(r2);
                double *q = sm + 6 * p;
                q[0] = r;
                q[1] = rule[5 * p + 4] * scale / r;
                q[2] = 1.0 - xh0; q[3] = xh0 - xh1;
                q[4] = 1.0 - yh0; q[5] = yh0 - yh1;
            }
            __syncthreads();
            // stable counting sort of the point pairs by lag cell: a block's
            // support is then one contiguous run of the order (no idle lanes)
            int16_t *order = reinterpret_cast<int16_t *>(sm + 6 * npp);
            {
                int base = 0;
                for (int cb = 0; cb < NEAR_CELLS; ++cb) {
                    if (threadIdx.x == 0) bstart[cb] = base;
                    for (int p0 = 0; p0 < npp; p0 += NEAR_THREADS) {
                        const int p = p0 + threadIdx.x;
                        int cl = NEAR_CELLS;
                        if (p < npp) cl = min((int)floor(sm[6 * p] * inv_dt), NEAR_CELLS - 1);
                        const bool in = cl == cb;
                        const unsigned bal = __ballot_sync(0xffffffffu, in);
                        if (lane == 0) wcnt[w] = __popc(bal);
                        __syncthreads();
                        int off = base;
                        for (int k = 0; k < w; ++k) off += wcnt[k];
                        if (in) order[off + __popc(bal & ((1u << lane) - 1u))] = (int16_t)p;
                        int tot = 0;
                        for (int k = 0; k < NEAR_WARPS; ++k) tot += wcnt[k];
                        __syncthreads();
                        base += tot;
                    }
                }
                if (threadIdx.x == 0) bstart[NEAR_CELLS] = base;
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
            for (int it = w; it < nitems; it += NEAR_WARPS) {
                const int c = items[it] >> 16;
                const int d = (int16_t)(items[it] & 0xffff);
                const int P = A.lt.P[c], rho = A.lt.rho[c];
                int p0 = 0;
                for (int x = 0; x < c; ++x) p0 += A.lt.P[x];
                double Sab[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, St = 0.0;
                // cells d + rho .. d + rho + P - 1 hold this block's support
                const int c0 = max(d + rho, 0), c1 = min(d + rho + P, NEAR_CELLS);
                const int k0 = c0 < c1 ? bstart[c0] : 0, k1 = c0 < c1 ? bstart[c1] : 0;
                for (int kk = k0 + lane; kk < k1; kk += 32) {
                    const int p = order[kk];
                    const double *q = sm + 6 * p;
                    const double v = q[0] * inv_dt - (double)d - (double)rho;
                    if (!(v >= 0.0 && v < (double)P)) continue;
                    const double jf = floor(v);
                    const int j = (int)jf;
                    double u = (v - jf) * S;
                    const double sf = floor(u);
                    const int sub = min((int)sf, S - 1);
                    u -= (double)sub;
                    const double x = 2.0 * u - 1.0;
                    const double *cf = A.cheb64 + ((size_t)((p0 + j) * S + sub) * NCHEB) * 2;
                    double ps = __ldg(cf) + __ldg(cf + 2) * x, pt = __ldg(cf + 1) + __ldg(cf + 3) * x;
                    double tm = 1.0, t = x;
                    const double x2 = x + x;
                    for (int n = 2; n < NCHEB; ++n) {
                        const double tn = x2 * t - tm;
                        tm = t; t = tn;
                        ps += __ldg(cf + 2 * n) * tn;
                        pt += __ldg(cf + 2 * n + 1) * tn;
                    }
                    const double lx[3] = {q[2], q[3], 1.0 - q[2] - q[3]};
                    const double ly[3] = {q[4], q[5], 1.0 - q[4] - q[5]};
                    const double wp = q[1] * ps;
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b) Sab[a][b] += wp * lx[a] * ly[b];
                    St += q[1] * pt;
                }
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b) Sab[a][b] = dsum_warp(Sab[a][b]);
                St = dsum_warp(St);
                if (lane < 9) {
                    const int a = lane / 3, b = lane % 3;
                    const int ca = pa[a], cb = pb[b];
                    const double *ct = g.geo64 + 16 * tau + 4 + 3 * ca, *cs = g.geo64 + 16 * sg + 4 + 3 * cb;
                    const double cc = ct[0] * cs[0] + ct[1] * cs[1] + ct[2] * cs[2];
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

// Special blocks (single blocks of the first / last time functions, support
// near r = 0 or near the corner lag) for element pairs WITHOUT a shared
// vertex, in FP64 with the 7-point rule on both triangles; used by the mixed
// path, whose FP32 kernel evaluates only the three lag classes. One CTA per
// test triangle of the current colour scans its pair records in trial order;
// its four warps take the qualifying pairs four at a time (lanes over the 49
// point pairs), and warp 0 adds their values into the far special-block
// windows in list order.
constexpr int FS_THREADS = 128;
constexpr int FS_WARPS = FS_THREADS / 32;
__global__ void __launch_bounds__(FS_THREADS)
farspec_kernel(const NearArgs A) {
    __shared__ int list[FS_THREADS];
    __shared__ int nlist;
    __shared__ double fs_val[FS_WARPS][NSPEC][9];  // one list entry per warp: its special-block values
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const Geo &g = A.g;
    const int64_t M = g.M, E = g.E, MM = M * M;
    const double inv_dt = A.lt.inv_dt;
    const int S = A.S;
    for (int64_t ti = blockIdx.x; ti < A.ncolor; ti += gridDim.x) {
        const int64_t tau = A.color_tris[ti];
        for (int64_t b0 = 0; b0 < E; b0 += FS_THREADS) {
            // ordered compaction of the qualifying trial triangles of this slice
            const int64_t sg = b0 + threadIdx.x;
            PairRec rc{};
            bool need = false;
            if (sg < E) {
                rc = A.rec[tau * E + sg];
                need = rc.adj == 0 && rc.smask != 0;
            }
            const unsigned bal = __ballot_sync(0xffffffffu, need);
            __shared__ int wcount[FS_THREADS / 32];
            if (lane == 0) wcount[w] = __popc(bal);
            __syncthreads();
            int off = 0;
            for (int k = 0; k < w; ++k) off += wcount[k];
            if (need) list[off + __popc(bal & ((1u << lane) - 1u))] = (int)sg;
            if (threadIdx.x == 0) {
                int t = 0;
                for (int k = 0; k < FS_THREADS / 32; ++k) t += wcount[k];
                nlist = t;
            }
            __syncthreads();
            // four list entries at a time, one per warp, into shared memory;
            // then warp 0 adds them in list order (entries can share a vertex
            // pair, so the adds stay in one fixed order)
            for (int q0 = 0; q0 < nlist; q0 += FS_WARPS) {
                const int q = q0 + w;
                if (q < nlist) {
                    const int64_t s2 = list[q];
                    const PairRec r2 = A.rec[tau * E + s2];
                    double nn = 0.0;
                    for (int d = 0; d < 3; ++d) nn += g.geo64[16 * tau + d] * g.geo64[16 * s2 + d];
                    const double scale = g.geo64[16 * tau + 3] * g.geo64[16 * s2 + 3] * 0.07957747154594767;
                    for (int sb = 0; sb < NSPEC; ++sb) {
                        if (!((r2.smask >> sb) & 1u)) continue;
                        const int c = NLAG + sb;
                        const int P = A.lt.P[c], rho = A.lt.rho[c];
                        int p0 = 0;
                        for (int x = 0; x < c; ++x) p0 += A.lt.P[x];
                        double Sab[3][3] = {{0, 0, 0}, {0, 0, 0}, {0, 0, 0}}, St = 0.0;
                        for (int pp = lane; pp < 49; pp += 32) {
                            const int ix = pp / 7, iy = pp % 7;
                            double r2s = 0.0;
                            for (int d = 0; d < 3; ++d) {
                                const double xd = g.cen[3 * tau + d] + g.dq[(tau * 7 + ix) * 3 + d];
                                const double yd = g.cen[3 * s2 + d] + g.dq[(s2 * 7 + iy) * 3 + d];
                                r2s += (xd - yd) * (xd - yd);
                            }
                            const double r = sqrt(r2s);
                            const double v = r * inv_dt - (double)rho;
                            if (!(v >= 0.0 && v < (double)P)) continue;
                            const double jf = floor(v);
                            double u = (v - jf) * S;
                            const int sub = min((int)floor(u), S - 1);
                            u -= (double)sub;
                            const double x = 2.0 * u - 1.0;
                            const double *cf = A.cheb64 + ((size_t)((p0 + (int)jf) * S + sub) * NCHEB) * 2;
                            double ps = __ldg(cf) + __ldg(cf + 2) * x, pt = __ldg(cf + 1) + __ldg(cf + 3) * x;
                            double tm = 1.0, t = x;
                            const double x2 = x + x;
                            for (int n = 2; n < NCHEB; ++n) {
                                const double tn = x2 * t - tm;
                                tm = t; t = tn;
                                ps += __ldg(cf + 2 * n) * tn;
                                pt += __ldg(cf + 2 * n + 1) * tn;
                            }
                            const double wgt = A.rule_w64[ix] * A.rule_w64[iy] * scale / r;
                            for (int a = 0; a < 3; ++a)
                                for (int b = 0; b < 3; ++b)
                                    Sab[a][b] += wgt * ps * A.rule_l64[3 * ix + a] * A.rule_l64[3 * iy + b];
                            St += wgt * pt;
                        }
                        for (int a = 0; a < 3; ++a)
                            for (int b = 0; b < 3; ++b) Sab[a][b] = dsum_warp(Sab[a][b]);
                        St = dsum_warp(St);
                        if (lane < 9) {
                            const int a = lane / 3, b = lane % 3;
                            const double *ct = g.geo64 + 16 * tau + 4 + 3 * a, *cs = g.geo64 + 16 * s2 + 4 + 3 * b;
                            const double cc = ct[0] * cs[0] + ct[1] * cs[1] + ct[2] * cs[2];
                            fs_val[w][sb][lane] = nn * Sab[a][b] + cc * St;
                        }
                    }
                }
                __syncthreads();
                if (w == 0 && lane < 9)
                    for (int k = 0; k < FS_WARPS && q0 + k < nlist; ++k) {
                        const int64_t s2 = list[q0 + k];
                        const PairRec r2 = A.rec[tau * E + s2];
                        const int a = lane / 3, b = lane % 3;
                        const int64_t l = g.F[3 * tau + a], j = g.F[3 * s2 + b];
                        for (int sb = 0; sb < NSPEC; ++sb)
                            if (((r2.smask >> sb) & 1u) && ((A.smask[l * M + j] >> sb) & 1u))
                                A.far_spec[sb * MM + l * M + j] += fs_val[k][sb][lane];
                    }
                __syncthreads();
            }
            __syncthreads();
        }
    }
}

void launch_farspec(const NearArgs &a, int grid, cudaStream_t st) {
    farspec_kernel<<<grid, FS_THREADS, 0, st>>>(a);
}

void launch_near(const NearArgs &a, int grid, cudaStream_t st) {
    int mx = 0;
    for (int k = 1; k <= 3; ++k) mx = a.ss_npp[k] > mx ? a.ss_npp[k] : mx;
    const size_t smem = (size_t)mx * 6 * sizeof(double) + (size_t)mx * sizeof(int16_t) + 16;
    cudaFuncSetAttribute(near_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    near_kernel<<<grid, NEAR_THREADS, smem, st>>>(a);
}

}  // namespace tdbem
