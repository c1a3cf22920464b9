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


void launch_near(const NearArgs &a, int grid, cudaStream_t st) {
    int mx = 0;
    for (int k = 1; k <= 3; ++k) mx = a.ss_npp[k] > mx ? a.ss_npp[k] : mx;
    const size_t smem = (size_t)mx * 6 * sizeof(double) + (size_t)mx * sizeof(int16_t) + 16;
    cudaFuncSetAttribute(near_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    near_kernel<<<grid, NEAR_THREADS, smem, st>>>(a);
}

}  // namespace tdbem
