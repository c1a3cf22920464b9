// psi / psi~ Chebyshev tables (paper Sec. 3.1): sample the time-convolved
// basis functions of Eq. psis by a direct 1-D Gauss-Legendre quadrature on
// the device (FP64), then transform the samples at Chebyshev points of the
// first kind into coefficients.
#include <math.h>

#include "tdbem_internal.h"
#include "time_basis.cuh"

namespace tdbem {

__device__ static double left_end(const double *t, int N, int i) { return i == 0 ? 0.0 : t[i - 1]; }
__device__ static double right_end(const double *t, int N, int i) { return i == N - 1 ? t[N - 1] : t[i + 1]; }

// psi_{k,i}(r) and psi~_{k,i}(r) of Eq. psis: integrate over the overlap of
// the test support and the shifted trial support, split at the interior
// breakpoints t_k and t_i + r, composite Gauss-Legendre on each piece. One
// warp evaluates one sample: lane L takes the nodes L, L + 32, ... of each
// piece (sub-interval-major), and the partial sums are added across the warp
// in a fixed order, so every lane returns the same values on every run.
__device__ static void psi_direct_warp(int bkind, const double *t, int N, int kb, int m2, int ib, int m1, double r,
                                       const double *gx, const double *gw, int gn, int gsub, int lane, double &psi,
                                       double &psit) {
    psi = 0.0; psit = 0.0;
    const double lo = fmax(left_end(t, N, kb), left_end(t, N, ib) + r);
    const double hi = fmin(right_end(t, N, kb), right_end(t, N, ib) + r);
    if (!(lo < hi)) return;
    double br[4];
    int nb = 0;
    br[nb++] = lo;
    if (kb > 0 && kb < N - 1 && t[kb] > lo && t[kb] < hi) br[nb++] = t[kb];
    if (ib > 0 && ib < N - 1 && t[ib] + r > lo && t[ib] + r < hi) br[nb++] = t[ib] + r;
    br[nb++] = hi;
    if (nb == 4 && br[1] > br[2]) { double x = br[1]; br[1] = br[2]; br[2] = x; }
    double s0 = 0.0, s1 = 0.0;
    const int nq = gsub * gn;
    for (int p = 0; p + 1 < nb; ++p) {
        const double a = br[p], w = (br[p + 1] - br[p]) / gsub;
        if (!(w > 0.0)) continue;
        for (int e = lane; e < nq; e += 32) {
            const int q = e / gn, g = e - q * gn;
            const double tt = (a + q * w) + w * gx[g];
            double bk[3], bi[3];
            basis_m(bkind, t, N, kb, m2, tt, bk);
            basis_m(bkind, t, N, ib, m1, tt - r, bi);
            s0 += w * gw[g] * bi[2] * bk[1];
            s1 += w * gw[g] * bi[0] * bk[1];
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        s0 += __shfl_xor_sync(0xffffffffu, s0, o);
        s1 += __shfl_xor_sync(0xffffffffu, s1, o);
    }
    psi = s0;
    psit = s1;
}

// One warp per (sub-panel, Chebyshev node), so that the few hundred samples
// of a table spread over every SM (the FP64 quadrature is the cost). Sub-panel
// p covers r in [r0[p], r0[p] + dr] of the block (kb[p], ib[p]); with pdr
// given, its width is pdr[p] instead (uneven panels of a graded grid); with
// pm2, pm1 given, the block's test and trial temporal orders (else 0).
__global__ void psi_samples_kernel(int bkind, const double *t, int N, const int *pkb, const int *pib,
                                   const int *pm2, const int *pm1, const double *pr0, double dr, const double *pdr,
                                   int total, const double *gx, const double *gw, int gn, int gsub,
                                   double *samples) {
    const int64_t id = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const int lane = threadIdx.x & 31;
    if (id >= (int64_t)total * NCHEB) return;
    const int p = (int)(id / NCHEB), m = (int)(id % NCHEB);
    const double xm = cos(M_PI * (m + 0.5) / NCHEB);
    const double w = pdr ? pdr[p] : dr;
    const double r = pr0[p] + 0.5 * w * (xm + 1.0);
    double a, b;
    psi_direct_warp(bkind, t, N, pkb[p], pm2 ? pm2[p] : 0, pib[p], pm1 ? pm1[p] : 0, r, gx, gw, gn, gsub, lane, a,
                    b);
    if (lane == 0) {
        samples[2 * id + 0] = a;
        samples[2 * id + 1] = b;
    }
}

// c_n = (2/K) sum_m f(x_m) cos(n pi (m + 1/2)/K), c_0 halved, K = NCHEB; the
// panel is then f(x) = sum_n c_n T_n(x) with x in [-1, 1].
__global__ void psi_dct_kernel(const double *samples, int total, double *coef) {
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= total * NCHEB) return;
    const int p = id / NCHEB, n = id % NCHEB;
    double s0 = 0.0, s1 = 0.0;
    for (int m = 0; m < NCHEB; ++m) {
        const double c = cos(M_PI * n * (m + 0.5) / NCHEB);
        s0 += samples[2 * (p * NCHEB + m) + 0] * c;
        s1 += samples[2 * (p * NCHEB + m) + 1] * c;
    }
    const double sc = (n == 0 ? 1.0 : 2.0) / NCHEB;
    coef[2 * id + 0] = s0 * sc;
    coef[2 * id + 1] = s1 * sc;
}

void launch_psi_samples(int bkind, const double *t, int N, const int *panel_class, const int *panel_kb,
                        const int *panel_ib, const double *panel_r0, double panel_dr, int S,
                        int total_sub, const double *gl_x, const double *gl_w, int gl_n, int gl_sub,
                        double *samples, cudaStream_t st) {
    (void)panel_class; (void)S;
    const int64_t n = (int64_t)total_sub * NCHEB * 32;
    psi_samples_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(bkind, t, N, panel_kb, panel_ib, nullptr, nullptr,
                                                       panel_r0, panel_dr, nullptr, total_sub, gl_x, gl_w, gl_n,
                                                       gl_sub, samples);
}

void launch_psi_samples_var(int bkind, const double *t, int N, const int *panel_kb, const int *panel_ib,
                            const int *panel_m2, const int *panel_m1, const double *panel_r0, const double *panel_dr,
                            int total_sub, const double *gl_x, const double *gl_w, int gl_n, int gl_sub,
                            double *samples, cudaStream_t st) {
    const int64_t n = (int64_t)total_sub * NCHEB * 32;
    if (n <= 0) return;
    psi_samples_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(bkind, t, N, panel_kb, panel_ib, panel_m2, panel_m1,
                                                       panel_r0, 0.0, panel_dr, total_sub, gl_x, gl_w, gl_n, gl_sub,
                                                       samples);
}

// Evaluation of one block's table at distances r (thread per r): the block
// of lag d in a class with prototype panels [rho, rho + P) in q = r / dt reads
// panel floor(q - d - rho); the FP64 set has S sub-panels per panel (c64),
// the FP32 set one (c32 with the FP32 residuals of the leading coefficients,
// summed here in FP64 so that only the table itself is measured).
__global__ void psi_table_kernel(const double *r, int64_t n, double inv_dt, int lag, int rho, int P, int panel0,
                                 int S, const double *c64, const ChebF32 c32, int use32, double *out) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n) return;
    const double z = r[id] * inv_dt - lag - rho;
    double a = 0.0, b = 0.0;
    if (z > 0.0 && z < (double)P) {
        const int p = min((int)floor(z), P - 1);
        double f = z - p;
        int sub = 0;
        if (!use32) {
            sub = min((int)floor(f * S), S - 1);
            f = f * S - sub;
        }
        const double x = 2.0 * f - 1.0;
        double tm = 1.0, t = x;
        for (int k = 0; k < NCHEB; ++k) {
            double ca, cb;
            if (use32) {
                ca = (double)c32.c[panel0 + p][k][0] + (k < NCHEB_LO ? (double)c32.lo[panel0 + p][k][0] : 0.0);
                cb = (double)c32.c[panel0 + p][k][1] + (k < NCHEB_LO ? (double)c32.lo[panel0 + p][k][1] : 0.0);
            } else {
                const double *c = c64 + ((size_t)((panel0 + p) * S + sub) * NCHEB + k) * 2;
                ca = c[0];
                cb = c[1];
            }
            const double tk = k == 0 ? 1.0 : (k == 1 ? x : 2.0 * x * t - tm);
            if (k >= 2) { tm = t; t = tk; }
            a += ca * tk;
            b += cb * tk;
        }
    }
    out[2 * id] = a;
    out[2 * id + 1] = b;
}

void launch_psi_table(const double *r, int64_t n, double inv_dt, int lag, int rho, int P, int panel0, int S,
                      const double *c64, const ChebF32 &c32, int use32, double *out, cudaStream_t st) {
    if (n <= 0) return;
    psi_table_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(r, n, inv_dt, lag, rho, P, panel0, S, c64, c32,
                                                                 use32, out);
}

void launch_psi_dct(const double *samples, int total_sub, double *coef, cudaStream_t st) {
    const int n = total_sub * NCHEB;
    psi_dct_kernel<<<(n + 127) / 128, 128, 0, st>>>(samples, total_sub, coef);
}

// ---- right-hand side g_k(l) = int_0^T int_Gamma g(x,t) phi_l(x) bdot_k(t) ----
// (the vector of the linear system, Sec. 3). Neumann data by kind (with the
// time grid scaled by the wave speed c, the data are taken at t = s / c):
//   RHS_PLANE_WAVE  u_inc = exp(-(t - x.d - c0)^2 / (2 w^2)), p = (d, c0, w):
//                   g = -du_inc/dn = (d.n) f'(t - x.d)  (sound-hard scatterer)
//   RHS_SPHERE_N0   g = Y_0^0 sin(3t) t^2 e^{-t}           (Sec. 6.1)
//   RHS_SPHERE_N1   g = Y_1^0(x) sin(2 pi t) t^3 e^{-2t}   (Sec. 6.1)
__device__ static double rhs_data(int kind, const double *prm, const double *x, const double *n, double t) {
    if (kind == RHS_PLANE_WAVE) {
        const double s = t - (x[0] * prm[0] + x[1] * prm[1] + x[2] * prm[2]) - prm[3];
        const double w = prm[4];
        const double fp = -s / (w * w) * exp(-0.5 * (s / w) * (s / w));
        return (n[0] * prm[0] + n[1] * prm[1] + n[2] * prm[2]) * fp;
    }
    if (t <= 0.0) return 0.0;
    if (kind == RHS_SPHERE_N0) return 0.28209479177387814 * sin(3.0 * t) * t * t * exp(-t);  // Y_0^0 = 1/sqrt(4 pi)
    return 0.48860251190291992 * x[2] * sin(2.0 * M_PI * t) * t * t * t * exp(-2.0 * t);     // Y_1^0 = sqrt(3/(4 pi)) z
}

// One thread per (time index k, vertex l): the triangles around l, 7 points
// each, and the support of bdot_k split at every grid point into `sub`
// panels of gn Gauss-Legendre points (FP64).
__global__ void rhs_kernel(int bkind, Geo g, const double *t, int N, int P1, double c, const double *rule_w,
                           const double *rule_l, const double *gx, const double *gw, int gn, int sub, int kind,
                           RhsParams prm, double *out) {
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= (int64_t)N * P1 * g.M) return;
    const int row = (int)(id / g.M), k = row / P1, mo = row % P1;  // time function b_{k,mo}: row k (p + 1) + mo
    const int64_t l = id % g.M;
    const int j0 = k == 0 ? 0 : k - 1, j1 = k == N - 1 ? N - 1 : k + 1;  // support [t_j0, t_j1]
    double acc = 0.0;
    for (int64_t q = g.vt_ptr[l]; q < g.vt_ptr[l + 1]; ++q) {
        const int64_t e = g.vt_tri[q];
        const int a = g.F[3 * e] == l ? 0 : (g.F[3 * e + 1] == l ? 1 : 2);
        const double *geo = g.geo64 + 16 * e;  // n(3), area
        for (int p = 0; p < 7; ++p) {
            double x[3];
            for (int d = 0; d < 3; ++d) x[d] = g.cen[3 * e + d] + g.dq[(e * 7 + p) * 3 + d];
            double it = 0.0;
            for (int j = j0; j < j1; ++j) {
                const double h = (t[j + 1] - t[j]) / sub;
                for (int sb = 0; sb < sub; ++sb)
                    for (int m = 0; m < gn; ++m) {
                        const double s = t[j] + (sb + gx[m]) * h;
                        double b[3];
                        basis_m(bkind, t, N, k, mo, s, b);
                        it += gw[m] * h * b[1] * rhs_data(kind, prm.p, x, geo, s / c);
                    }
            }
            acc += geo[3] * rule_w[p] * rule_l[3 * p + a] * it;
        }
    }
    out[id] = acc;
}

void launch_rhs(int bkind, const Geo &g, const double *t, int N, int P1, double c, const double *rule_w,
                const double *rule_l, const double *gx, const double *gw, int gn, int sub, int kind,
                const RhsParams &prm, double *out, cudaStream_t st) {
    const int64_t n = (int64_t)N * P1 * g.M;
    rhs_kernel<<<(unsigned)((n + 127) / 128), 128, 0, st>>>(bkind, g, t, N, P1, c, rule_w, rule_l, gx, gw, gn, sub, kind,
                                                          prm, out);
}

}  // namespace tdbem
