// Retarded double layer potential at points off the surface (Sec. 2, Eq.
// RetardedPotential): the evaluation of a solution of the boundary integral
// equation in the domain,
//
//   u(x, t) = -1/(4 pi) int_Gamma n_y.(x - y)/|x - y|
//               [ phi(y, t - r)/r^2 + d_t phi(y, t - r)/r ] dGamma_y,  r = |x - y|,
//
// with the density phi(y, s) = sum_{k, j} alpha[k M + j] b_k(s) phi_j(y) of
// the space-time basis (p = 0). Every flat triangle is integrated by the
// collapsed Gauss product rule: (u, v) in [0, 1]^2 with n Gauss-Legendre
// points per direction, barycentric (1 - u, u (1 - v), u v), weight
// 2 u w_u w_v |T|. FP64 throughout. Times are scaled by the wave speed as the
// time grid is, so r enters as r / c.
//
// One thread per (point, time); the quadrature points pass through shared
// memory in tiles, so a warp reads each point once. At a retarded time s
// in (t_j, t_{j+1}) only b_j (falling flank) and b_{j+1} (rising flank) are
// nonzero, and both come from one evaluation of the smooth step; beyond
// t_{N-1} only b_{N-1} = 1 remains; before 0 nothing (causality). The step is
// read from a quintic Hermite interpolant of its values and first two
// derivatives at 1025 equidistant nodes on [-1, 1], built from the exact
// step at every call (interpolation error 3e-16 in f, 3e-13 in f'), instead
// of an artanh, an exp and two erfc per point.
#include <math.h>

#include "tdbem_internal.h"
#include "time_basis.cuh"

namespace tdbem {

constexpr int DL_THREADS = 256;
constexpr int DL_TILE = 128;
constexpr int DL_NODES = 1024;  // Hermite intervals of the step table on [-1, 1]

// step table: (f, h f', h^2 f'') at x_i = -1 + i h, h = 2 / DL_NODES
__global__ void dl_step_table_kernel(int bkind, double3 *tab) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i > DL_NODES) return;
    const double h = 2.0 / DL_NODES;
    const double x = -1.0 + i * h;
    double f0, fm, f1, f2;
    smooth_step2(bkind, x, f0, fm, f1, f2);
    tab[i] = make_double3(f0, h * f1, h * h * f2);
}

// f(x) and f'(x) from the quintic Hermite interpolant of the table
__device__ __forceinline__ void step_hermite(const double3 *tab, double x, double &f, double &d) {
    if (x <= -1.0) { f = 0.0; d = 0.0; return; }
    if (x >= 1.0) { f = 1.0; d = 0.0; return; }
    const double u = (x + 1.0) * (0.5 * DL_NODES);
    const int i = min((int)u, DL_NODES - 1);
    const double t = u - i, t2 = t * t, t3 = t2 * t, t4 = t3 * t, t5 = t4 * t;
    const double3 a = tab[i], b = tab[i + 1];
    f = a.x * (1.0 - 10.0 * t3 + 15.0 * t4 - 6.0 * t5) + a.y * (t - 6.0 * t3 + 8.0 * t4 - 3.0 * t5) +
        a.z * 0.5 * (t2 - 3.0 * t3 + 3.0 * t4 - t5) + b.x * (10.0 * t3 - 15.0 * t4 + 6.0 * t5) +
        b.y * (-4.0 * t3 + 7.0 * t4 - 3.0 * t5) + b.z * 0.5 * (t3 - 2.0 * t4 + t5);
    d = (a.x * (-30.0 * t2 + 60.0 * t3 - 30.0 * t4) + a.y * (1.0 - 18.0 * t2 + 32.0 * t3 - 15.0 * t4) +
         a.z * 0.5 * (2.0 * t - 9.0 * t2 + 12.0 * t3 - 5.0 * t4) + b.x * (30.0 * t2 - 60.0 * t3 + 30.0 * t4) +
         b.y * (-12.0 * t2 + 28.0 * t3 - 15.0 * t4) + b.z * 0.5 * (3.0 * t2 - 8.0 * t3 + 5.0 * t4)) *
        (0.5 * DL_NODES);
}

// quadrature points: y (xyz, 0) and the weighted normal w n_T (xyz, 0)
__global__ void dl_points_kernel(const Geo g, const double *gx, const double *gw, int n, double4 *yw) {
    const int64_t Q = (int64_t)n * n;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= g.E * Q) return;
    const int64_t e = id / Q;
    const int q = (int)(id % Q), iu = q / n, iv = q % n;
    const double u = gx[iu], v = gx[iv];
    const double l0 = 1.0 - u, l1 = u * (1.0 - v), l2 = u * v;
    const double *geo = g.geo64 + 16 * e;
    const double w = 2.0 * u * gw[iu] * gw[iv] * geo[3];
    const double *P0 = g.V + 3 * g.F[3 * e], *P1 = g.V + 3 * g.F[3 * e + 1], *P2 = g.V + 3 * g.F[3 * e + 2];
    yw[2 * id] = make_double4(l0 * P0[0] + l1 * P1[0] + l2 * P2[0], l0 * P0[1] + l1 * P1[1] + l2 * P2[1],
                              l0 * P0[2] + l1 * P1[2] + l2 * P2[2], 0.0);
    yw[2 * id + 1] = make_double4(w * geo[0], w * geo[1], w * geo[2], 0.0);
}

// density coefficients at the quadrature points: coef[k EQ + id] =
// sum_a lambda_a(q) alpha[k M + F[e][a]]
__global__ void dl_coef_kernel(const Geo g, const double *gx, int n, int N, const double *alpha, double *coef) {
    const int64_t Q = (int64_t)n * n, EQ = g.E * Q;
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= EQ * N) return;
    const int k = (int)(id / EQ);
    const int64_t r = id % EQ, e = r / Q;
    const int q = (int)(r % Q), iu = q / n, iv = q % n;
    const double u = gx[iu], v = gx[iv];
    const double *a = alpha + (int64_t)k * g.M;
    coef[id] = (1.0 - u) * a[g.F[3 * e]] + u * (1.0 - v) * a[g.F[3 * e + 1]] + u * v * a[g.F[3 * e + 2]];
}

__global__ void __launch_bounds__(DL_THREADS)
dl_eval_kernel(const double3 *tab, const double *X, int64_t P, const double *times, int nt, double c, const double *tg,
               int N, int equi, const double4 *yw, const double *coef, int64_t EQ, double *out) {
    __shared__ double4 sy[DL_TILE], sw[DL_TILE];
    __shared__ double st[1024];
    __shared__ double3 stab[DL_NODES + 1];
    for (int i = threadIdx.x; i < N; i += blockDim.x) st[i] = tg[i];
    for (int i = threadIdx.x; i <= DL_NODES; i += blockDim.x) stab[i] = tab[i];
    const double idt = (N - 1) / tg[N - 1];
    const int64_t id = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool act = id < P * nt;
    const int64_t p = act ? id / nt : 0;
    const int it = act ? (int)(id % nt) : 0;
    const double x0 = act ? X[3 * p] : 0.0, x1 = act ? X[3 * p + 1] : 0.0, x2 = act ? X[3 * p + 2] : 0.0;
    const double ts = act ? c * times[it] : -1.0;
    const double T = tg[N - 1];
    double acc = 0.0;
    for (int64_t base = 0; base < EQ; base += DL_TILE) {
        __syncthreads();
        for (int j = threadIdx.x; j < DL_TILE && base + j < EQ; j += blockDim.x) {
            sy[j] = yw[2 * (base + j)];
            sw[j] = yw[2 * (base + j) + 1];
        }
        __syncthreads();
        const int nj = (int)min((int64_t)DL_TILE, EQ - base);
        for (int j = 0; j < nj; ++j) {
            const double d0 = x0 - sy[j].x, d1 = x1 - sy[j].y, d2 = x2 - sy[j].z;
            const double r2 = d0 * d0 + d1 * d1 + d2 * d2;
            const double r = sqrt(r2);
            const double s = ts - r;
            if (!(s > 0.0)) continue;
            const double ir = 1.0 / r;
            const double kern = (sw[j].x * d0 + sw[j].y * d1 + sw[j].z * d2) * ir;
            double phi, dphi;
            if (s >= T) {
                phi = coef[(int64_t)(N - 1) * EQ + base + j];
                dphi = 0.0;
            } else {
                // interval t_lo <= s < t_lo+1: index on an equidistant grid
                // (corrected by one for rounding), binary search otherwise
                int lo;
                if (equi) {
                    lo = min(max((int)(s * idt), 0), N - 2);
                    if (st[lo] > s) --lo;
                    else if (st[lo + 1] <= s) ++lo;
                } else {
                    lo = 0;
                    int hi = N - 1;
                    while (hi - lo > 1) {
                        const int mid = (lo + hi) >> 1;
                        if (st[mid] <= s) lo = mid;
                        else hi = mid;
                    }
                }
                const double h = st[lo + 1] - st[lo];
                const double xx = 2.0 * (s - st[lo]) / h - 1.0;
                double fr, f1;
                step_hermite(stab, xx, fr, f1);
                const double ff = 1.0 - fr;  // f(-x): the step is odd about 1/2
                const double df = f1 * 2.0 / h;
                // b_lo falls (times 8 (s/h)^2 for the first function), b_lo+1 rises
                double b0 = ff, db0 = -df;
                if (lo == 0) {
                    const double q = s / h;
                    db0 = 8.0 * (-df * q * q + 2.0 * ff * q / h);
                    b0 = 8.0 * ff * q * q;
                }
                const double c0 = coef[(int64_t)lo * EQ + base + j], c1 = coef[(int64_t)(lo + 1) * EQ + base + j];
                phi = c0 * b0 + c1 * fr;
                dphi = c0 * db0 + c1 * df;
            }
            acc += kern * ir * (phi * ir + dphi);
        }
    }
    if (act) out[id] = -acc * 0.079577471545947668;  // 1 / (4 pi)
}

cudaError_t launch_double_layer(int bkind, const Geo &g, const double *tg, int N, int equi, double c, const double *gx,
                                const double *gw, int n, const double *alpha, const double *X, int64_t P,
                                const double *times, int nt, double4 *yw, double *coef, double3 *tab, double *out,
                                cudaStream_t st) {
    const int64_t EQ = g.E * (int64_t)n * n;
    dl_step_table_kernel<<<(DL_NODES + 1 + 127) / 128, 128, 0, st>>>(bkind, tab);
    dl_points_kernel<<<(unsigned)((EQ + 255) / 256), 256, 0, st>>>(g, gx, gw, n, yw);
    dl_coef_kernel<<<(unsigned)((EQ * N + 255) / 256), 256, 0, st>>>(g, gx, n, N, alpha, coef);
    const int64_t nth = P * nt;
    if (nth > 0)
        dl_eval_kernel<<<(unsigned)((nth + DL_THREADS - 1) / DL_THREADS), DL_THREADS, 0, st>>>(
            tab, X, P, times, nt, c, tg, N, equi, yw, coef, EQ, out);
    return cudaGetLastError();
}

}  // namespace tdbem
