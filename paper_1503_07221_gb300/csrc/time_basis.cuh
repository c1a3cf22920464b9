// Device time basis of Sec. 3 (Eq. BasisFunctions) shared by the psi-table
// build (table.cu) and the potential evaluation (potential.cu): the p = 0
// functions (basis) and those of order m (basis_m).
#pragma once
#include <math.h>

namespace tdbem {

// Smooth step of Sec. 3: f(x) = erf(2 artanh x)/2 + 1/2 on |x| < 1, with
// u = 2 artanh x:  f' = (2/sqrt(pi)) e^{-u^2} / (1 - x^2),
//                  f'' = (4/sqrt(pi)) e^{-u^2} (x - 2u) / (1 - x^2)^2.
// kind 1: the step built from h(s) = e^{-1/s} (s = (x + 1)/2),
//   F = h(s) / (h(s) + h(1 - s)) = 1 / (1 + e^g), g = 1/s - 1/(1 - s),
//   dF/ds = F (1 - F) q, q = 1/s^2 + 1/(1 - s)^2,
//   d2F/ds2 = dF/ds (1 - 2F) q + F (1 - F) (2/(1 - s)^3 - 2/s^3), d/dx = d/ds / 2;
// fm = f(-x) = 1 - f(x) without cancellation (both steps are odd about 1/2).
__device__ static inline void smooth_step2(int kind, double x, double &f0, double &fm, double &f1, double &f2) {
    if (x <= -1.0) { f0 = 0.0; fm = 1.0; f1 = 0.0; f2 = 0.0; return; }
    if (x >= 1.0) { f0 = 1.0; fm = 0.0; f1 = 0.0; f2 = 0.0; return; }
    if (kind == 1) {
        const double s = 0.5 * (x + 1.0), sm = 0.5 * (1.0 - x);
        const double g = 1.0 / s - 1.0 / sm;
        f0 = 1.0 / (1.0 + exp(g));
        fm = 1.0 / (1.0 + exp(-g));
        const double ff = f0 * fm;
        if (ff == 0.0) { f1 = 0.0; f2 = 0.0; return; }
        const double q = 1.0 / (s * s) + 1.0 / (sm * sm);
        const double dq = 2.0 / (sm * sm * sm) - 2.0 / (s * s * s);
        const double d1 = ff * q;
        f1 = 0.5 * d1;
        f2 = 0.25 * (d1 * (fm - f0) * q + ff * dq);
        return;
    }
    const double u = 2.0 * atanh(x);
    const double gg = (1.0 - x) * (1.0 + x);
    const double e = exp(-u * u);
    const double k = 1.1283791670955126;  // 2 / sqrt(pi)
    f0 = 0.5 * erfc(-u);
    fm = 0.5 * erfc(u);
    f1 = k * e / gg;
    f2 = 2.0 * k * e * (x - 2.0 * u) / (gg * gg);
}
__device__ static inline void smooth_step(int kind, double x, double &f0, double &f1, double &f2) {
    double fm;
    smooth_step2(kind, x, f0, fm, f1, f2);
}

// Rising cutoff f_j(s) = f(2 (s - t_j)/h - 1), h = t_{j+1} - t_j, and the
// falling one 1 - f_j(s) = f(-(2 (s - t_j)/h - 1)), each with d/ds, d2/ds2.
__device__ static inline void rising(int kind, double s, double tj, double h, double out[3]) {
    double a, b, c;
    smooth_step(kind, 2.0 * (s - tj) / h - 1.0, a, b, c);
    out[0] = a; out[1] = b * 2.0 / h; out[2] = c * 4.0 / (h * h);
}
__device__ static inline void falling(int kind, double s, double tj, double h, double out[3]) {
    double a, b, c;
    smooth_step(kind, 1.0 - 2.0 * (s - tj) / h, a, b, c);
    out[0] = a; out[1] = -b * 2.0 / h; out[2] = c * 4.0 / (h * h);
}

// Time basis function i (0-based) of Eq. BasisFunctions with p = 0 (step of
// the given kind) and its
// first two derivatives at s; causal (zero for s < 0).
//   i = 0:     8 mu_1 (s/h)^2,   mu_1 = 1 - f_0
//   inner i:   mu_{i+1} = rho_i, rising on [t_{i-1}, t_i], falling on [t_i, t_{i+1}]
//   i = N-1:   mu_N = f_{N-2} (1 beyond t_{N-1})
__device__ static inline void basis(int kind, const double *t, int N, int i, double s, double out[3]) {
    out[0] = out[1] = out[2] = 0.0;
    if (s < 0.0) return;
    double m[3];
    if (i == 0) {
        const double h = t[1] - t[0];
        if (s >= t[1]) return;
        falling(kind, s, t[0], h, m);
        const double q = s / h;
        out[0] = 8.0 * m[0] * q * q;
        out[1] = 8.0 * m[1] * q * q + 16.0 * m[0] * q / h;
        out[2] = 8.0 * m[2] * q * q + 32.0 * m[1] * q / h + 16.0 * m[0] / (h * h);
        return;
    }
    if (i == N - 1) {
        if (s <= t[N - 2]) return;
        if (s >= t[N - 1]) { out[0] = 1.0; return; }
        rising(kind, s, t[N - 2], t[N - 1] - t[N - 2], out);
        return;
    }
    if (s <= t[i - 1] || s >= t[i + 1]) return;
    if (s <= t[i]) rising(kind, s, t[i - 1], t[i] - t[i - 1], out);
    else falling(kind, s, t[i], t[i + 1] - t[i], out);
}

// Legendre polynomial P_m and its first two derivatives at x, from the
// three-term recurrence (n + 1) P_{n+1} = (2n + 1) x P_n - n P_{n-1} and
// P'_{n+1} = P'_{n-1} + (2n + 1) P_n, P''_{n+1} = P''_{n-1} + (2n + 1) P'_n.
__device__ static inline void legendre3(int m, double x, double out[3]) {
    double p0 = 1.0, d0 = 0.0, e0 = 0.0;  // P_n, P'_n, P''_n at n = 0
    double pm = 0.0, dm = 0.0, em = 0.0;  // n - 1
    for (int n = 0; n < m; ++n) {
        const double p1 = ((2 * n + 1) * x * p0 - n * pm) / (n + 1);
        const double d1 = dm + (2 * n + 1) * p0, e1 = em + (2 * n + 1) * d0;
        pm = p0; dm = d0; em = e0;
        p0 = p1; d0 = d1; e0 = e1;
    }
    out[0] = p0; out[1] = d0; out[2] = e0;
}

// Time basis function b_{i,m} of order m (Eq. BasisFunctions): the p = 0
// function of basis() times the Legendre polynomial P_m of the coordinate
// that maps its support onto [-1, 1]:
//   i = 0:     P_m(2 s / h - 1),            h = t_1 - t_0
//   inner i:   P_m(2 (s - t_{i-1}) / (t_{i+1} - t_{i-1}) - 1)  (= (s - t_{i-1})/dt - 1 when equidistant)
//   i = N-1:   P_m(2 (s - t_{N-2}) / h - 1), h = t_{N-1} - t_{N-2};
// with the first two derivatives by the product rule.
__device__ static inline void basis_m(int kind, const double *t, int N, int i, int m, double s, double out[3]) {
    basis(kind, t, N, i, s, out);
    if (m == 0 || (out[0] == 0.0 && out[1] == 0.0 && out[2] == 0.0)) return;
    double a, c;
    if (i == 0) { a = 2.0 / (t[1] - t[0]); c = -1.0 - a * t[0]; }
    else if (i == N - 1) { a = 2.0 / (t[N - 1] - t[N - 2]); c = -1.0 - a * t[N - 2]; }
    else { a = 2.0 / (t[i + 1] - t[i - 1]); c = -1.0 - a * t[i - 1]; }
    double L[3];
    legendre3(m, a * s + c, L);
    const double l0 = L[0], l1 = a * L[1], l2 = a * a * L[2];
    const double b0 = out[0], b1 = out[1], b2 = out[2];
    out[0] = b0 * l0;
    out[1] = b1 * l0 + b0 * l1;
    out[2] = b2 * l0 + 2.0 * b1 * l1 + b0 * l2;
}
}  // namespace tdbem
