/*
 * tdbem_oracle.c -- plain, slow, FP64 CPU oracle for the space-time Galerkin
 * assembly of the time-domain hypersingular operator (3-D wave equation,
 * Neumann data), following Veit, Merta, Zapletal, Lukas, "Efficient solution
 * of time-domain boundary integral equations arising in sound-hard
 * scattering" (arXiv 1503.07221).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline leg of the benchmark load this library. It shares no code, header,
 * table or constant generator with the CUDA library; it receives the same
 * mesh and time-grid arrays as plain input data.
 *
 * What it computes, step by step (paper section in brackets):
 *   smooth step f(x) = erf(2 artanh x)/2 + 1/2               [Sec. 3]
 *     (option: the step of h(s) = e^{-1/s}, s = (x+1)/2, below)
 *   bump / partition of unity mu_i, basis b_{i,m}              [Sec. 3, Eq. BasisFunctions]
 *   psi_{k,i}(r)  = int_0^T  b''_i(t-r) b'_k(t) dt             [Eq. psis]
 *   psi~_{k,i}(r) = int_0^T  b_i(t-r)   b'_k(t) dt             [Eq. psis]
 *   A_{k,i}(j,l)  = int int [ n_x.n_y phi_j(y) phi_l(x) psi(|x-y|)
 *                    + curl phi_j(y).curl phi_l(x) psi~(|x-y|) ] / (4 pi |x-y|)
 *                                                              [Eq. MatrixEntries]
 *   sparsity: entry (l,j) of block (k~,i~) is structural iff
 *     [mindist_{l,j}, maxdist_{l,j}] meets supp psi_{k,i}     [Eq. SparsitySmallBlock]
 *   supp psi_{k,i} = [t_{k~-2} - t_{i~}, t_{k~} - t_{i~-2}] >= 0  [Sec. 3.2]
 *   unique blocks: first two block columns, last block row, (2,3), (N-1,N)
 *                                                              [Sec. 5.1, Eq. relationAtildeBlock]
 *
 * Quadrature (the paper does not fix the spatial rule; the workloads fix it):
 *   far element pairs (no shared vertex): 7-point degree-5 rule (Radon) on
 *   each triangle, tensor product of 49 point pairs; element pairs sharing a
 *   vertex, an edge or the whole triangle: Sauter-Schwab regularising maps of
 *   [0,1]^4 (Sauter & Schwab, Boundary Element Methods, Sec. 5.2) with
 *   Gauss-Legendre points per direction.
 *
 * Readings where the paper is silent or ambiguous:
 *   - the paper's N counts grid points t_0..t_{N-1}; basis index i = 1..N;
 *     0-based index ib = i-1 is used here; t_{-1} := 0 and t_N := T
 *   - basis functions are causal: b_i(s) := 0 for s < 0
 *   - non-equidistant grids: f_i uses the local width t_{i+1}-t_i, the
 *     Legendre argument of an inner function uses t_i - t_{i-2}
 *   - support endpoints are open: a block keeps an entry iff mindist < b and
 *     maxdist > a (equality culls); bounds within 1e-12 T of an endpoint
 *     count as equal, since psi vanishes to all orders there and symmetric
 *     meshes put exact ties on multiples of the time step
 *   - wave speed c = 1
 *
 * Exposed through a plain C ABI (ctypes) for the tests; see oracle.py.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_PI 3.14159265358979323846

/* ------------------------------------------------------------------------ */
/* Gauss-Legendre nodes on [0,1] by Newton's method on P_n                  */
/* ------------------------------------------------------------------------ */
static void gauss_legendre01(int n, double *x, double *w)
{
    for (int i = 0; i < n; ++i) {
        double z = cos(OR_PI * (i + 0.75) / (n + 0.5));
        double dp = 1.0;
        for (int it = 0; it < 100; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            if (n == 1) { p1 = z; p0 = 1.0; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-16) break;
        }
        {   /* final derivative at the converged node */
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) {
                double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
                p0 = p1;
                p1 = p2;
            }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
        }
        x[i] = 0.5 * (1.0 - z);
        w[i] = 1.0 / ((1.0 - z * z) * dp * dp);  /* 2/((1-z^2)P'^2) on [-1,1], halved */
    }
}

/* ------------------------------------------------------------------------ */
/* Problem                                                                  */
/* ------------------------------------------------------------------------ */
typedef struct {
    int64_t nb;            /* panels */
    double *edge;          /* nb*S+1 sub-panel edges */
    int S, n;              /* sub-panels per panel, interpolation degree */
    int64_t nsub;
    double *val;           /* nsub*(n+1)*2  (psi, psi~) at 2nd-kind Chebyshev points */
} or_interp;

typedef struct {
    int64_t M, E, N;
    int p;
    double *V;       /* M*3 */
    int32_t *F;      /* E*3 */
    double *t;       /* N */
    double T;
    /* triangle data */
    double *nrm;     /* E*3 */
    double *area;    /* E */
    double *curl;    /* E*9: curl of the hat function of corner a, a=0..2 */
    /* vertex -> (triangle, corner) adjacency */
    int64_t *vt_ptr;
    int32_t *vt_tri;
    int32_t *vt_cor;
    /* quadrature parameters */
    int gl_n, gl_sub;          /* psi direct: Gauss points per piece, pieces */
    double *gl_x, *gl_w;
    int ss_n;                  /* Sauter-Schwab points per direction */
    double *ss_x, *ss_w;
    int psi_mode;              /* 0 direct, 1 own interpolant */
    int interp_S, interp_n;
    double diam;
    double tie;                /* support-endpoint tie band: 1e-12 T */
    int maxval;                /* maximum number of triangles at a vertex */
    /* unique blocks */
    int64_t nblk;
    int32_t *bk, *bi;          /* 0-based test / trial basis index */
    int32_t *bm2, *bm1;        /* temporal orders */
    or_interp *interp;         /* per block (built at creation when psi_mode==1) */
    int first_kind;            /* 0: paper's b_1 = 8 mu_1 (t/dt)^2 P_m; 1: mu_1 (test hook) */
    int basis_kind;            /* smooth step: 0 erf(2 artanh x)/2 + 1/2 (Sec. 3), 1 exp(-1/s) step */
} orc_t;

static double tl(const orc_t *P, int ib) { return ib == 0 ? 0.0 : P->t[ib - 1]; }
static double tr(const orc_t *P, int ib) { return ib == P->N - 1 ? P->T : P->t[ib + 1]; }

/* ------------------------------------------------------------------------ */
/* Smooth step f and its derivatives (Sec. 3)                               */
/*   f(x) = erf(2 artanh x)/2 + 1/2 on |x|<1, 0 for x<=-1, 1 for x>=1       */
/*   with u = 2 artanh x: f' = (2/sqrt(pi)) e^{-u^2} / (1-x^2)              */
/*                        f''= (4/sqrt(pi)) e^{-u^2} (x-2u) / (1-x^2)^2     */
/* ------------------------------------------------------------------------ */
static void step_erf(double x, double out[3])
{
    if (x <= -1.0) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
    if (x >= 1.0) { out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; return; }
    double u = 2.0 * atanh(x);
    double omx2 = (1.0 - x) * (1.0 + x);
    double e = exp(-u * u);
    out[0] = 0.5 * erfc(-u);
    out[1] = (2.0 / sqrt(OR_PI)) * e / omx2;
    out[2] = (4.0 / sqrt(OR_PI)) * e * (x - 2.0 * u) / (omx2 * omx2);
}

/* The other smooth step: with s = (x+1)/2 and h(s) = exp(-1/s) (0 for s<=0),
 *   F(s) = h(s) / (h(s) + h(1-s)).
 * Differentiating the quotient directly:
 *   h'(s) = h(s)/s^2,   h''(s) = h(s) (1 - 2 s)/s^4,
 *   with a = h(s), b = h(1-s): F = a/(a+b),
 *   F' = (a' b - a b')/(a+b)^2,  b' = -h'(1-s),
 *   F'' = [(a'' b - a b'')(a+b) - 2 (a' b - a b')(a' + b')]/(a+b)^3,  b'' = h''(1-s),
 * and d/dx = (1/2) d/ds. Near the ends a or b underflows to 0; then F is 0
 * or 1 and its derivatives 0 to working precision. */
static void step_expinv(double x, double out[3])
{
    if (x <= -1.0) { out[0] = 0.0; out[1] = 0.0; out[2] = 0.0; return; }
    if (x >= 1.0) { out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; return; }
    double s = 0.5 * (x + 1.0), z = 0.5 * (1.0 - x);
    double a = exp(-1.0 / s), b = exp(-1.0 / z);
    double den = a + b;
    if (a == 0.0 || b == 0.0) { out[0] = a == 0.0 ? 0.0 : 1.0; out[1] = 0.0; out[2] = 0.0; return; }
    double a1 = a / (s * s), b1 = -b / (z * z);
    double a2 = a * (1.0 - 2.0 * s) / (s * s * s * s), b2 = b * (1.0 - 2.0 * z) / (z * z * z * z);
    double num1 = a1 * b - a * b1;
    out[0] = a / den;
    out[1] = 0.5 * num1 / (den * den);
    out[2] = 0.25 * ((a2 * b - a * b2) * den - 2.0 * num1 * (a1 + b1)) / (den * den * den);
}

static void step_f(int kind, double x, double out[3])
{
    if (kind == 1) step_expinv(x, out);
    else step_erf(x, out);
}

/* Legendre polynomial P_m and its first two derivatives at x */
static void legendre(int m, double x, double out[3])
{
    double p0 = 1.0, d0 = 0.0, s0 = 0.0;
    if (m == 0) { out[0] = 1.0; out[1] = 0.0; out[2] = 0.0; return; }
    double p1 = x, d1 = 1.0, s1 = 0.0;
    for (int k = 2; k <= m; ++k) {
        double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
        double d2 = ((2.0 * k - 1.0) * (p1 + x * d1) - (k - 1.0) * d0) / k;
        double s2 = ((2.0 * k - 1.0) * (2.0 * d1 + x * s1) - (k - 1.0) * s0) / k;
        p0 = p1; p1 = p2; d0 = d1; d1 = d2; s0 = s1; s1 = s2;
    }
    out[0] = p1; out[1] = d1; out[2] = s1;
}

/* mu_i (0-based ib) with first and second time derivative at s (Sec. 3):
 *   mu_1 = 1 - f_0, mu_N = f_{N-2}, mu_i = rho_{i-1} (bump on [t_{i-2}, t_i]),
 *   falling flanks 1 - f(x) evaluated as f(-x),
 *   f_j(t) = f(2 (t - t_j)/(t_{j+1}-t_j) - 1). Causal: mu(s) = 0 for s < 0. */
static void mu_eval(const orc_t *P, int ib, double s, double out[3])
{
    const double *t = P->t;
    int64_t N = P->N;
    out[0] = out[1] = out[2] = 0.0;
    if (s < 0.0) return;
    double f[3];
    if (ib == 0) {
        if (s >= t[1]) return;
        double h = t[1] - t[0];
        /* 1 - f(x) = f(-x) (erf is odd): no cancellation near the top */
        step_f(P->basis_kind, -(2.0 * (s - t[0]) / h - 1.0), f);
        out[0] = f[0];
        out[1] = -f[1] * (2.0 / h);
        out[2] = f[2] * (4.0 / (h * h));
        return;
    }
    if (ib == N - 1) {
        if (s <= t[N - 2]) return;
        if (s >= t[N - 1]) { out[0] = 1.0; return; }
        double h = t[N - 1] - t[N - 2];
        step_f(P->basis_kind, 2.0 * (s - t[N - 2]) / h - 1.0, f);
        out[0] = f[0];
        out[1] = f[1] * (2.0 / h);
        out[2] = f[2] * (4.0 / (h * h));
        return;
    }
    if (s <= t[ib - 1] || s >= t[ib + 1]) return;
    if (s <= t[ib]) {
        double h = t[ib] - t[ib - 1];
        step_f(P->basis_kind, 2.0 * (s - t[ib - 1]) / h - 1.0, f);
        out[0] = f[0];
        out[1] = f[1] * (2.0 / h);
        out[2] = f[2] * (4.0 / (h * h));
    } else {
        double h = t[ib + 1] - t[ib];
        step_f(P->basis_kind, -(2.0 * (s - t[ib]) / h - 1.0), f);
        out[0] = f[0];
        out[1] = -f[1] * (2.0 / h);
        out[2] = f[2] * (4.0 / (h * h));
    }
}

/* basis b_{i,m} = mu_i * (Legendre factor) and derivatives (Eq. BasisFunctions) */
static void basis_eval(const orc_t *P, int ib, int m, double s, double out[3])
{
    double mu[3], L[3], Pm[3];
    mu_eval(P, ib, s, mu);
    if (mu[0] == 0.0 && mu[1] == 0.0 && mu[2] == 0.0) { out[0] = out[1] = out[2] = 0.0; return; }
    const double *t = P->t;
    int64_t N = P->N;
    if (ib == 0) {
        double h = t[1] - t[0];
        if (P->first_kind == 1) {
            out[0] = mu[0]; out[1] = mu[1]; out[2] = mu[2];
            return;
        }
        /* 8 (s/h)^2 P_m(2 s/h - 1) */
        legendre(m, 2.0 * s / h - 1.0, Pm);
        double q = s / h;
        double g0 = 8.0 * q * q, g1 = 16.0 * q / h, g2 = 16.0 / (h * h);
        L[0] = g0 * Pm[0];
        L[1] = g1 * Pm[0] + g0 * Pm[1] * (2.0 / h);
        L[2] = g2 * Pm[0] + 2.0 * g1 * Pm[1] * (2.0 / h) + g0 * Pm[2] * (4.0 / (h * h));
    } else if (ib == N - 1) {
        double h = t[N - 1] - t[N - 2];
        legendre(m, 2.0 * (s - t[N - 2]) / h - 1.0, Pm);
        L[0] = Pm[0]; L[1] = Pm[1] * (2.0 / h); L[2] = Pm[2] * (4.0 / (h * h));
    } else {
        double h2 = t[ib + 1] - t[ib - 1];
        legendre(m, 2.0 * (s - t[ib - 1]) / h2 - 1.0, Pm);
        L[0] = Pm[0]; L[1] = Pm[1] * (2.0 / h2); L[2] = Pm[2] * (4.0 / (h2 * h2));
    }
    out[0] = mu[0] * L[0];
    out[1] = mu[1] * L[0] + mu[0] * L[1];
    out[2] = mu[2] * L[0] + 2.0 * mu[1] * L[1] + mu[0] * L[2];
}

/* ------------------------------------------------------------------------ */
/* psi, psi~ by direct 1-D quadrature (Eq. psis), split at all breakpoints  */
/* ------------------------------------------------------------------------ */
static int cmp_dbl(const void *a, const void *b)
{
    double x = *(const double *)a, y = *(const double *)b;
    return (x > y) - (x < y);
}

static void psi_direct(const orc_t *P, int kb, int m2, int ib, int m1, double r, double out[2])
{
    out[0] = out[1] = 0.0;
    double TL = tl(P, kb), TR = tr(P, kb);
    double SL = tl(P, ib) + r, SR = tr(P, ib) + r;
    double lo = TL > SL ? TL : SL;
    double hi = TR < SR ? TR : SR;
    if (!(lo < hi)) return;
    double pts[8];
    int np = 0;
    pts[np++] = lo;
    pts[np++] = hi;
    double cand[2];
    int nc = 0;
    if (kb > 0 && kb < P->N - 1) cand[nc++] = P->t[kb];
    if (ib > 0 && ib < P->N - 1) cand[nc++] = P->t[ib] + r;
    for (int c = 0; c < nc; ++c)
        if (cand[c] > lo && cand[c] < hi) pts[np++] = cand[c];
    qsort(pts, np, sizeof(double), cmp_dbl);
    double s0 = 0.0, s1 = 0.0;
    for (int seg = 0; seg + 1 < np; ++seg) {
        double a = pts[seg], b = pts[seg + 1];
        if (!(b > a)) continue;
        double hsub = (b - a) / P->gl_sub;
        for (int q = 0; q < P->gl_sub; ++q) {
            double a0 = a + q * hsub;
            for (int g = 0; g < P->gl_n; ++g) {
                double tt = a0 + hsub * P->gl_x[g];
                double wt = hsub * P->gl_w[g];
                double bk[3], bi[3];
                basis_eval(P, kb, m2, tt, bk);
                basis_eval(P, ib, m1, tt - r, bi);
                s0 += wt * bi[2] * bk[1];
                s1 += wt * bi[0] * bk[1];
            }
        }
    }
    out[0] = s0;
    out[1] = s1;
}

/* support of psi_{k,i} on r >= 0 (Sec. 3.2) */
static void block_support(const orc_t *P, int kb, int ib, double *a, double *b)
{
    double lo = tl(P, kb) - tr(P, ib);
    *a = lo > 0.0 ? lo : 0.0;
    *b = tr(P, kb) - tl(P, ib);
}

/* ------------------------------------------------------------------------ */
/* The oracle's own interpolant of psi (fast mode): barycentric Lagrange     */
/* interpolation at Chebyshev points of the second kind on sub-panels of    */
/* the pieces between breakpoints t_{k~-a} - t_{i~-b} of psi in r.          */
/* ------------------------------------------------------------------------ */
static void interp_build(const orc_t *P, int64_t blk, or_interp *I)
{
    int kb = P->bk[blk], ib = P->bi[blk], m2 = P->bm2[blk], m1 = P->bm1[blk];
    double a, b;
    block_support(P, kb, ib, &a, &b);
    double tk[3] = {tl(P, kb), (kb > 0 && kb < P->N - 1) ? P->t[kb] : tl(P, kb), tr(P, kb)};
    double ti[3] = {tl(P, ib), (ib > 0 && ib < P->N - 1) ? P->t[ib] : tl(P, ib), tr(P, ib)};
    double br[12];
    int nbr = 0;
    br[nbr++] = a;
    br[nbr++] = b;
    for (int x = 0; x < 3; ++x)
        for (int y = 0; y < 3; ++y) {
            double d = tk[x] - ti[y];
            if (d > a && d < b) br[nbr++] = d;
        }
    qsort(br, nbr, sizeof(double), cmp_dbl);
    double uniq[12];
    int nu = 0;
    for (int q = 0; q < nbr; ++q)
        if (nu == 0 || br[q] > uniq[nu - 1] + 1e-14 * (1.0 + fabs(br[q]))) uniq[nu++] = br[q];
    I->nb = nu - 1;
    I->S = P->interp_S;
    I->n = P->interp_n;
    I->nsub = I->nb * I->S;
    I->edge = (double *)malloc(sizeof(double) * (I->nsub + 1));
    I->val = (double *)malloc(sizeof(double) * I->nsub * (I->n + 1) * 2);
    for (int64_t pnl = 0; pnl < I->nb; ++pnl) {
        double pa = uniq[pnl], pb = uniq[pnl + 1];
        for (int s = 0; s < I->S; ++s) I->edge[pnl * I->S + s] = pa + (pb - pa) * s / I->S;
    }
    I->edge[I->nsub] = uniq[nu - 1];
    for (int64_t s = 0; s < I->nsub; ++s) {
        double ea = I->edge[s], eb = I->edge[s + 1];
        for (int j = 0; j <= I->n; ++j) {
            double xj = cos(OR_PI * j / I->n);   /* from +1 down to -1 */
            double rr = 0.5 * (ea + eb) + 0.5 * (eb - ea) * xj;
            double v[2];
            psi_direct(P, kb, m2, ib, m1, rr, v);
            I->val[(s * (I->n + 1) + j) * 2 + 0] = v[0];
            I->val[(s * (I->n + 1) + j) * 2 + 1] = v[1];
        }
    }
}

static void interp_eval(const or_interp *I, double r, double out[2])
{
    out[0] = out[1] = 0.0;
    if (!(r > I->edge[0] && r < I->edge[I->nsub])) return;
    int64_t lo = 0, hi = I->nsub;
    while (hi - lo > 1) {
        int64_t mid = (lo + hi) / 2;
        if (I->edge[mid] <= r) lo = mid; else hi = mid;
    }
    double ea = I->edge[lo], eb = I->edge[lo + 1];
    double x = (2.0 * r - ea - eb) / (eb - ea);
    const double *v = I->val + lo * (I->n + 1) * 2;
    double num0 = 0.0, num1 = 0.0, den = 0.0;
    for (int j = 0; j <= I->n; ++j) {
        double xj = cos(OR_PI * j / I->n);
        double d = x - xj;
        if (d == 0.0) { out[0] = v[2 * j]; out[1] = v[2 * j + 1]; return; }
        double wj = (j & 1) ? -1.0 : 1.0;
        if (j == 0 || j == I->n) wj *= 0.5;
        wj /= d;
        num0 += wj * v[2 * j];
        num1 += wj * v[2 * j + 1];
        den += wj;
    }
    out[0] = num0 / den;
    out[1] = num1 / den;
}

static void psi_block(const orc_t *P, int64_t blk, double r, double out[2])
{
    if (P->psi_mode == 1) interp_eval(&P->interp[blk], r, out);
    else psi_direct(P, P->bk[blk], P->bm2[blk], P->bi[blk], P->bm1[blk], r, out);
}

/* ------------------------------------------------------------------------ */
/* Geometry                                                                  */
/* ------------------------------------------------------------------------ */
static void sub3(const double *a, const double *b, double *o) { o[0] = a[0] - b[0]; o[1] = a[1] - b[1]; o[2] = a[2] - b[2]; }
static double dot3(const double *a, const double *b) { return a[0] * b[0] + a[1] * b[1] + a[2] * b[2]; }
static void cross3(const double *a, const double *b, double *o)
{
    o[0] = a[1] * b[2] - a[2] * b[1];
    o[1] = a[2] * b[0] - a[0] * b[2];
    o[2] = a[0] * b[1] - a[1] * b[0];
}

/* per triangle: unit normal, area and surface curls of the three hat
 * functions. The surface gradient is J G^{-1} grad_(u,v) for the
 * parametrisation x = P0 + u (P1-P0) + v (P2-P0), G = J^T J; the surface
 * curl is n x grad (Sec. 2). */
static void triangle_geometry(orc_t *P)
{
    for (int64_t e = 0; e < P->E; ++e) {
        const double *p0 = P->V + 3 * P->F[3 * e], *p1 = P->V + 3 * P->F[3 * e + 1], *p2 = P->V + 3 * P->F[3 * e + 2];
        double e1[3], e2[3], c[3];
        sub3(p1, p0, e1);
        sub3(p2, p0, e2);
        cross3(e1, e2, c);
        double len = sqrt(dot3(c, c));
        double *n = P->nrm + 3 * e;
        n[0] = c[0] / len; n[1] = c[1] / len; n[2] = c[2] / len;
        P->area[e] = 0.5 * len;
        double g11 = dot3(e1, e1), g12 = dot3(e1, e2), g22 = dot3(e2, e2);
        double det = g11 * g22 - g12 * g12;
        double i11 = g22 / det, i12 = -g12 / det, i22 = g11 / det;
        double gr[3][3];
        for (int d = 0; d < 3; ++d) {
            gr[1][d] = i11 * e1[d] + i12 * e2[d];
            gr[2][d] = i12 * e1[d] + i22 * e2[d];
            gr[0][d] = -gr[1][d] - gr[2][d];
        }
        for (int a = 0; a < 3; ++a) cross3(n, gr[a], P->curl + 9 * e + 3 * a);
    }
}

/* distance from point x to segment [a,b] */
static double pt_seg_dist2(const double *x, const double *a, const double *b)
{
    double ab[3], ax[3];
    sub3(b, a, ab);
    sub3(x, a, ax);
    double l2 = dot3(ab, ab);
    double s = l2 > 0.0 ? dot3(ax, ab) / l2 : 0.0;
    if (s < 0.0) s = 0.0;
    if (s > 1.0) s = 1.0;
    double d[3] = {ax[0] - s * ab[0], ax[1] - s * ab[1], ax[2] - s * ab[2]};
    return dot3(d, d);
}

/* squared distance between segments [p,p+d1] and [q,q+d2]: the minimum of
 * |p + s d1 - q - u d2|^2 over [0,1]^2 is at the interior critical point or
 * on one of the four sides of the square. */
static double seg_seg_dist2(const double *p0, const double *p1, const double *q0, const double *q1)
{
    double best = pt_seg_dist2(p0, q0, q1);
    double v = pt_seg_dist2(p1, q0, q1); if (v < best) best = v;
    v = pt_seg_dist2(q0, p0, p1); if (v < best) best = v;
    v = pt_seg_dist2(q1, p0, p1); if (v < best) best = v;
    double d1[3], d2[3], w[3];
    sub3(p1, p0, d1);
    sub3(q1, q0, d2);
    sub3(p0, q0, w);
    double a = dot3(d1, d1), b = dot3(d1, d2), c = dot3(d2, d2), d = dot3(d1, w), e = dot3(d2, w);
    double den = a * c - b * b;
    if (den > 1e-300 * (a * c + 1e-300)) {
        double s = (b * e - c * d) / den, u = (a * e - b * d) / den;
        if (s > 0.0 && s < 1.0 && u > 0.0 && u < 1.0) {
            double diff[3] = {w[0] + s * d1[0] - u * d2[0], w[1] + s * d1[1] - u * d2[1], w[2] + s * d1[2] - u * d2[2]};
            v = dot3(diff, diff);
            if (v < best) best = v;
        }
    }
    return best;
}

/* squared distance from point x to triangle (a,b,c): projection onto the
 * plane if it falls inside, else the nearest edge */
static double pt_tri_dist2(const double *x, const double *a, const double *b, const double *c)
{
    double e1[3], e2[3], n[3], ax[3];
    sub3(b, a, e1);
    sub3(c, a, e2);
    cross3(e1, e2, n);
    sub3(x, a, ax);
    double g11 = dot3(e1, e1), g12 = dot3(e1, e2), g22 = dot3(e2, e2);
    double r1 = dot3(ax, e1), r2 = dot3(ax, e2);
    double det = g11 * g22 - g12 * g12;
    double u = (g22 * r1 - g12 * r2) / det, v = (g11 * r2 - g12 * r1) / det;
    if (u >= 0.0 && v >= 0.0 && u + v <= 1.0) {
        double nn = dot3(n, n);
        double h = dot3(ax, n);
        return h * h / nn;
    }
    double best = pt_seg_dist2(x, a, b);
    double q = pt_seg_dist2(x, b, c); if (q < best) best = q;
    q = pt_seg_dist2(x, c, a); if (q < best) best = q;
    return best;
}

static int shared_vertices(const int32_t *A, const int32_t *B)
{
    int s = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) s += (A[i] == B[j]);
    return s;
}

/* exact minimum and maximum distance between two triangles: 0 if they share
 * a vertex; otherwise the minimum over 6 point-triangle and 9 segment-segment
 * distances (disjoint triangles). The maximum is attained at vertices. */
static void tri_tri_bounds(const orc_t *P, int64_t s, int64_t q, double *dmin, double *dmax)
{
    const int32_t *A = P->F + 3 * s, *B = P->F + 3 * q;
    double mx = 0.0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double d[3];
            sub3(P->V + 3 * A[i], P->V + 3 * B[j], d);
            double v = dot3(d, d);
            if (v > mx) mx = v;
        }
    *dmax = sqrt(mx);
    if (shared_vertices(A, B) > 0) { *dmin = 0.0; return; }
    const double *a[3] = {P->V + 3 * A[0], P->V + 3 * A[1], P->V + 3 * A[2]};
    const double *b[3] = {P->V + 3 * B[0], P->V + 3 * B[1], P->V + 3 * B[2]};
    double best = 1e300;
    for (int i = 0; i < 3; ++i) {
        double v = pt_tri_dist2(a[i], b[0], b[1], b[2]); if (v < best) best = v;
        v = pt_tri_dist2(b[i], a[0], a[1], a[2]); if (v < best) best = v;
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            double v = seg_seg_dist2(a[i], a[(i + 1) % 3], b[j], b[(j + 1) % 3]);
            if (v < best) best = v;
        }
    *dmin = sqrt(best);
}

/* ------------------------------------------------------------------------ */
/* Quadrature rules                                                          */
/* ------------------------------------------------------------------------ */
/* Radon's 7-point degree-5 rule on a triangle: barycentric points, weights
 * summing to 1 (centroid 9/40; two orbits of three points with coordinates
 * (6 -+ sqrt15)/21 and (9 +- 2 sqrt15)/21, weights (155 -+ sqrt15)/1200). */
static void rule7(double bary[7][3], double w[7])
{
    double s = sqrt(15.0);
    double a1 = (6.0 - s) / 21.0, b1 = (9.0 + 2.0 * s) / 21.0, w1 = (155.0 - s) / 1200.0;
    double a2 = (6.0 + s) / 21.0, b2 = (9.0 - 2.0 * s) / 21.0, w2 = (155.0 + s) / 1200.0;
    double B[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3},
                      {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                      {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
    double W[7] = {9.0 / 40.0, w1, w1, w1, w2, w2, w2};
    memcpy(bary, B, sizeof(B));
    memcpy(w, W, sizeof(W));
}

/* Collapsed (Duffy) Gauss product rule with n points per direction on a
 * triangle, used only for brute-force reference values:
 * (u,v) in [0,1]^2 -> barycentric (1-u, u(1-v), uv), weight 2 u w_u w_v
 * (normalised so the weights sum to 1). */
static int rule_product(int n, double *bary, double *w)
{
    double *x = (double *)malloc(sizeof(double) * n), *wx = (double *)malloc(sizeof(double) * n);
    gauss_legendre01(n, x, wx);
    int k = 0;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) {
            double u = x[i], v = x[j];
            bary[3 * k + 0] = 1.0 - u;
            bary[3 * k + 1] = u * (1.0 - v);
            bary[3 * k + 2] = u * v;
            w[k] = 2.0 * u * wx[i] * wx[j];
            ++k;
        }
    free(x);
    free(wx);
    return k;
}

/* Sauter-Schwab maps (Sec. 5.2 of Sauter & Schwab) on the reference triangle
 * {0 <= x2 <= x1 <= 1}; (xi, e1, e2, e3) in [0,1]^4. Returns the number of
 * regions; xh/yh receive the reference points, jac the region Jacobian.
 * case 3: identical triangles, 2: common edge x2 = 0 (from (0,0) to (1,0)),
 * 1: common vertex (0,0). */
static int ss_points(int kase, double xi, double e1, double e2, double e3,
                     double xh[6][2], double yh[6][2], double jac[6])
{
    if (kase == 3) {
        double w = xi * xi * xi * e1 * e1 * e2;
        xh[0][0] = xi;                    xh[0][1] = xi * (1 - e1 + e1 * e2);
        yh[0][0] = xi * (1 - e1 * e2 * e3); yh[0][1] = xi * (1 - e1);
        xh[1][0] = yh[0][0]; xh[1][1] = yh[0][1];
        yh[1][0] = xh[0][0]; yh[1][1] = xh[0][1];
        xh[2][0] = xi;                    xh[2][1] = xi * e1 * (1 - e2 + e2 * e3);
        yh[2][0] = xi * (1 - e1 * e2);    yh[2][1] = xi * e1 * (1 - e2);
        xh[3][0] = yh[2][0]; xh[3][1] = yh[2][1];
        yh[3][0] = xh[2][0]; yh[3][1] = xh[2][1];
        xh[4][0] = xi * (1 - e1 * e2 * e3); xh[4][1] = xi * e1 * (1 - e2 * e3);
        yh[4][0] = xi;                    yh[4][1] = xi * e1 * (1 - e2);
        xh[5][0] = yh[4][0]; xh[5][1] = yh[4][1];
        yh[5][0] = xh[4][0]; yh[5][1] = xh[4][1];
        for (int k = 0; k < 6; ++k) jac[k] = w;
        return 6;
    }
    if (kase == 2) {
        double w0 = xi * xi * xi * e1 * e1, w = w0 * e2;
        xh[0][0] = xi;                        xh[0][1] = xi * e1 * e3;
        yh[0][0] = xi * (1 - e1 * e2);        yh[0][1] = xi * e1 * (1 - e2);
        jac[0] = w0;
        xh[1][0] = xi;                        xh[1][1] = xi * e1;
        yh[1][0] = xi * (1 - e1 * e2 * e3);   yh[1][1] = xi * e1 * e2 * (1 - e3);
        jac[1] = w;
        xh[2][0] = xi * (1 - e1 * e2);        xh[2][1] = xi * e1 * (1 - e2);
        yh[2][0] = xi;                        yh[2][1] = xi * e1 * e2 * e3;
        jac[2] = w;
        xh[3][0] = xi * (1 - e1 * e2 * e3);   xh[3][1] = xi * e1 * e2 * (1 - e3);
        yh[3][0] = xi;                        yh[3][1] = xi * e1;
        jac[3] = w;
        xh[4][0] = xi * (1 - e1 * e2 * e3);   xh[4][1] = xi * e1 * (1 - e2 * e3);
        yh[4][0] = xi;                        yh[4][1] = xi * e1 * e2;
        jac[4] = w;
        return 5;
    }
    {
        double w = xi * xi * xi * e2;
        xh[0][0] = xi;           xh[0][1] = xi * e1;
        yh[0][0] = xi * e2;      yh[0][1] = xi * e2 * e3;
        xh[1][0] = yh[0][0]; xh[1][1] = yh[0][1];
        yh[1][0] = xh[0][0]; yh[1][1] = xh[0][1];
        jac[0] = jac[1] = w;
        return 2;
    }
}

/* ------------------------------------------------------------------------ */
/* Element-pair local matrices (Eq. MatrixEntries)                          */
/* L[blk][a][b] += for test corner a of s, trial corner b of q.             */
/* far_n == 0: 7-point rule; far_n > 0: collapsed Gauss product (reference) */
/* ------------------------------------------------------------------------ */
typedef struct {
    int n;
    double *bary, *w;
} tri_rule;

static void pair_far(const orc_t *P, int64_t s, int64_t q, const tri_rule *R,
                     const int64_t *blks, int nb, double *L /* nb*9 */)
{
    const int32_t *A = P->F + 3 * s, *B = P->F + 3 * q;
    double nn = dot3(P->nrm + 3 * s, P->nrm + 3 * q);
    double cc[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cc[a][b] = dot3(P->curl + 9 * s + 3 * a, P->curl + 9 * q + 3 * b);
    double scale = P->area[s] * P->area[q] / (4.0 * OR_PI);
    for (int i = 0; i < R->n; ++i) {
        const double *bx = R->bary + 3 * i;
        double x[3];
        for (int d = 0; d < 3; ++d) x[d] = bx[0] * P->V[3 * A[0] + d] + bx[1] * P->V[3 * A[1] + d] + bx[2] * P->V[3 * A[2] + d];
        for (int j = 0; j < R->n; ++j) {
            const double *by = R->bary + 3 * j;
            double y[3];
            for (int d = 0; d < 3; ++d) y[d] = by[0] * P->V[3 * B[0] + d] + by[1] * P->V[3 * B[1] + d] + by[2] * P->V[3 * B[2] + d];
            double dxy[3];
            sub3(x, y, dxy);
            double r = sqrt(dot3(dxy, dxy));
            double wgt = R->w[i] * R->w[j] * scale / r;
            for (int k = 0; k < nb; ++k) {
                double ps[2];
                psi_block(P, blks[k], r, ps);
                if (ps[0] == 0.0 && ps[1] == 0.0) continue;
                double *Lk = L + 9 * k;
                for (int a = 0; a < 3; ++a)
                    for (int b = 0; b < 3; ++b)
                        Lk[3 * a + b] += wgt * (nn * bx[a] * by[b] * ps[0] + cc[a][b] * ps[1]);
            }
        }
    }
}

/* near pair by Sauter-Schwab with n Gauss points per direction */
static void pair_near(const orc_t *P, int64_t s, int64_t q, int n, const double *gx, const double *gw,
                      const int64_t *blks, int nb, double *L)
{
    const int32_t *A = P->F + 3 * s, *B = P->F + 3 * q;
    int kase = shared_vertices(A, B);
    /* reorder corners: permA[slot] = corner of s placed at reference vertex slot */
    int pa[3] = {0, 1, 2}, pb[3] = {0, 1, 2};
    if (kase == 2) {
        /* shared edge (u,v): s = (u, v, w), q = (u, v, z) */
        int sh[2], k = 0;
        for (int i = 0; i < 3 && k < 2; ++i)
            for (int j = 0; j < 3; ++j)
                if (A[i] == B[j]) { sh[k++] = i; break; }
        int u = sh[0], v = sh[1];
        int wcor = 3 - u - v;
        pa[0] = u; pa[1] = v; pa[2] = wcor;
        int ub = -1, vb = -1;
        for (int j = 0; j < 3; ++j) { if (B[j] == A[u]) ub = j; if (B[j] == A[v]) vb = j; }
        pb[0] = ub; pb[1] = vb; pb[2] = 3 - ub - vb;
    } else if (kase == 1) {
        int ia = -1, jb = -1;
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j)
                if (A[i] == B[j]) { ia = i; jb = j; }
        pa[0] = ia; pa[1] = (ia + 1) % 3; pa[2] = (ia + 2) % 3;
        pb[0] = jb; pb[1] = (jb + 1) % 3; pb[2] = (jb + 2) % 3;
    }
    const double *X0 = P->V + 3 * A[pa[0]], *X1 = P->V + 3 * A[pa[1]], *X2 = P->V + 3 * A[pa[2]];
    const double *Y0 = P->V + 3 * B[pb[0]], *Y1 = P->V + 3 * B[pb[1]], *Y2 = P->V + 3 * B[pb[2]];
    double ex1[3], ex2[3], ey1[3], ey2[3], d0[3];
    sub3(X1, X0, ex1); sub3(X2, X1, ex2);
    sub3(Y1, Y0, ey1); sub3(Y2, Y1, ey2);
    sub3(X0, Y0, d0);
    double nn = dot3(P->nrm + 3 * s, P->nrm + 3 * q);
    double cc[3][3];
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) cc[a][b] = dot3(P->curl + 9 * s + 3 * a, P->curl + 9 * q + 3 * b);
    /* reference triangle has area 1/2: |J| = 2|T| */
    double scale = (2.0 * P->area[s]) * (2.0 * P->area[q]) / (4.0 * OR_PI);
    for (int i0 = 0; i0 < n; ++i0)
        for (int i1 = 0; i1 < n; ++i1)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i3 = 0; i3 < n; ++i3) {
                    double W = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    double xh[6][2], yh[6][2], jac[6];
                    int nr = ss_points(kase, gx[i0], gx[i1], gx[i2], gx[i3], xh, yh, jac);
                    for (int rg = 0; rg < nr; ++rg) {
                        double dxy[3];
                        for (int d = 0; d < 3; ++d)
                            dxy[d] = d0[d] + xh[rg][0] * ex1[d] + xh[rg][1] * ex2[d] - yh[rg][0] * ey1[d] - yh[rg][1] * ey2[d];
                        double r = sqrt(dot3(dxy, dxy));
                        double lx[3] = {1.0 - xh[rg][0], xh[rg][0] - xh[rg][1], xh[rg][1]};
                        double ly[3] = {1.0 - yh[rg][0], yh[rg][0] - yh[rg][1], yh[rg][1]};
                        double wgt = W * jac[rg] * scale / r;
                        for (int k = 0; k < nb; ++k) {
                            double ps[2];
                            psi_block(P, blks[k], r, ps);
                            if (ps[0] == 0.0 && ps[1] == 0.0) continue;
                            double *Lk = L + 9 * k;
                            for (int a = 0; a < 3; ++a)
                                for (int b = 0; b < 3; ++b)
                                    Lk[3 * pa[a] + pb[b]] += wgt * (nn * lx[a] * ly[b] * ps[0] + cc[pa[a]][pb[b]] * ps[1]);
                        }
                    }
                }
}

/* ------------------------------------------------------------------------ */
/* Public API                                                                */
/* ------------------------------------------------------------------------ */
void *or_create(const double *V, int64_t M, const int32_t *F, int64_t E, const double *t, int64_t N,
                int p, int equidistant, int gl_n, int gl_sub, int ss_n, int psi_mode, int interp_S, int interp_n,
                int basis_kind)
{
    orc_t *P = (orc_t *)calloc(1, sizeof(orc_t));
    P->M = M; P->E = E; P->N = N; P->p = p;
    P->V = (double *)malloc(sizeof(double) * 3 * M); memcpy(P->V, V, sizeof(double) * 3 * M);
    P->F = (int32_t *)malloc(sizeof(int32_t) * 3 * E); memcpy(P->F, F, sizeof(int32_t) * 3 * E);
    P->t = (double *)malloc(sizeof(double) * N); memcpy(P->t, t, sizeof(double) * N);
    P->T = t[N - 1];
    P->tie = 1e-12 * P->T;
    P->nrm = (double *)malloc(sizeof(double) * 3 * E);
    P->area = (double *)malloc(sizeof(double) * E);
    P->curl = (double *)malloc(sizeof(double) * 9 * E);
    triangle_geometry(P);
    P->vt_ptr = (int64_t *)calloc(M + 1, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) P->vt_ptr[F[3 * e + a] + 1]++;
    for (int64_t v = 0; v < M; ++v) P->vt_ptr[v + 1] += P->vt_ptr[v];
    P->vt_tri = (int32_t *)malloc(sizeof(int32_t) * 3 * E);
    P->vt_cor = (int32_t *)malloc(sizeof(int32_t) * 3 * E);
    int64_t *fill = (int64_t *)calloc(M, sizeof(int64_t));
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) {
            int32_t v = F[3 * e + a];
            int64_t pos = P->vt_ptr[v] + fill[v]++;
            P->vt_tri[pos] = (int32_t)e;
            P->vt_cor[pos] = a;
        }
    free(fill);
    P->maxval = 0;
    for (int64_t v = 0; v < M; ++v)
        if (P->vt_ptr[v + 1] - P->vt_ptr[v] > P->maxval) P->maxval = (int)(P->vt_ptr[v + 1] - P->vt_ptr[v]);
    P->gl_n = gl_n; P->gl_sub = gl_sub;
    P->gl_x = (double *)malloc(sizeof(double) * gl_n); P->gl_w = (double *)malloc(sizeof(double) * gl_n);
    gauss_legendre01(gl_n, P->gl_x, P->gl_w);
    P->ss_n = ss_n;
    P->ss_x = (double *)malloc(sizeof(double) * ss_n); P->ss_w = (double *)malloc(sizeof(double) * ss_n);
    gauss_legendre01(ss_n, P->ss_x, P->ss_w);
    P->psi_mode = psi_mode; P->interp_S = interp_S; P->interp_n = interp_n;
    P->basis_kind = basis_kind;
    /* diameter = max vertex distance */
    double dm = 0.0;
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = i + 1; j < M; ++j) {
            double d[3];
            sub3(P->V + 3 * i, P->V + 3 * j, d);
            double v = dot3(d, d);
            if (v > dm) dm = v;
        }
    P->diam = sqrt(dm);
    /* unique blocks: equidistant -> first two columns, last row, (2,3),
     * (N-1,N) (Sec. 5.1); graded -> every (k~,i~) with i~ <= k~+1.
     * Blocks whose support starts at or beyond diam(Gamma) are zero (Sec. 3.2). */
    int64_t cap = N * N * (p + 1) * (p + 1);
    P->bk = (int32_t *)malloc(sizeof(int32_t) * cap); P->bi = (int32_t *)malloc(sizeof(int32_t) * cap);
    P->bm2 = (int32_t *)malloc(sizeof(int32_t) * cap); P->bm1 = (int32_t *)malloc(sizeof(int32_t) * cap);
    char *want = (char *)calloc(N * N, 1);
    if (equidistant) {
        for (int64_t k = 0; k < N; ++k) { want[k * N + 0] = 1; if (N > 1) want[k * N + 1] = 1; }
        for (int64_t i = 0; i < N; ++i) want[(N - 1) * N + i] = 1;
        if (N > 2) want[1 * N + 2] = 1;
        if (N > 2) want[(N - 2) * N + (N - 1)] = 1;
    } else {
        for (int64_t k = 0; k < N; ++k)
            for (int64_t i = 0; i < N && i <= k + 1; ++i) want[k * N + i] = 1;
    }
    P->nblk = 0;
    for (int64_t k = 0; k < N; ++k)
        for (int64_t i = 0; i < N; ++i) {
            if (!want[k * N + i]) continue;
            if (i > k + 1) continue;  /* block Hessenberg zeros (Eq. Apartitioned) */
            double a, b;
            block_support(P, (int)k, (int)i, &a, &b);
            if (!(b > a)) continue;
            if (a >= P->diam - P->tie) continue;
            for (int m2 = 0; m2 <= p; ++m2)
                for (int m1 = 0; m1 <= p; ++m1) {
                    P->bk[P->nblk] = (int32_t)k; P->bi[P->nblk] = (int32_t)i;
                    P->bm2[P->nblk] = m2; P->bm1[P->nblk] = m1;
                    P->nblk++;
                }
        }
    free(want);
    P->interp = NULL;
    if (psi_mode == 1) {
        P->interp = (or_interp *)calloc(P->nblk, sizeof(or_interp));
#pragma omp parallel for schedule(dynamic)
        for (int64_t b = 0; b < P->nblk; ++b) interp_build(P, b, &P->interp[b]);
    }
    return P;
}

void or_destroy(void *h)
{
    orc_t *P = (orc_t *)h;
    if (!P) return;
    if (P->interp) {
        for (int64_t b = 0; b < P->nblk; ++b) { free(P->interp[b].edge); free(P->interp[b].val); }
        free(P->interp);
    }
    free(P->V); free(P->F); free(P->t); free(P->nrm); free(P->area); free(P->curl);
    free(P->vt_ptr); free(P->vt_tri); free(P->vt_cor); free(P->gl_x); free(P->gl_w);
    free(P->ss_x); free(P->ss_w); free(P->bk); free(P->bi); free(P->bm2); free(P->bm1);
    free(P);
}

int64_t or_num_blocks(void *h) { return ((orc_t *)h)->nblk; }

void or_block(void *h, int64_t b, int32_t *out4, double *ab)
{
    orc_t *P = (orc_t *)h;
    out4[0] = P->bk[b]; out4[1] = P->bi[b]; out4[2] = P->bm2[b]; out4[3] = P->bm1[b];
    block_support(P, P->bk[b], P->bi[b], &ab[0], &ab[1]);
}

double or_diam(void *h) { return ((orc_t *)h)->diam; }

/* unit normal (3), area (1) and the surface curls of the three hat
 * functions (9, corner-major) of triangle e */
void or_tri_geom(void *h, int64_t e, double *out13)
{
    orc_t *P = (orc_t *)h;
    memcpy(out13, P->nrm + 3 * e, sizeof(double) * 3);
    out13[3] = P->area[e];
    memcpy(out13 + 4, P->curl + 9 * e, sizeof(double) * 9);
}

void or_set_first_kind(void *h, int kind) { ((orc_t *)h)->first_kind = kind; }
/* the smooth step of the given kind and its first two derivatives at x */
void or_step(int kind, double x, double *out) { step_f(kind, x, out); }

void or_basis(void *h, int ib, int m, const double *s, int64_t n, double *out /* n*3 */)
{
    orc_t *P = (orc_t *)h;
    for (int64_t k = 0; k < n; ++k) basis_eval(P, ib, m, s[k], out + 3 * k);
}

void or_mu(void *h, int ib, const double *s, int64_t n, double *out)
{
    orc_t *P = (orc_t *)h;
    for (int64_t k = 0; k < n; ++k) mu_eval(P, ib, s[k], out + 3 * k);
}

/* psi / psi~ of test basis (kb,m2) against trial basis (ib,m1); mode 0 direct */
void or_psi(void *h, int kb, int m2, int ib, int m1, const double *r, int64_t n, double *out /* n*2 */)
{
    orc_t *P = (orc_t *)h;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) psi_direct(P, kb, m2, ib, m1, r[k], out + 2 * k);
}

void or_psi_block(void *h, int64_t blk, const double *r, int64_t n, double *out)
{
    orc_t *P = (orc_t *)h;
#pragma omp parallel for schedule(static)
    for (int64_t k = 0; k < n; ++k) psi_block(P, blk, r[k], out + 2 * k);
}

void or_tri_bounds(void *h, int64_t s, int64_t q, double *out2)
{
    tri_tri_bounds((orc_t *)h, s, q, &out2[0], &out2[1]);
}

void or_rule7(double *bary /*21*/, double *w /*7*/)
{
    double B[7][3], W[7];
    rule7(B, W);
    memcpy(bary, B, sizeof(B));
    memcpy(w, W, sizeof(W));
}

/* Sauter-Schwab nodes with n points per direction: returns count; fills
 * xh (cnt*2), yh (cnt*2), w (cnt) with w including Gauss weights and
 * region Jacobian (integrates over T^ x T^, T^ of area 1/2). */
int64_t or_ss_rule(int kase, int n, double *xh, double *yh, double *w)
{
    double *gx = (double *)malloc(sizeof(double) * n), *gw = (double *)malloc(sizeof(double) * n);
    gauss_legendre01(n, gx, gw);
    int64_t c = 0;
    for (int i0 = 0; i0 < n; ++i0)
        for (int i1 = 0; i1 < n; ++i1)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i3 = 0; i3 < n; ++i3) {
                    double X[6][2], Y[6][2], J[6];
                    int nr = ss_points(kase, gx[i0], gx[i1], gx[i2], gx[i3], X, Y, J);
                    for (int rg = 0; rg < nr; ++rg) {
                        if (xh) { xh[2 * c] = X[rg][0]; xh[2 * c + 1] = X[rg][1]; yh[2 * c] = Y[rg][0]; yh[2 * c + 1] = Y[rg][1]; w[c] = gw[i0] * gw[i1] * gw[i2] * gw[i3] * J[rg]; }
                        ++c;
                    }
                }
    free(gx); free(gw);
    return c;
}

void or_gauss_legendre(int n, double *x, double *w) { gauss_legendre01(n, x, w); }

/* local 3x3 matrices of one element pair for a list of blocks.
 * far_n: 0 = production 7-point rule, >0 collapsed Gauss product with far_n
 * points per direction; near_n: Sauter-Schwab points per direction (0 = the
 * problem's default). Pairs sharing a vertex always use Sauter-Schwab. */
void or_pair_local(void *h, int64_t s, int64_t q, const int64_t *blks, int nb, int far_n, int near_n, double *L)
{
    orc_t *P = (orc_t *)h;
    memset(L, 0, sizeof(double) * 9 * nb);
    if (shared_vertices(P->F + 3 * s, P->F + 3 * q) > 0) {
        int n = near_n > 0 ? near_n : P->ss_n;
        double *gx = (double *)malloc(sizeof(double) * n), *gw = (double *)malloc(sizeof(double) * n);
        gauss_legendre01(n, gx, gw);
        pair_near(P, s, q, n, gx, gw, blks, nb, L);
        free(gx); free(gw);
    } else {
        tri_rule R;
        if (far_n <= 0) {
            double B[7][3], W[7];
            rule7(B, W);
            R.n = 7;
            R.bary = (double *)malloc(sizeof(double) * 21); R.w = (double *)malloc(sizeof(double) * 7);
            memcpy(R.bary, B, sizeof(B)); memcpy(R.w, W, sizeof(W));
        } else {
            R.n = far_n * far_n;
            R.bary = (double *)malloc(sizeof(double) * 3 * R.n); R.w = (double *)malloc(sizeof(double) * R.n);
            rule_product(far_n, R.bary, R.w);
        }
        pair_far(P, s, q, &R, blks, nb, L);
        free(R.bary); free(R.w);
    }
}

/* per-row work: distances from the triangles of row l to every triangle */
typedef struct {
    double *m, *Mx;   /* per trial triangle: min dmin / max dmax over test triangles of l */
    double *dmin, *dmax; /* per (test triangle of l, trial triangle) */
} rowscratch;

static int row_tris(const orc_t *P, int64_t l) { return (int)(P->vt_ptr[l + 1] - P->vt_ptr[l]); }

static void row_bounds(const orc_t *P, int64_t l, rowscratch *S)
{
    int nt = row_tris(P, l);
    for (int64_t q = 0; q < P->E; ++q) {
        double mn = 1e300, mx = 0.0;
        for (int k = 0; k < nt; ++k) {
            int64_t s = P->vt_tri[P->vt_ptr[l] + k];
            double a, b;
            tri_tri_bounds(P, s, q, &a, &b);
            S->dmin[k * P->E + q] = a;
            S->dmax[k * P->E + q] = b;
            if (a < mn) mn = a;
            if (b > mx) mx = b;
        }
        S->m[q] = mn;
        S->Mx[q] = mx;
    }
}

/* column pattern of row l in block blk: mindist/maxdist over the supports of
 * phi_l and phi_j (Eq. SparsitySmallBlock), open support endpoints */
static int64_t row_pattern(const orc_t *P, int64_t blk, const rowscratch *S, const double *mind, const double *maxd, int32_t *cols)
{
    double a, b;
    block_support(P, P->bk[blk], P->bi[blk], &a, &b);
    int64_t c = 0;
    for (int64_t j = 0; j < P->M; ++j)
        if (mind[j] < b - P->tie && maxd[j] > a + P->tie) { if (cols) cols[c] = (int32_t)j; ++c; }
    (void)S;
    return c;
}

static void vertex_bounds(const orc_t *P, const rowscratch *S, double *mind, double *maxd)
{
    for (int64_t j = 0; j < P->M; ++j) {
        double mn = 1e300, mx = 0.0;
        for (int64_t k = P->vt_ptr[j]; k < P->vt_ptr[j + 1]; ++k) {
            int64_t q = P->vt_tri[k];
            if (S->m[q] < mn) mn = S->m[q];
            if (S->Mx[q] > mx) mx = S->Mx[q];
        }
        mind[j] = mn;
        maxd[j] = mx;
    }
}

/* pattern counts for rows x blocks: counts[b*nrows + r] */
void or_pattern_counts(void *h, const int64_t *rows, int64_t nrows, const int64_t *blks, int64_t nb, int64_t *counts)
{
    orc_t *P = (orc_t *)h;
#pragma omp parallel
    {
        rowscratch S;
        S.m = (double *)malloc(sizeof(double) * P->E);
        S.Mx = (double *)malloc(sizeof(double) * P->E);
        S.dmin = (double *)malloc(sizeof(double) * P->E * P->maxval);
        S.dmax = (double *)malloc(sizeof(double) * P->E * P->maxval);
        double *mind = (double *)malloc(sizeof(double) * P->M), *maxd = (double *)malloc(sizeof(double) * P->M);
#pragma omp for schedule(dynamic)
        for (int64_t r = 0; r < nrows; ++r) {
            row_bounds(P, rows[r], &S);
            vertex_bounds(P, &S, mind, maxd);
            for (int64_t b = 0; b < nb; ++b) counts[b * nrows + r] = row_pattern(P, blks[b], &S, mind, maxd, NULL);
        }
        free(S.m); free(S.Mx); free(S.dmin); free(S.dmax); free(mind); free(maxd);
    }
}

/* Pattern fingerprint of rows x blocks: per block, the number of structural
 * entries and the sum mod 2^64 of splitmix64(l M + j) over its entries (l, j)
 * in the given rows -- the output function of Steele, Lea and Flood's
 * SplitMix64 as published. A sum does not depend on the order of the rows or
 * threads, and two patterns with the same count and sum are the same pattern
 * but for a 2^-64 coincidence. */
static uint64_t splitmix64_out(uint64_t z)
{
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

void or_pattern_hash(void *h, const int64_t *rows, int64_t nrows, const int64_t *blks, int64_t nb, uint64_t *hash,
                     int64_t *nnz)
{
    orc_t *P = (orc_t *)h;
    for (int64_t b = 0; b < nb; ++b) { hash[b] = 0; nnz[b] = 0; }
#pragma omp parallel
    {
        rowscratch S;
        S.m = (double *)malloc(sizeof(double) * P->E);
        S.Mx = (double *)malloc(sizeof(double) * P->E);
        S.dmin = (double *)malloc(sizeof(double) * P->E * P->maxval);
        S.dmax = (double *)malloc(sizeof(double) * P->E * P->maxval);
        double *mind = (double *)malloc(sizeof(double) * P->M), *maxd = (double *)malloc(sizeof(double) * P->M);
        int32_t *cols = (int32_t *)malloc(sizeof(int32_t) * P->M);
        uint64_t *hs = (uint64_t *)calloc(nb, sizeof(uint64_t));
        int64_t *ns = (int64_t *)calloc(nb, sizeof(int64_t));
#pragma omp for schedule(dynamic)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t l = rows[r];
            row_bounds(P, l, &S);
            vertex_bounds(P, &S, mind, maxd);
            for (int64_t b = 0; b < nb; ++b) {
                int64_t c = row_pattern(P, blks[b], &S, mind, maxd, cols);
                for (int64_t q = 0; q < c; ++q) hs[b] += splitmix64_out((uint64_t)l * (uint64_t)P->M + (uint64_t)cols[q]);
                ns[b] += c;
            }
        }
#pragma omp critical
        for (int64_t b = 0; b < nb; ++b) { hash[b] += hs[b]; nnz[b] += ns[b]; }
        free(S.m); free(S.Mx); free(S.dmin); free(S.dmax); free(mind); free(maxd); free(cols); free(hs); free(ns);
    }
}

/* assemble rows x blocks. offsets[b*nrows + r] = start of that (block,row)
 * segment in cols/vfar/vnear (lengths from or_pattern_counts). Values are
 * split into the far part (7-point rule on pairs without a shared vertex)
 * and the near part (Sauter-Schwab on pairs sharing a vertex). */
void or_assemble_rows(void *h, const int64_t *rows, int64_t nrows, const int64_t *blks, int64_t nb,
                      const int64_t *offsets, int32_t *cols, double *vfar, double *vnear)
{
    orc_t *P = (orc_t *)h;
    double B7[7][3], W7[7];
    rule7(B7, W7);
    tri_rule R7;
    R7.n = 7;
    R7.bary = &B7[0][0];
    R7.w = W7;
#pragma omp parallel
    {
        rowscratch S;
        S.m = (double *)malloc(sizeof(double) * P->E);
        S.Mx = (double *)malloc(sizeof(double) * P->E);
        S.dmin = (double *)malloc(sizeof(double) * P->E * P->maxval);
        S.dmax = (double *)malloc(sizeof(double) * P->E * P->maxval);
        double *mind = (double *)malloc(sizeof(double) * P->M), *maxd = (double *)malloc(sizeof(double) * P->M);
        double *accf = (double *)malloc(sizeof(double) * P->M * nb);
        double *accn = (double *)malloc(sizeof(double) * P->M * nb);
        double *L = (double *)malloc(sizeof(double) * 9 * nb);
        int64_t *kb = (int64_t *)malloc(sizeof(int64_t) * nb);
        int64_t *kidx = (int64_t *)malloc(sizeof(int64_t) * nb);
        double *ba = (double *)malloc(sizeof(double) * nb), *bb = (double *)malloc(sizeof(double) * nb);
        for (int64_t b = 0; b < nb; ++b) block_support(P, P->bk[blks[b]], P->bi[blks[b]], &ba[b], &bb[b]);
#pragma omp for schedule(dynamic)
        for (int64_t r = 0; r < nrows; ++r) {
            int64_t l = rows[r];
            row_bounds(P, l, &S);
            vertex_bounds(P, &S, mind, maxd);
            memset(accf, 0, sizeof(double) * P->M * nb);
            memset(accn, 0, sizeof(double) * P->M * nb);
            int nt = row_tris(P, l);
            for (int k = 0; k < nt; ++k) {
                int64_t s = P->vt_tri[P->vt_ptr[l] + k];
                int a = P->vt_cor[P->vt_ptr[l] + k];
                for (int64_t q = 0; q < P->E; ++q) {
                    double dmn = S.dmin[k * P->E + q], dmx = S.dmax[k * P->E + q];
                    int nk = 0;
                    for (int64_t b = 0; b < nb; ++b)
                        if (dmn < bb[b] - P->tie && dmx > ba[b] + P->tie) { kb[nk] = blks[b]; kidx[nk] = b; ++nk; }
                    if (nk == 0) continue;
                    memset(L, 0, sizeof(double) * 9 * nk);
                    int near = shared_vertices(P->F + 3 * s, P->F + 3 * q) > 0;
                    if (near) pair_near(P, s, q, P->ss_n, P->ss_x, P->ss_w, kb, nk, L);
                    else pair_far(P, s, q, &R7, kb, nk, L);
                    double *acc = near ? accn : accf;
                    for (int c = 0; c < nk; ++c)
                        for (int bcor = 0; bcor < 3; ++bcor) {
                            int32_t j = P->F[3 * q + bcor];
                            acc[kidx[c] * P->M + j] += L[9 * c + 3 * a + bcor];
                        }
                }
            }
            for (int64_t b = 0; b < nb; ++b) {
                int64_t off = offsets[b * nrows + r];
                int64_t c = row_pattern(P, blks[b], &S, mind, maxd, cols + off);
                for (int64_t e = 0; e < c; ++e) {
                    int32_t j = cols[off + e];
                    vfar[off + e] = accf[b * P->M + j];
                    vnear[off + e] = accn[b * P->M + j];
                }
            }
        }
        free(S.m); free(S.Mx); free(S.dmin); free(S.dmax); free(mind); free(maxd);
        free(accf); free(accn); free(L); free(kb); free(kidx); free(ba); free(bb);
    }
}

int or_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Thread count of later parallel regions (n >= 1); returns the previous
 * count. Only the timing of the oracle uses it (its single-thread rate). */
int or_set_threads(int n)
{
#ifdef _OPENMP
    const int prev = omp_get_max_threads();
    if (n >= 1) omp_set_num_threads(n);
    return prev;
#else
    (void)n;
    return 1;
#endif
}
