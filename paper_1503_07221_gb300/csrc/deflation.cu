// Host side of DGMRES(m, l) (Sec. 4.1): the deflation subspace from the
// cycle's small Hessenberg matrix H_m (m <= 62). The solver keeps the
// invariant subspace of H_m for its eigenvalues of smallest modulus, written
// as V_m times an orthonormal real basis B of that subspace of R^m, and uses
// the largest modulus as the estimate of |lambda_max|.
//
// H_m is brought to complex Schur form H = Z T Z^H (T upper triangular) by
// the shifted QR algorithm on the Hessenberg matrix: explicit single-shift
// steps with Givens rotations on the active window, Wilkinson shifts from the
// trailing 2 x 2 block, an exceptional shift after 10 steps without
// deflation, and deflation where a subdiagonal entry falls below the unit
// roundoff times its diagonal neighbours. The selected eigenvalues (modulus
// at most the l-th smallest modulus, relative slack 1e-12, so both members of
// a complex pair come together) are then moved to the leading positions by
// swaps of adjacent diagonal entries: for t11 = T[k][k], t22 = T[k+1][k+1],
// the rotation G with G (t12, t22 - t11)^T = (r, 0)^T maps the eigenvector of
// t22 onto e_1, so G T G^H holds t22 before t11. The leading sdim columns of
// Z span the selected invariant subspace; it is closed under conjugation (H
// is real), so the real and imaginary parts of those columns span its real
// points, and a modified Gram-Schmidt pass over them gives B.
#include <algorithm>
#include <cfloat>
#include <cmath>
#include <complex>
#include <vector>

#include "tdbem_internal.h"

namespace tdbem {

typedef std::complex<double> cd;

// c real, s complex with [c s; -conj(s) c] (f, g)^T = (r, 0)^T
static void cgivens(cd f, cd g, double &c, cd &s) {
    if (g == cd(0.0)) { c = 1.0; s = 0.0; return; }
    if (f == cd(0.0)) { c = 0.0; s = std::conj(g) / std::abs(g); return; }
    const double fa = std::abs(f), ga = std::abs(g), nrm = std::hypot(fa, ga);
    c = fa / nrm;
    s = (f / fa) * std::conj(g) / nrm;
}

namespace {
struct Cmat {
    int n;
    std::vector<cd> a;
    explicit Cmat(int n_) : n(n_), a((size_t)n_ * n_) {}
    cd &operator()(int i, int j) { return a[(size_t)i * n + j]; }
};
}  // namespace

// rows p = k, q = k + 1 from the left for columns [c0, n); columns k, k + 1
// from the right (by G^H) for rows [0, r1)
static void rot_left(Cmat &T, int k, int c0, double c, cd s) {
    for (int j = c0; j < T.n; ++j) {
        const cd x = T(k, j), y = T(k + 1, j);
        T(k, j) = c * x + s * y;
        T(k + 1, j) = -std::conj(s) * x + c * y;
    }
}
static void rot_right(Cmat &T, int k, int r1, double c, cd s) {
    for (int i = 0; i < r1; ++i) {
        const cd x = T(i, k), y = T(i, k + 1);
        T(i, k) = c * x + std::conj(s) * y;
        T(i, k + 1) = -s * x + c * y;
    }
}

static bool complex_schur(Cmat &T, Cmat &Z) {
    const int n = T.n;
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Z(i, j) = i == j ? 1.0 : 0.0;
    double hn = 0.0;
    for (const cd &v : T.a) hn = std::max(hn, std::abs(v));
    if (hn == 0.0) return true;
    std::vector<double> cs(n);
    std::vector<cd> sn(n);
    int hi = n - 1, its = 0, total = 0;
    while (hi > 0) {
        int lo = hi;
        while (lo > 0) {
            const double nb = std::abs(T(lo - 1, lo - 1)) + std::abs(T(lo, lo));
            if (std::abs(T(lo, lo - 1)) <= DBL_EPSILON * (nb > 0.0 ? nb : hn)) {
                T(lo, lo - 1) = 0.0;
                break;
            }
            --lo;
        }
        if (lo == hi) {
            --hi;
            its = 0;
            continue;
        }
        if (++total > 100 * n) return false;
        ++its;
        cd mu;
        if (its % 11 == 10) {
            mu = T(hi, hi) + 0.75 * std::abs(T(hi, hi - 1));  // exceptional shift
        } else {
            const cd a = T(hi - 1, hi - 1), b = T(hi - 1, hi), c = T(hi, hi - 1), d = T(hi, hi);
            const cd del = 0.5 * (a - d), bc = b * c;
            cd disc = std::sqrt(del * del + bc);
            if (std::abs(del + disc) < std::abs(del - disc)) disc = -disc;
            mu = (del + disc) == cd(0.0) ? d : d - bc / (del + disc);
        }
        for (int i = lo; i <= hi; ++i) T(i, i) -= mu;
        for (int k = lo; k < hi; ++k) {
            cgivens(T(k, k), T(k + 1, k), cs[k], sn[k]);
            rot_left(T, k, k, cs[k], sn[k]);
            T(k + 1, k) = 0.0;
        }
        for (int k = lo; k < hi; ++k) {
            rot_right(T, k, std::min(k + 2, hi + 1), cs[k], sn[k]);
            rot_right(Z, k, n, cs[k], sn[k]);
        }
        for (int i = lo; i <= hi; ++i) T(i, i) += mu;
    }
    return true;
}

// swap the diagonal entries k and k + 1 of the triangular T, Z along
static void schur_swap(Cmat &T, Cmat &Z, int k) {
    const cd t11 = T(k, k), t22 = T(k + 1, k + 1);
    double c;
    cd s;
    cgivens(T(k, k + 1), t22 - t11, c, s);
    rot_left(T, k, k, c, s);
    rot_right(T, k, k + 2, c, s);
    rot_right(Z, k, Z.n, c, s);
    T(k, k) = t22;
    T(k + 1, k + 1) = t11;
    T(k + 1, k) = 0.0;
}

int deflation_basis(const double *H, int m, int ldh, int l, double *B, int *sdim, double *lam_max) {
    *sdim = 0;
    *lam_max = 0.0;
    if (m <= 0) return 0;
    Cmat T(m), Z(m);
    for (int i = 0; i < m; ++i)
        for (int j = 0; j < m; ++j) T(i, j) = (j >= i - 1) ? H[(size_t)i * ldh + j] : 0.0;
    if (!complex_schur(T, Z)) return -1;
    std::vector<double> mod(m);
    for (int k = 0; k < m; ++k) mod[k] = std::abs(T(k, k));
    std::vector<double> srt(mod);
    std::sort(srt.begin(), srt.end());
    *lam_max = srt[m - 1];
    if (l <= 0) return 0;
    const double cut = srt[std::min(l, m) - 1] * (1.0 + 1e-12);
    std::vector<char> sel(m);
    for (int k = 0; k < m; ++k) sel[k] = mod[k] <= cut;
    // selected entries to the front, in their order
    int pos = 0;
    for (int k = 0; k < m; ++k) {
        if (!sel[k]) continue;
        for (int j = k - 1; j >= pos; --j) {
            schur_swap(T, Z, j);
            std::swap(sel[j], sel[j + 1]);
        }
        ++pos;
    }
    const int ns = pos;
    // real orthonormal basis of span(Z[:, :ns]): modified Gram-Schmidt over
    // the real and imaginary parts, keeping a direction when at least 1e-6 of
    // its norm is new
    std::vector<double> v(m);
    int nb = 0;
    for (int k = 0; k < ns && nb < ns; ++k)
        for (int part = 0; part < 2 && nb < ns; ++part) {
            double n0 = 0.0;
            for (int i = 0; i < m; ++i) {
                v[i] = part ? Z(i, k).imag() : Z(i, k).real();
                n0 += v[i] * v[i];
            }
            n0 = std::sqrt(n0);
            if (n0 == 0.0) continue;
            for (int pass = 0; pass < 2; ++pass)
                for (int q = 0; q < nb; ++q) {
                    double d = 0.0;
                    for (int i = 0; i < m; ++i) d += B[(size_t)i * m + q] * v[i];
                    for (int i = 0; i < m; ++i) v[i] -= d * B[(size_t)i * m + q];
                }
            double n1 = 0.0;
            for (int i = 0; i < m; ++i) n1 += v[i] * v[i];
            n1 = std::sqrt(n1);
            if (n1 <= 1e-6 * n0) continue;
            for (int i = 0; i < m; ++i) B[(size_t)i * m + nb] = v[i] / n1;
            ++nb;
        }
    *sdim = nb;
    return 0;
}

}  // namespace tdbem
