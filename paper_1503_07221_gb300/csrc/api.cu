// Host side of libtdbem: the C ABI declared in include/tdbem.h, input
// validation, the planner (unique blocks, block classes, colouring, chunk
// plans, neighbour lists, quadrature rules) and the launch sequence of one
// assembly.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <cstdio>
#include <map>
#include <mutex>
#include <numeric>
#include <set>
#include <string>
#include <vector>

#include "tdbem_internal.h"

using namespace tdbem;

// ------------------------------------------------------------ error state
static thread_local std::string g_err = "no error";

static tdbem_status fail(tdbem_status code, const std::string &msg) {
    g_err = msg;
    return code;
}

#define CUDA_TRY(call)                                                                      \
    do {                                                                                    \
        cudaError_t e_ = (call);                                                            \
        if (e_ != cudaSuccess)                                                              \
            return fail(TDBEM_E_CUDA, std::string(#call) + ": " + cudaGetErrorString(e_)); \
    } while (0)

// --------------------------------------------------------------- allocator
static void *(*g_alloc)(size_t, void *, void *) = nullptr;
static void (*g_free)(void *, void *, void *) = nullptr;
static void *g_alloc_ctx = nullptr;

struct DevBuf {
    void *p = nullptr;
    size_t n = 0;
    void *(*alloc)(size_t, void *, void *) = nullptr;
    void (*free_)(void *, void *, void *) = nullptr;
    void *ctx = nullptr;
    cudaStream_t st = nullptr;
    void release() {
        if (!p) return;
        if (free_) free_(p, st, ctx);
        else cudaFree(p);
        p = nullptr;
        n = 0;
    }
    ~DevBuf() { release(); }
};

static tdbem_status dev_alloc(DevBuf &b, size_t bytes, cudaStream_t st) {
    b.release();
    if (bytes == 0) bytes = 16;
    b.alloc = g_alloc; b.free_ = g_free; b.ctx = g_alloc_ctx; b.st = st;
    if (g_alloc) b.p = g_alloc(bytes, st, g_alloc_ctx);
    else if (cudaMalloc(&b.p, bytes) != cudaSuccess) b.p = nullptr;
    if (!b.p) {
        cudaGetLastError();
        return fail(TDBEM_E_OOM, "device allocation of " + std::to_string(bytes) + " bytes failed");
    }
    b.n = bytes;
    return TDBEM_OK;
}

template <typename T>
static tdbem_status upload(DevBuf &b, const std::vector<T> &v, cudaStream_t st) {
    tdbem_status s = dev_alloc(b, v.size() * sizeof(T), st);
    if (s) return s;
    if (!v.empty()) CUDA_TRY(cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, st));
    return TDBEM_OK;
}

// ------------------------------------------------------- quadrature rules
// Gauss-Legendre nodes and weights on [0,1] (Newton on P_n from the
// Chebyshev-like initial guess cos(pi (i + 3/4)/(n + 1/2))).
static void gauss_legendre01(int n, std::vector<double> &x, std::vector<double> &w) {
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = cos(M_PI * (i + 0.75) / (n + 0.5)), dp = 1.0;
        for (int it = 0; it < 200; ++it) {
            double p0 = 1.0, p1 = z;
            for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
            if (n == 1) { p0 = 1.0; p1 = z; }
            dp = n * (z * p1 - p0) / (z * z - 1.0);
            const double dz = p1 / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double p0 = 1.0, p1 = z;
        for (int k = 2; k <= n; ++k) { const double p2 = ((2 * k - 1) * z * p1 - (k - 1) * p0) / k; p0 = p1; p1 = p2; }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        x[n - 1 - i] = 0.5 * (z + 1.0);
        w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
    }
}

// Radon's 7-point rule of degree 5 on a triangle: barycentric points and
// weights summing to 1 (centroid, and two 3-point orbits built from sqrt(15)).
static void radon7(double L[7][3], double W[7]) {
    const double s = sqrt(15.0);
    const double a1 = (6.0 - s) / 21.0, b1 = 1.0 - 2.0 * a1, w1 = (155.0 - s) / 1200.0;
    const double a2 = (6.0 + s) / 21.0, b2 = 1.0 - 2.0 * a2, w2 = (155.0 + s) / 1200.0;
    const double P[7][3] = {{1.0 / 3, 1.0 / 3, 1.0 / 3}, {b1, a1, a1}, {a1, b1, a1}, {a1, a1, b1},
                            {b2, a2, a2}, {a2, b2, a2}, {a2, a2, b2}};
    for (int k = 0; k < 7; ++k) {
        for (int d = 0; d < 3; ++d) L[k][d] = P[k][d];
        W[k] = k == 0 ? 9.0 / 40.0 : (k < 4 ? w1 : w2);
    }
}

// Sauter-Schwab rule on T x T with T = {0 <= x2 <= x1 <= 1} (area 1/2):
// the regularising substitutions for identical triangles (6 regions, weight
// xi^3 e1^2 e2), a common edge from (0,0) to (1,0) (5 regions, weights
// xi^3 e1^2 and xi^3 e1^2 e2) and a common vertex (0,0) (2 regions, weight
// xi^3 e2), tensor Gauss-Legendre with n points per direction on [0,1]^4.
// Output rows: x1, x2, y1, y2, weight.
static std::vector<double> sauter_schwab(int kase, int n) {
    std::vector<double> gx, gw;
    gauss_legendre01(n, gx, gw);
    std::vector<double> out;
    for (int i0 = 0; i0 < n; ++i0)
        for (int i1 = 0; i1 < n; ++i1)
            for (int i2 = 0; i2 < n; ++i2)
                for (int i3 = 0; i3 < n; ++i3) {
                    const double xi = gx[i0], a = gx[i1], b = gx[i2], c = gx[i3];
                    const double W = gw[i0] * gw[i1] * gw[i2] * gw[i3];
                    auto put = [&](double x1, double x2, double y1, double y2, double j) {
                        out.push_back(x1); out.push_back(x2); out.push_back(y1); out.push_back(y2);
                        out.push_back(W * j);
                    };
                    if (kase == 3) {
                        const double j = xi * xi * xi * a * a * b;
                        const double u1 = xi, u2 = xi * (1 - a + a * b), v1 = xi * (1 - a * b * c), v2 = xi * (1 - a);
                        put(u1, u2, v1, v2, j); put(v1, v2, u1, u2, j);
                        const double p1 = xi, p2 = xi * a * (1 - b + b * c), q1 = xi * (1 - a * b), q2 = xi * a * (1 - b);
                        put(p1, p2, q1, q2, j); put(q1, q2, p1, p2, j);
                        const double r1 = xi * (1 - a * b * c), r2 = xi * a * (1 - b * c), s1 = xi, s2 = xi * a * (1 - b);
                        put(r1, r2, s1, s2, j); put(s1, s2, r1, r2, j);
                    } else if (kase == 2) {
                        const double j0 = xi * xi * xi * a * a, j1 = j0 * b;
                        put(xi, xi * a * c, xi * (1 - a * b), xi * a * (1 - b), j0);
                        put(xi, xi * a, xi * (1 - a * b * c), xi * a * b * (1 - c), j1);
                        put(xi * (1 - a * b), xi * a * (1 - b), xi, xi * a * b * c, j1);
                        put(xi * (1 - a * b * c), xi * a * b * (1 - c), xi, xi * a, j1);
                        put(xi * (1 - a * b * c), xi * a * (1 - b * c), xi, xi * a * b, j1);
                    } else {
                        const double j = xi * xi * xi * b;
                        put(xi, xi * a, xi * b, xi * b * c, j);
                        put(xi * b, xi * b * c, xi, xi * a, j);
                    }
                }
    return out;
}

// ------------------------------------------------------------------- mesh
struct tdbem_mesh {
    int64_t M = 0, E = 0;
    std::vector<double> V;
    std::vector<int32_t> F;
    std::vector<double> cen, dq, geo64;
    std::vector<float> dq32, geo32;
    std::vector<int64_t> vt_ptr;
    std::vector<int32_t> vt_tri;
    std::vector<int64_t> adj_ptr;
    std::vector<int32_t> adj_tri;
    std::vector<int8_t> adj_perm;
    std::vector<int32_t> adj_nbr;
    std::vector<int64_t> nbr_ptr;
    std::vector<int32_t> nbr;
    int NB = 0;
    std::vector<std::vector<int32_t>> colors;
    std::vector<int32_t> chunk_vptr, chunk_vert, chunk_sptr, chunk_src;
    int max_nv = 0;
    int64_t nchunks = 0;
    double diam = 0.0, max_dq = 0.0, max_star = 0.0, coord_scale = 0.0;
    double rule_L[7][3], rule_W[7];
};

static tdbem_status build_mesh(tdbem_mesh &m) {
    const int64_t M = m.M, E = m.E;
    const double *V = m.V.data();
    const int32_t *F = m.F.data();
    radon7(m.rule_L, m.rule_W);
    m.cen.assign(3 * E, 0.0);
    m.dq.assign(21 * E, 0.0);
    m.dq32.assign(21 * E, 0.f);
    m.geo64.assign(16 * E, 0.0);
    m.geo32.assign(16 * E, 0.f);
    for (int64_t e = 0; e < E; ++e) {
        const double *P[3] = {V + 3 * F[3 * e], V + 3 * F[3 * e + 1], V + 3 * F[3 * e + 2]};
        double u[3], v[3], c[3];
        for (int d = 0; d < 3; ++d) { u[d] = P[1][d] - P[0][d]; v[d] = P[2][d] - P[0][d]; }
        c[0] = u[1] * v[2] - u[2] * v[1];
        c[1] = u[2] * v[0] - u[0] * v[2];
        c[2] = u[0] * v[1] - u[1] * v[0];
        const double len = sqrt(c[0] * c[0] + c[1] * c[1] + c[2] * c[2]);
        if (!(len > 0.0) || !std::isfinite(len))
            return fail(TDBEM_E_MESH, "triangle " + std::to_string(e) + " has zero area");
        const double area = 0.5 * len;
        double *g = m.geo64.data() + 16 * e;
        for (int d = 0; d < 3; ++d) g[d] = c[d] / len;
        g[3] = area;
        // surface curl of the hat function of corner a: n x grad lambda_a = -(P_{a+2} - P_{a+1}) / (2|T|)
        for (int a = 0; a < 3; ++a)
            for (int d = 0; d < 3; ++d) g[4 + 3 * a + d] = -(P[(a + 2) % 3][d] - P[(a + 1) % 3][d]) / (2.0 * area);
        for (int k = 0; k < 16; ++k) m.geo32[16 * e + k] = (float)g[k];
        for (int d = 0; d < 3; ++d) m.cen[3 * e + d] = (P[0][d] + P[1][d] + P[2][d]) / 3.0;
        for (int k = 0; k < 7; ++k)
            for (int d = 0; d < 3; ++d) {
                const double x = m.rule_L[k][0] * P[0][d] + m.rule_L[k][1] * P[1][d] + m.rule_L[k][2] * P[2][d];
                m.dq[21 * e + 3 * k + d] = x - m.cen[3 * e + d];
                m.dq32[21 * e + 3 * k + d] = (float)m.dq[21 * e + 3 * k + d];
            }
        for (int k = 0; k < 7; ++k) {
            const double *q = m.dq.data() + 21 * e + 3 * k;
            m.max_dq = std::max(m.max_dq, sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]));
        }
    }
    // vertex -> triangles
    m.vt_ptr.assign(M + 1, 0);
    for (int64_t e = 0; e < E; ++e)
        for (int a = 0; a < 3; ++a) m.vt_ptr[F[3 * e + a] + 1]++;
    for (int64_t v = 0; v < M; ++v) m.vt_ptr[v + 1] += m.vt_ptr[v];
    m.vt_tri.assign(3 * E, 0);
    {
        std::vector<int64_t> fill(m.vt_ptr.begin(), m.vt_ptr.end() - 1);
        for (int64_t e = 0; e < E; ++e)
            for (int a = 0; a < 3; ++a) m.vt_tri[fill[F[3 * e + a]]++] = (int32_t)e;
    }
    for (int64_t v = 0; v < M; ++v)
        if (m.vt_ptr[v + 1] == m.vt_ptr[v]) return fail(TDBEM_E_MESH, "vertex " + std::to_string(v) + " belongs to no triangle");
    // triangles sharing a vertex with tau (tau included), with the corner
    // permutations that put the shared vertices first in the same order
    m.adj_ptr.assign(E + 1, 0);
    m.adj_tri.clear();
    m.adj_perm.clear();
    for (int64_t t = 0; t < E; ++t) {
        std::set<int32_t> s;
        for (int a = 0; a < 3; ++a)
            for (int64_t x = m.vt_ptr[F[3 * t + a]]; x < m.vt_ptr[F[3 * t + a] + 1]; ++x) s.insert(m.vt_tri[x]);
        for (int32_t q : s) {
            int pa[3] = {0, 1, 2}, pb[3] = {0, 1, 2};
            int shared = 0, ia[3], ib[3];
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b)
                    if (F[3 * t + a] == F[3 * q + b]) { ia[shared] = a; ib[shared] = b; ++shared; }
            if (shared == 2) {
                pa[0] = ia[0]; pa[1] = ia[1]; pa[2] = 3 - ia[0] - ia[1];
                pb[0] = ib[0]; pb[1] = ib[1]; pb[2] = 3 - ib[0] - ib[1];
            } else if (shared == 1) {
                for (int k = 0; k < 3; ++k) { pa[k] = (ia[0] + k) % 3; pb[k] = (ib[0] + k) % 3; }
            } else if (shared == 3) {
                if (q != t) return fail(TDBEM_E_MESH, "triangles " + std::to_string(t) + " and " + std::to_string(q) + " repeat the same vertices");
            }
            m.adj_tri.push_back(q);
            const int8_t rec[8] = {(int8_t)shared, (int8_t)pa[0], (int8_t)pa[1], (int8_t)pa[2],
                                   (int8_t)pb[0], (int8_t)pb[1], (int8_t)pb[2], 0};
            m.adj_perm.insert(m.adj_perm.end(), rec, rec + 8);
        }
        m.adj_ptr[t + 1] = (int64_t)m.adj_tri.size();
    }
    // near neighbour lists: j reached from l by an adjacent element pair
    std::vector<std::vector<int32_t>> nb(M);
    for (int64_t t = 0; t < E; ++t)
        for (int64_t x = m.adj_ptr[t]; x < m.adj_ptr[t + 1]; ++x)
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) nb[F[3 * t + a]].push_back(F[3 * m.adj_tri[x] + b]);
    m.nbr_ptr.assign(M + 1, 0);
    m.nbr.clear();
    m.NB = 0;
    for (int64_t v = 0; v < M; ++v) {
        std::sort(nb[v].begin(), nb[v].end());
        nb[v].erase(std::unique(nb[v].begin(), nb[v].end()), nb[v].end());
        m.nbr.insert(m.nbr.end(), nb[v].begin(), nb[v].end());
        m.nbr_ptr[v + 1] = (int64_t)m.nbr.size();
        m.NB = std::max(m.NB, (int)nb[v].size());
    }
    m.adj_nbr.assign(9 * m.adj_tri.size(), -1);
    for (int64_t t = 0; t < E; ++t)
        for (int64_t x = m.adj_ptr[t]; x < m.adj_ptr[t + 1]; ++x) {
            const int8_t *pm = m.adj_perm.data() + 8 * x;
            for (int a = 0; a < 3; ++a)
                for (int b = 0; b < 3; ++b) {
                    const int32_t l = F[3 * t + pm[1 + a]], j = F[3 * m.adj_tri[x] + pm[4 + b]];
                    const auto &L = nb[l];
                    m.adj_nbr[9 * x + 3 * a + b] = (int32_t)(std::lower_bound(L.begin(), L.end(), j) - L.begin());
                }
        }
    // greedy colouring: no two triangles of one colour share a vertex
    std::vector<int> col(E, -1);
    int ncol = 0;
    for (int64_t t = 0; t < E; ++t) {
        std::vector<char> used(64, 0);
        for (int64_t x = m.adj_ptr[t]; x < m.adj_ptr[t + 1]; ++x) {
            const int c = col[m.adj_tri[x]];
            if (c >= 0 && c < 64) used[c] = 1;
        }
        int c = 0;
        while (c < 64 && used[c]) ++c;
        if (c == 64) return fail(TDBEM_E_MESH, "vertex valence too high for the colouring");
        col[t] = c;
        ncol = std::max(ncol, c + 1);
    }
    m.colors.assign(ncol, {});
    for (int64_t t = 0; t < E; ++t) m.colors[col[t]].push_back((int32_t)t);
    // chunk plans: for 32 consecutive trial triangles, their vertices and
    // the (triangle, corner) sources of each vertex
    m.nchunks = (E + 31) / 32;
    m.chunk_vptr.assign(m.nchunks + 1, 0);
    m.chunk_vert.clear();
    m.chunk_sptr.clear();
    m.chunk_src.clear();
    for (int64_t ch = 0; ch < m.nchunks; ++ch) {
        std::map<int32_t, std::vector<int32_t>> vs;
        for (int s = 0; s < 32 && ch * 32 + s < E; ++s)
            for (int b = 0; b < 3; ++b) vs[F[3 * (ch * 32 + s) + b]].push_back(3 * s + b);
        for (auto &kv : vs) {
            m.chunk_vert.push_back(kv.first);
            m.chunk_sptr.push_back((int32_t)m.chunk_src.size());
            m.chunk_src.insert(m.chunk_src.end(), kv.second.begin(), kv.second.end());
        }
        m.chunk_vptr[ch + 1] = (int32_t)m.chunk_vert.size();
        m.max_nv = std::max(m.max_nv, m.chunk_vptr[ch + 1] - m.chunk_vptr[ch]);
    }
    m.chunk_sptr.push_back((int32_t)m.chunk_src.size());
    // diameter (largest vertex distance) and largest star diameter
    double dm = 0.0;
    for (int64_t i = 0; i < M; ++i)
        for (int64_t j = i + 1; j < M; ++j) {
            const double a = V[3 * i] - V[3 * j], b = V[3 * i + 1] - V[3 * j + 1], c = V[3 * i + 2] - V[3 * j + 2];
            const double v = a * a + b * b + c * c;
            if (v > dm) dm = v;
        }
    m.diam = sqrt(dm);
    for (int64_t i = 0; i < 3 * M; ++i) m.coord_scale = std::max(m.coord_scale, fabs(V[i]));
    for (int64_t v = 0; v < M; ++v) {
        std::vector<int32_t> pts;
        for (int64_t x = m.vt_ptr[v]; x < m.vt_ptr[v + 1]; ++x)
            for (int a = 0; a < 3; ++a) pts.push_back(F[3 * m.vt_tri[x] + a]);
        for (size_t i = 0; i < pts.size(); ++i)
            for (size_t j = i + 1; j < pts.size(); ++j) {
                const double *p = V + 3 * pts[i], *q = V + 3 * pts[j];
                const double d = sqrt((p[0] - q[0]) * (p[0] - q[0]) + (p[1] - q[1]) * (p[1] - q[1]) + (p[2] - q[2]) * (p[2] - q[2]));
                m.max_star = std::max(m.max_star, d);
            }
    }
    return TDBEM_OK;
}

// --------------------------------------------------------------- time grid
struct tdbem_timegrid {
    int64_t N = 0;
    int p = 0, kind = 0;
    double c = 1.0, T = 0.0, dt = 0.0;
    bool equidistant = false;
    std::vector<double> t;
};

// -------------------------------------------------------------- assembler
struct Block {
    int kb, ib, cls, lag;
    double a, b;
    int m2 = 0, m1 = 0;  // temporal orders of the test and trial functions (p >= 1)
};

struct tdbem_asm {
    const tdbem_mesh *mesh = nullptr;
    const tdbem_timegrid *tg = nullptr;
    tdbem_opts opts{};
    bool fp64 = false;
    int OFF = 1, KW = 8, S64 = 4;
    std::vector<Block> blocks;
    int cls_dlo[NCLASS], cls_dhi[NCLASS], cls_rho[NCLASS], cls_P[NCLASS];
    std::vector<int> blk_of_lag, lag_base, blk_of_spec;
    std::vector<std::vector<double>> lag_a, lag_b;
    // device buffers
    DevBuf F, V, cen, dq, dq32, geo32, geo64, vt_ptr, vt_tri, adj_ptr, adj_tri, adj_perm, adj_nbr,
        nbr_ptr, nbr, chunk_vptr, chunk_vert, chunk_sptr, chunk_src, chunk_hdr, colors, rule_w, rule_l, tgrid,
        rule_w64, rule_l64, lagA, lagB, rec, wdlo, wdhi, wsmask, dense, dense_spec, ndense, ndense_spec, status,
        cls_dlo_d, cls_dhi_d, blk_of_lag_d, lag_base_d, blk_of_spec_d, cnt_far, cnt_near, rp_far,
        rp_near, tot_far, tot_near, off_far_d, off_near_d, col_far, val_far, col_near, val_near,
        tab_kb, tab_ib, tab_r0, tab_samples, tab_coef1, tab_coef4, gl_x, gl_w, ss[4], quad_partial;
    std::vector<int64_t> color_off;
    int ss_npp[4] = {0, 0, 0, 0};
    ChebF32 c32{};
    ChebLag32 c32s{};  // lag-class panels for the mixed far kernel (term-major, signed)
    std::vector<int64_t> nnz_far, nnz_near, off_far, off_near;
    bool assembled = false;
    tdbem_stats_t stats{};
    size_t col_far_cap = 0, col_near_cap = 0;
    // block-Hessenberg matvec: run descriptors and the transposed-x scratch
    DevBuf mv_blk, mv_xT;
    std::vector<MvBlock> mv_host;
    // mixed path on an equidistant grid: the Toeplitz class (inner blocks
    // (k, 1) and (1, 2)) as per-pair lag windows (toeplitz.cu), every other
    // block by the CSR kernel (mv_rest)
    DevBuf pb_list, pb_cnt;
    int64_t pb_cap = 0;
    bool tw_on = false;
    int tw_TL = 8, tw_S = 0, tw_PADL = 0;
    int64_t tw_nfar = 0, tw_nnear = 0;
    size_t tw_cap_far = 0, tw_cap_near = 0;
    DevBuf tw_cnt, tw_ptr, tw_tot, tw_fhdr, tw_fval, tw_nhdr, tw_nval, mv_rest;
    std::vector<MvBlock> mv_rest_host;
    mutable int mv_variant = -1;  // matvec launch shape chosen by the autotuner
    // repeated assemblies: the recorded device sequence (CUDA graph)
    cudaEvent_t ev[5] = {nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t cap_stream = nullptr;
    cudaGraphExec_t gexec[4] = {nullptr, nullptr, nullptr, nullptr};  // the four timed phases
    bool use_graph = true;
    // graded (non-equidistant) grids: every nonzero block is its own unique
    // block; column-major block numbering, panels and batches (graded.cu)
    bool graded = false;
    std::vector<int> g_colblk, g_colk0, g_cb2api, g_pan0, g_p64, g_kw;
    std::vector<double> g_ga, g_gb;
    std::vector<GPan64> g_pan64;
    std::vector<float4> g_pan32;
    int g_npan = 0, g_nset64 = 0, g_maxpan = 0, g_njob32 = 0;
    int g_ncol = 0;  // block columns: one per trial function (i, m1)
    double g_smax = -1.0;  // window spread Dmax - Dmin the batches were planned for
    std::vector<int> g_bi0, g_bi1;           // batches of trial columns [i0, i1)
    std::vector<int64_t> g_doff, g_ndoff;    // per column: window offsets inside its batch
    size_t g_dense_max = 0, g_ndense_max = 0;
    DevBuf gpair, gvmin, gvmax, gpartial, g_ga_d, g_gb_d, g_colblk_d, g_colk0_d, g_cb2api_d, g_pan0_d, g_pan64_d,
        g_pan32_d, g_p64_d, g_kw_d, g_doff_d, g_ndoff_d, g_tkb, g_tib, g_tr0, g_tdr, g_samples, g_coef, g_coef32,
        g_geol, g_cenh, g_cenl, g_coloff_d, g_dense, g_ndense, g_tm2, g_tm1;
    std::vector<cudaEvent_t> g_ev;
    // one block on its own (tdbem_assemble_block): the planner keeps only
    // block (only_k, only_i); `single` is the sub-assembler of the last call
    int only_k = -1, only_i = -1;
    tdbem_asm *single = nullptr;
    ~tdbem_asm() {
        delete single;
        for (auto &e : g_ev)
            if (e) cudaEventDestroy(e);
        for (auto &g : gexec)
            if (g) cudaGraphExecDestroy(g);
        if (cap_stream) cudaStreamDestroy(cap_stream);
        for (auto &e : ev)
            if (e) cudaEventDestroy(e);
    }
};

// rows of x and y: the L = N (p + 1) time functions (Sec. 3 numbering)
static int64_t time_rows(const tdbem_asm *A) { return A->tg->N * (A->tg->p + 1); }

static int kind_of(int64_t i, int64_t N) { return i == 0 ? 0 : (i == N - 1 ? 2 : 1); }  // F, I, L

// Rebalanced copy of the mesh's vertex-disjoint triangle colouring for the
// equidistant far and near kernels, which take one colour per launch with G
// CTAs, each a whole test triangle at a time: a colour of n triangles costs
// about ceil(n / G) rounds. Triangles move from a colour's last partial round
// into colours with room in theirs wherever none of their vertices is used
// there (the colouring stays vertex-disjoint), until no colour's excess can
// move; empty colours are dropped. Deterministic: colours and triangles are
// taken in a fixed order.
static std::vector<std::vector<int32_t>> balance_colours(const tdbem_mesh &m, int G) {
    const int ncol = (int)m.colors.size();
    std::vector<std::vector<int32_t>> out = m.colors;
    if (ncol < 2 || ncol > 64 || G < 1) return out;
    const int32_t *F = m.F.data();
    std::vector<uint64_t> vmask(m.M, 0);
    std::vector<int> col(m.E, -1);
    std::vector<int64_t> size(ncol, 0);
    for (int c = 0; c < ncol; ++c)
        for (int32_t t : m.colors[c]) {
            col[t] = c;
            ++size[c];
            for (int k = 0; k < 3; ++k) vmask[F[3 * t + k]] |= 1ull << c;
        }
    auto rounds = [&]() {
        int64_t w = 0;
        for (int c = 0; c < ncol; ++c) w += (size[c] + G - 1) / G;
        return w;
    };
    for (int it = 0; it < 4 * ncol + 64; ++it) {
        const int64_t w0 = rounds();
        std::vector<int> order(ncol);
        std::iota(order.begin(), order.end(), 0);
        auto excess = [&](int c) { return size[c] % G ? size[c] % G : (int64_t)G; };
        std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return excess(a) < excess(b); });
        bool improved = false;
        for (int c : order) {
            const int64_t ex = size[c] % G;
            if (ex == 0) continue;
            std::vector<int> tg;
            for (int d = 0; d < ncol; ++d)
                if (d != c && size[d] % G != 0) tg.push_back(d);
            std::stable_sort(tg.begin(), tg.end(), [&](int a, int b) { return size[a] % G > size[b] % G; });
            int64_t moved = 0;
            for (int64_t t = 0; t < m.E && moved < ex; ++t) {
                if (col[t] != c) continue;
                const uint64_t used = vmask[F[3 * t]] | vmask[F[3 * t + 1]] | vmask[F[3 * t + 2]];
                for (int d : tg) {
                    if (size[d] % G == 0 || ((used >> d) & 1ull)) continue;
                    for (int k = 0; k < 3; ++k) vmask[F[3 * t + k]] = (vmask[F[3 * t + k]] & ~(1ull << c)) | (1ull << d);
                    col[t] = d;
                    --size[c];
                    ++size[d];
                    ++moved;
                    break;
                }
            }
            if (moved == ex || rounds() < w0) {
                improved = true;
                break;
            }
        }
        if (!improved) break;
    }
    out.assign(ncol, {});
    for (int64_t t = 0; t < m.E; ++t) out[col[t]].push_back((int32_t)t);
    out.erase(std::remove_if(out.begin(), out.end(), [](const std::vector<int32_t> &v) { return v.empty(); }),
              out.end());
    // every colour vertex-disjoint, every triangle once: else keep the mesh's colouring
    std::vector<int> stamp(m.M, -1);
    int64_t total = 0;
    for (size_t c = 0; c < out.size(); ++c) {
        total += (int64_t)out[c].size();
        for (int32_t t : out[c])
            for (int k = 0; k < 3; ++k) {
                int &st = stamp[F[3 * t + k]];
                if (st == (int)c) return m.colors;
                st = (int)c;
            }
    }
    if (total != m.E) return m.colors;
    return out;
}

static tdbem_status plan_blocks(tdbem_asm &A) {
    const tdbem_timegrid &tg = *A.tg;
    const int64_t N = tg.N;
    const double *t = tg.t.data();
    const double T = t[N - 1];
    auto tl = [&](int64_t q) { return q == 0 ? 0.0 : t[q - 1]; };
    auto tr = [&](int64_t q) { return q == N - 1 ? T : t[q + 1]; };
    A.blocks.clear();
    for (int c = 0; c < NCLASS; ++c) { A.cls_dlo[c] = 1 << 20; A.cls_dhi[c] = -(1 << 20); }
    for (int64_t k = 0; k < N; ++k)
        for (int64_t i = 0; i < N; ++i) {
            const bool want = i == 0 || i == 1 || k == N - 1 || (k == 1 && i == 2) || (k == N - 2 && i == N - 1);
            if (!want || i > k + 1) continue;
            const double a = std::max(0.0, tl(k) - tr(i)), b = tr(k) - tl(i);
            if (!(b > a) || a >= A.mesh->diam - 1e-12 * T) continue;
            const int kk = kind_of(k, N), ki = kind_of(i, N);
            int cls, lag;
            if (kk == 1 && ki == 0) { cls = C1; lag = (int)k; }
            else if (kk == 1 && ki == 1) { cls = C2; lag = (int)(k - i); }
            else if (kk == 2 && ki == 1) { cls = C3; lag = (int)(N - 1 - i); }
            else if (kk == 0 && ki == 0) { cls = S00; lag = 0; }
            else if (kk == 0 && ki == 1) { cls = S01; lag = 0; }
            else if (kk == 2 && ki == 0) { cls = SN0; lag = 0; }
            else if (kk == 2 && ki == 2) { cls = SNN; lag = 0; }
            else if (kk == 1 && ki == 2) { cls = SN1N; lag = 0; }
            else return fail(TDBEM_E_UNSUPPORTED, "unexpected block kind");
            A.blocks.push_back({(int)k, (int)i, cls, lag, a, b});
            A.cls_dlo[cls] = std::min(A.cls_dlo[cls], lag);
            A.cls_dhi[cls] = std::max(A.cls_dhi[cls], lag);
        }
    // lag tables and block lookup
    A.lag_a.assign(NCLASS, {});
    A.lag_b.assign(NCLASS, {});
    A.lag_base.assign(NLAG + 1, 0);
    A.blk_of_spec.assign(NSPEC, -1);
    for (int c = 0; c < NLAG; ++c) {
        const int n = A.cls_dhi[c] >= A.cls_dlo[c] ? A.cls_dhi[c] - A.cls_dlo[c] + 1 : 0;
        A.lag_base[c + 1] = A.lag_base[c] + n;
        A.lag_a[c].assign(n, NAN);
        A.lag_b[c].assign(n, NAN);
    }
    A.blk_of_lag.assign(std::max(1, A.lag_base[NLAG]), -1);
    for (size_t bi = 0; bi < A.blocks.size(); ++bi) {
        const Block &b = A.blocks[bi];
        if (b.cls < NLAG) {
            const int x = b.lag - A.cls_dlo[b.cls];
            A.lag_a[b.cls][x] = b.a;
            A.lag_b[b.cls][x] = b.b;
            A.blk_of_lag[A.lag_base[b.cls] + x] = (int)bi;
        } else {
            A.lag_a[b.cls] = {b.a};
            A.lag_b[b.cls] = {b.b};
            A.blk_of_spec[b.cls - NLAG] = (int)bi;
        }
    }
    for (int c = 0; c < NLAG; ++c)
        for (size_t x = 0; x < A.lag_a[c].size(); ++x)
            if (std::isnan(A.lag_a[c][x])) return fail(TDBEM_E_UNSUPPORTED, "non-contiguous lag range");
    // panels of each class: rho in units of dt, P panels
    const double dt = tg.dt;
    const int Pc[NCLASS] = {3, 4, 3, 1, 1, 2, 1, 1};
    for (int c = 0; c < NCLASS; ++c) {
        A.cls_P[c] = Pc[c];
        A.cls_rho[c] = c < NLAG ? -2 : (c == SN0 ? (int)(N - 3) : 0);
    }
    (void)dt;
    return TDBEM_OK;
}

// Graded grid: every (k, i) with i <= k + 1 whose support (a, b) starts below
// diam(Gamma) is assembled (Sec. 3.2; no reuse without shift invariance).
// The caller's list is k-major like the equidistant one; internally the
// blocks of each trial column i form a contiguous k-range (a and b grow with
// k). psi_{k,i} is smooth between the breakpoints t_{k-a} - t_{i-b},
// a, b in {0, 1, 2} (Sec. 3.1), which bound its Chebyshev panels.
static tdbem_status plan_graded(tdbem_asm &A) {
    const tdbem_timegrid &tg = *A.tg;
    const int64_t N = tg.N, P1 = tg.p + 1;
    const double *t = tg.t.data();
    const double T = t[N - 1];
    const double tie = 1e-12 * T;
    auto tl = [&](int64_t q) { return q == 0 ? 0.0 : t[q - 1]; };
    auto tr = [&](int64_t q) { return q == N - 1 ? T : t[q + 1]; };
    A.blocks.clear();
    // block (k, i) of every order pair (m2, m1): api_of[((k N + i) P1 + m2) P1 + m1]
    std::vector<int> api_of((size_t)(N * N * P1 * P1), -1);
    auto aidx = [&](int64_t k, int64_t i, int64_t m2, int64_t m1) { return (size_t)(((k * N + i) * P1 + m2) * P1 + m1); };
    for (int64_t k = 0; k < N; ++k)
        for (int64_t i = 0; i < N && i <= k + 1; ++i) {
            const double a = std::max(0.0, tl(k) - tr(i)), b = tr(k) - tl(i);
            if (!(b > a) || a >= A.mesh->diam - tie) continue;
            if (A.only_k >= 0 && (k != A.only_k || i != A.only_i)) continue;
            for (int64_t m2 = 0; m2 < P1; ++m2)
                for (int64_t m1 = 0; m1 < P1; ++m1) {
                    api_of[aidx(k, i, m2, m1)] = (int)A.blocks.size();
                    Block B{(int)k, (int)i, -1, 0, a, b};
                    B.m2 = (int)m2;
                    B.m1 = (int)m1;
                    A.blocks.push_back(B);
                }
        }
    // columns: one per trial function (i, m1), column index i P1 + m1; the
    // blocks of a column in order of (k, m2) (a and b do not decrease)
    A.g_ncol = (int)(N * P1);
    A.g_colblk.assign(A.g_ncol + 1, 0);
    A.g_colk0.assign(A.g_ncol, 0);
    A.g_cb2api.clear();
    A.g_ga.clear();
    A.g_gb.clear();
    A.g_pan0.clear();
    A.g_pan64.clear();
    A.g_pan32.clear();
    A.g_maxpan = 0;
    for (int64_t i = 0; i < N; ++i)
        for (int64_t m1 = 0; m1 < P1; ++m1) {
            const int64_t col = i * P1 + m1;
            A.g_colblk[col] = (int)A.g_cb2api.size();
            int64_t kfirst = -1, klast = -2;
            for (int64_t k = 0; k < N; ++k)
                if (api_of[aidx(k, i, 0, m1)] >= 0) {
                    if (kfirst < 0) kfirst = k;
                    else if (k != klast + 1) return fail(TDBEM_E_UNSUPPORTED, "non-contiguous block column");
                    klast = k;
                }
            A.g_colk0[col] = kfirst < 0 ? 0 : (int)(kfirst * P1);
            if ((klast - kfirst + 1) * P1 > GP_MAXK)
                return fail(TDBEM_E_UNSUPPORTED, "more than 256 blocks (times orders) in one block column");
            const int pcol0 = (int)A.g_pan64.size();
            for (int64_t k = kfirst; kfirst >= 0 && k <= klast; ++k)
                for (int64_t m2 = 0; m2 < P1; ++m2) {
                    const Block &B = A.blocks[api_of[aidx(k, i, m2, m1)]];
                    A.g_cb2api.push_back(api_of[aidx(k, i, m2, m1)]);
                    A.g_ga.push_back(B.a);
                    A.g_gb.push_back(B.b);
                    A.g_pan0.push_back((int)A.g_pan64.size());
                    const double X[3] = {tl(k), t[k], tr(k)}, Y[3] = {tl(i), t[i], tr(i)};
                    std::vector<double> br = {B.a, B.b};
                    for (double x : X)
                        for (double y : Y)
                            if (x - y > B.a && x - y < B.b) br.push_back(x - y);
                    std::sort(br.begin(), br.end());
                    std::vector<double> m = {br[0]};
                    for (size_t q = 1; q < br.size(); ++q)
                        if (br[q] - m.back() > 1e-13 * T) m.push_back(br[q]);
                    if (m.back() != B.b) m.back() = B.b;
                    if (m.size() < 2 || m.size() - 1 > (size_t)GP_MAXPAN) return fail(TDBEM_E_UNSUPPORTED, "bad panel count");
                    for (size_t q = 0; q + 1 < m.size(); ++q) {
                        const double s0 = m[q], w = m[q + 1] - m[q], mid = s0 + 0.5 * w;
                        A.g_pan64.push_back({s0, w, 0.0, 0.0});
                        const float mh = (float)mid;
                        A.g_pan32.push_back(make_float4((float)s0, mh, (float)(mid - (double)mh), (float)(2.0 / w)));
                    }
                }
            A.g_maxpan = std::max(A.g_maxpan, (int)A.g_pan64.size() - pcol0);
        }
    A.g_colblk[A.g_ncol] = (int)A.g_cb2api.size();
    A.g_pan0.push_back((int)A.g_pan64.size());
    A.g_npan = (int)A.g_pan64.size();
    // FP64 coefficient sets: S64 sub-panels per panel; the mixed path needs them
    // only where near pairs (r <= the largest vertex star) evaluate psi
    const double rnear = A.mesh->max_star * (1.0 + 1e-9) + tie;
    A.g_p64.assign(A.g_npan, -1);
    A.g_nset64 = 0;
    for (int p = 0; p < A.g_npan; ++p) {
        GPan64 &q = A.g_pan64[p];
        q.z = A.S64 / q.y;
        if (A.fp64 || q.x < rnear) { A.g_p64[p] = A.g_nset64; A.g_nset64 += A.S64; }
    }
    return TDBEM_OK;
}

// Longest window [K1, K2] of a vertex pair in column i when Dmax - Dmin <=
// smax: with K1 = k (Dmin just below b_k), K2 is at most the last k' with
// a_k' < b_k + smax.
static int graded_kw(const tdbem_asm &A, int64_t i, double smax) {
    const int c0 = A.g_colblk[i], nk = A.g_colblk[i + 1] - c0;
    int best = 1;
    for (int x = 0; x < nk; ++x) {
        int y = x;
        while (y + 1 < nk && A.g_ga[c0 + y + 1] < A.g_gb[c0 + x] + smax) ++y;
        best = std::max(best, y - x + 1);
    }
    return best;
}

// Uploads and allocations of a graded-grid assembler (the time-grid and
// geometry parts the equidistant path also uses, plus the graded block,
// panel and table-job arrays). Window sizes and batches follow in the
// first assembly, once the vertex-pair bounds are known.
static tdbem_status create_graded(tdbem_asm &A, cudaStream_t st) {
    A.graded = true;
    A.use_graph = false;
    A.S64 = 4;
    tdbem_status s = plan_graded(A);
    if (s) return s;
    const tdbem_mesh &m = *A.mesh;
    const int64_t M = m.M, E = m.E;
    // the colouring rebalanced for the far kernel's grid (one CTA per SM)
    int nsm_dev = 0;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm_dev, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return fail(TDBEM_E_CUDA, std::string("device attributes: ") + cudaGetErrorString(e));
    }
    const std::vector<std::vector<int32_t>> bal = balance_colours(m, nsm_dev);
    std::vector<int32_t> colors;
    A.color_off.assign(1, 0);
    for (auto &c : bal) { colors.insert(colors.end(), c.begin(), c.end()); A.color_off.push_back((int64_t)colors.size()); }
    std::vector<float> geol(16 * E), cenh(3 * E), cenl(3 * E);
    for (int64_t k = 0; k < 16 * E; ++k) geol[k] = (float)(m.geo64[k] - (double)m.geo32[k]);
    for (int64_t k = 0; k < 3 * E; ++k) {
        cenh[k] = (float)m.cen[k];
        cenl[k] = (float)(m.cen[k] - (double)cenh[k]);
    }
    std::vector<double> rw64(7), rl64(21);
    for (int k = 0; k < 7; ++k) { rw64[k] = m.rule_W[k]; for (int d = 0; d < 3; ++d) rl64[3 * k + d] = m.rule_L[k][d]; }
    std::vector<double> gx, gw;
    gauss_legendre01(24, gx, gw);
    // psi table jobs: FP32 set (one per panel, mixed path), then the FP64 sets
    std::vector<int> kb, ib, tm2, tm1;
    std::vector<double> r0, dr;
    const int ncb = (int)A.g_cb2api.size();
    auto add_jobs = [&](bool fp64set) {
        for (int cb = 0; cb < ncb; ++cb) {
            const Block &B = A.blocks[A.g_cb2api[cb]];
            for (int p = A.g_pan0[cb]; p < A.g_pan0[cb + 1]; ++p) {
                const GPan64 &q = A.g_pan64[p];
                if (!fp64set) {
                    kb.push_back(B.kb); ib.push_back(B.ib); tm2.push_back(B.m2); tm1.push_back(B.m1);
                    r0.push_back(q.x); dr.push_back(q.y);
                    continue;
                }
                if (A.g_p64[p] < 0) continue;
                for (int sb = 0; sb < A.S64; ++sb) {
                    kb.push_back(B.kb);
                    ib.push_back(B.ib);
                    tm2.push_back(B.m2);
                    tm1.push_back(B.m1);
                    r0.push_back(q.x + q.y * sb / A.S64);
                    dr.push_back(q.y / A.S64);
                }
            }
        }
    };
    if (!A.fp64) add_jobs(false);
    const size_t njob32 = kb.size();
    add_jobs(true);
    if (kb.size() - njob32 != (size_t)A.g_nset64) return fail(TDBEM_E_UNSUPPORTED, "FP64 table job count");
#define UPG(buf, vec) if ((s = upload(A.buf, vec, st))) return s
    UPG(F, m.F); UPG(V, m.V); UPG(cen, m.cen); UPG(dq, m.dq); UPG(dq32, m.dq32); UPG(geo32, m.geo32);
    UPG(geo64, m.geo64); UPG(vt_ptr, m.vt_ptr); UPG(vt_tri, m.vt_tri); UPG(adj_ptr, m.adj_ptr);
    UPG(adj_tri, m.adj_tri); UPG(adj_perm, m.adj_perm); UPG(adj_nbr, m.adj_nbr); UPG(nbr_ptr, m.nbr_ptr);
    UPG(nbr, m.nbr); UPG(colors, colors); UPG(tgrid, A.tg->t); UPG(rule_w64, rw64); UPG(rule_l64, rl64);
    UPG(gl_x, gx); UPG(gl_w, gw); UPG(g_geol, geol); UPG(g_cenh, cenh); UPG(g_cenl, cenl);
    UPG(g_coloff_d, A.color_off); UPG(g_ga_d, A.g_ga); UPG(g_gb_d, A.g_gb); UPG(g_colblk_d, A.g_colblk);
    UPG(g_colk0_d, A.g_colk0); UPG(g_cb2api_d, A.g_cb2api); UPG(g_pan0_d, A.g_pan0); UPG(g_pan64_d, A.g_pan64);
    UPG(g_pan32_d, A.g_pan32); UPG(g_p64_d, A.g_p64); UPG(g_tkb, kb); UPG(g_tib, ib); UPG(g_tr0, r0);
    UPG(g_tdr, dr); UPG(g_tm2, tm2); UPG(g_tm1, tm1);
    for (int k = 1; k <= 3; ++k) {
        std::vector<double> r = sauter_schwab(k, A.opts.near_order);
        A.ss_npp[k] = (int)(r.size() / 5);
        UPG(ss[k], r);
    }
    std::vector<double> dummy(5, 0.0);
    UPG(ss[0], dummy);
#undef UPG
    const size_t njob = kb.size(), nb = A.blocks.size();
    if ((s = dev_alloc(A.g_samples, njob * NCHEB * 2 * sizeof(double), st))) return s;
    if ((s = dev_alloc(A.g_coef, njob * NCHEB * 2 * sizeof(double), st))) return s;
    if ((s = dev_alloc(A.g_coef32, (size_t)A.g_npan * 76 * sizeof(float), st))) return s;
    if ((s = dev_alloc(A.gpair, (size_t)E * E * sizeof(double2), st))) return s;
    if ((s = dev_alloc(A.gvmin, (size_t)M * M * sizeof(double), st))) return s;
    if ((s = dev_alloc(A.gvmax, (size_t)M * M * sizeof(double), st))) return s;
    if ((s = dev_alloc(A.gpartial, 1024 * sizeof(double), st))) return s;
    if ((s = dev_alloc(A.status, 16, st))) return s;
    if ((s = dev_alloc(A.cnt_far, nb * M * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.cnt_near, nb * M * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.rp_far, nb * (M + 1) * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.rp_near, nb * (M + 1) * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.tot_far, nb * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.tot_near, nb * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.off_far_d, nb * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.off_near_d, nb * sizeof(int64_t), st))) return s;
    if ((s = dev_alloc(A.quad_partial, 2048 * sizeof(int64_t), st))) return s;
    CUDA_TRY(cudaStreamSynchronize(st));
    A.nnz_far.assign(nb, -1);
    A.nnz_near.assign(nb, -1);
    A.g_njob32 = (int)njob32;
    return TDBEM_OK;
}

// ---------------------------------------------------------------- C ABI
extern "C" {

const char *tdbem_last_error(void) { return g_err.c_str(); }

tdbem_status tdbem_set_allocator(void *(*alloc)(size_t, void *, void *), void (*free_)(void *, void *, void *),
                                 void *ctx) {
    if ((alloc == nullptr) != (free_ == nullptr)) return fail(TDBEM_E_INVALID_ARG, "alloc and free must both be set or both NULL");
    g_alloc = alloc;
    g_free = free_;
    g_alloc_ctx = ctx;
    return TDBEM_OK;
}

tdbem_status tdbem_mesh_create(const double *verts, int64_t M, const int32_t *tris, int64_t E, tdbem_mesh **out) {
    if (!out) return fail(TDBEM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!verts || !tris || M < 3 || E < 1) return fail(TDBEM_E_INVALID_ARG, "need M >= 3 vertices and E >= 1 triangles");
    if (M > 65535 || E > 65535) return fail(TDBEM_E_UNSUPPORTED, "this build takes M <= 65535 and E <= 65535");
    for (int64_t i = 0; i < 3 * M; ++i)
        if (!std::isfinite(verts[i])) return fail(TDBEM_E_MESH, "non-finite vertex coordinate");
    for (int64_t e = 0; e < E; ++e) {
        for (int a = 0; a < 3; ++a)
            if (tris[3 * e + a] < 0 || tris[3 * e + a] >= M) return fail(TDBEM_E_MESH, "triangle " + std::to_string(e) + " has a vertex index out of range");
        if (tris[3 * e] == tris[3 * e + 1] || tris[3 * e] == tris[3 * e + 2] || tris[3 * e + 1] == tris[3 * e + 2])
            return fail(TDBEM_E_MESH, "triangle " + std::to_string(e) + " repeats a vertex");
    }
    tdbem_mesh *m = new tdbem_mesh();
    m->M = M;
    m->E = E;
    m->V.assign(verts, verts + 3 * M);
    m->F.assign(tris, tris + 3 * E);
    tdbem_status s = build_mesh(*m);
    if (s) { delete m; return s; }
    *out = m;
    return TDBEM_OK;
}

tdbem_status tdbem_timegrid_create(const double *t, int64_t N, int32_t p, int32_t kind, double c, tdbem_timegrid **out) {
    if (!out) return fail(TDBEM_E_INVALID_ARG, "out is NULL");
    *out = nullptr;
    if (!t) return fail(TDBEM_E_INVALID_ARG, "t is NULL");
    if (N < 3) return fail(TDBEM_E_TIMEGRID, "need N >= 3 grid points");
    if (t[0] != 0.0) return fail(TDBEM_E_TIMEGRID, "t[0] must be 0");
    for (int64_t i = 1; i < N; ++i)
        if (!(t[i] > t[i - 1]) || !std::isfinite(t[i])) return fail(TDBEM_E_TIMEGRID, "t must be finite and strictly increasing");
    if (p < 0 || p > 2) return fail(TDBEM_E_UNSUPPORTED, "this build takes temporal degree p = 0, 1 or 2");
    if (kind != 0 && kind != 1) return fail(TDBEM_E_INVALID_ARG, "basis_kind must be 0 (erf(2 artanh)) or 1 (exp(-1/s))");
    if (!(c > 0.0) || !std::isfinite(c)) return fail(TDBEM_E_INVALID_ARG, "wave speed must be positive");
    tdbem_timegrid *g = new tdbem_timegrid();
    g->N = N;
    g->p = p;
    g->kind = kind;
    g->c = c;
    // r = |x - y| / c: scale time by c so the kernels work with c = 1
    g->t.resize(N);
    for (int64_t i = 0; i < N; ++i) g->t[i] = t[i] * c;
    g->T = g->t[N - 1];
    g->dt = g->T / (double)(N - 1);
    g->equidistant = true;
    for (int64_t i = 0; i < N; ++i)
        if (fabs(g->t[i] - i * g->dt) > 1e-12 * g->T) g->equidistant = false;
    *out = g;
    return TDBEM_OK;
}

void tdbem_mesh_destroy(tdbem_mesh *m) { delete m; }
void tdbem_timegrid_destroy(tdbem_timegrid *t) { delete t; }
void tdbem_asm_destroy(tdbem_asm *a) { delete a; }

tdbem_status tdbem_assembler_create(const tdbem_mesh *mesh, const tdbem_timegrid *tg, const tdbem_opts *opts,
                                    void *stream, tdbem_asm **out) {
    if (!out || !mesh || !tg) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (tg->N < 5 || tg->N > 1000) return fail(TDBEM_E_UNSUPPORTED, "need 5 <= N <= 1000 grid points");
    if (tg->c != 1.0 && tg->c <= 0.0) return fail(TDBEM_E_INVALID_ARG, "bad wave speed");
    tdbem_opts o{};
    o.precision = TDBEM_PREC_MIXED;
    o.near_order = 4;
    o.cheb_degree = 32;
    if (opts) o = *opts;
    if (o.precision != TDBEM_PREC_FP64 && o.precision != TDBEM_PREC_MIXED) return fail(TDBEM_E_INVALID_ARG, "precision");
    if (o.near_order < 1 || o.near_order > 5) return fail(TDBEM_E_INVALID_ARG, "near_order must be in 1..5");
    if (o.cheb_degree != 32) return fail(TDBEM_E_UNSUPPORTED, "cheb_degree must be 32");
    if (o.staging_mb < 0) return fail(TDBEM_E_INVALID_ARG, "staging_mb must be >= 0");
    cudaStream_t st = (cudaStream_t)stream;
    tdbem_asm *A = new tdbem_asm();
    A->mesh = mesh;
    A->tg = tg;
    A->opts = o;
    A->fp64 = o.precision == TDBEM_PREC_FP64;
    auto bail = [&](tdbem_status s) { delete A; return s; };
    // non-equidistant grids, and p >= 1 on any grid: every nonzero block
    // (and order pair) assembled from its own psi
    if (!tg->equidistant || tg->p > 0) {
        tdbem_status gs = create_graded(*A, st);
        if (gs) return bail(gs);
        *out = A;
        return TDBEM_OK;
    }
    tdbem_status s = plan_blocks(*A);
    if (s) return bail(s);
    const double dt = tg->dt;
    const double spread = 2.0 * mesh->max_dq / dt;
    A->OFF = (int)ceil(spread + 1e-9);
    if (A->OFF < 1) A->OFF = 1;
    if (A->OFF > 3) return bail(fail(TDBEM_E_UNSUPPORTED, "triangles too large for the time step (2 max|x - c|/dt > 3)"));
    if (!A->fp64 && far32_window(mesh->max_dq, dt) > 5)
        return bail(fail(TDBEM_E_UNSUPPORTED, "mixed precision: triangles too large for the time step"));
    A->KW = 4 + (int)ceil(2.0 * mesh->max_star / dt) + 2;
    if (A->KW > 16) return bail(fail(TDBEM_E_UNSUPPORTED, "vertex stars too large for the time step (lag window > 16)"));
    if (!A->fp64 && 3.0 * (double)mesh->M * (double)mesh->M >= 2147483647.0)
        return bail(fail(TDBEM_E_UNSUPPORTED, "mixed precision: 3 M^2 lag-window rows exceed the int32 row index"));
    if (!A->fp64 && far32_smem(far32_window(mesh->max_dq, dt), A->KW, mesh->max_nv) > 227 * 1024)
        return bail(fail(TDBEM_E_UNSUPPORTED, "mixed precision: far-kernel shared memory exceeds 227 KB"));
    const tdbem_mesh &m = *mesh;
    // uploads; the colouring rebalanced for the far kernel's grid on this device
    int nsm_dev = 0;
    {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e == cudaSuccess) e = cudaDeviceGetAttribute(&nsm_dev, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return bail(fail(TDBEM_E_CUDA, std::string("device attributes: ") + cudaGetErrorString(e)));
    }
    const int far_grid = (A->fp64 || far32_window(m.max_dq, dt) > 2) ? nsm_dev : 2 * nsm_dev;
    const std::vector<std::vector<int32_t>> bal = balance_colours(m, far_grid);
    std::vector<int32_t> colors;
    A->color_off.assign(1, 0);
    for (auto &c : bal) { colors.insert(colors.end(), c.begin(), c.end()); A->color_off.push_back((int64_t)colors.size()); }
    std::vector<float> rw(7), rl(21);
    for (int k = 0; k < 7; ++k) { rw[k] = (float)m.rule_W[k]; for (int d = 0; d < 3; ++d) rl[3 * k + d] = (float)m.rule_L[k][d]; }
#define UP(buf, vec) if ((s = upload(A->buf, vec, st))) return bail(s)
    UP(F, m.F); UP(V, m.V); UP(cen, m.cen); UP(dq, m.dq); UP(dq32, m.dq32); UP(geo32, m.geo32); UP(geo64, m.geo64);
    UP(vt_ptr, m.vt_ptr); UP(vt_tri, m.vt_tri); UP(adj_ptr, m.adj_ptr); UP(adj_tri, m.adj_tri);
    UP(adj_perm, m.adj_perm); UP(adj_nbr, m.adj_nbr); UP(nbr_ptr, m.nbr_ptr); UP(nbr, m.nbr);
    UP(chunk_vptr, m.chunk_vptr); UP(chunk_vert, m.chunk_vert); UP(chunk_sptr, m.chunk_sptr);
    {
        std::vector<int32_t> hdr(4 * m.nchunks);
        for (int64_t ch = 0; ch < m.nchunks; ++ch) {
            const int32_t v0 = m.chunk_vptr[ch], v1 = m.chunk_vptr[ch + 1];
            hdr[4 * ch] = v0; hdr[4 * ch + 1] = v1 - v0;
            hdr[4 * ch + 2] = m.chunk_sptr[v0]; hdr[4 * ch + 3] = m.chunk_sptr[v1] - m.chunk_sptr[v0];
        }
        UP(chunk_hdr, hdr);
    }
    UP(chunk_src, m.chunk_src); UP(colors, colors); UP(rule_w, rw); UP(rule_l, rl); UP(tgrid, tg->t);
    {
        std::vector<float> geol(16 * m.E), cenh(3 * m.E), cenl(3 * m.E);
        for (int64_t k = 0; k < 16 * m.E; ++k) geol[k] = (float)(m.geo64[k] - (double)m.geo32[k]);
        for (int64_t k = 0; k < 3 * m.E; ++k) {
            cenh[k] = (float)m.cen[k];
            cenl[k] = (float)(m.cen[k] - (double)cenh[k]);
        }
        UP(g_geol, geol); UP(g_cenh, cenh); UP(g_cenl, cenl);
    }
    std::vector<double> rw64(7), rl64(21);
    for (int k = 0; k < 7; ++k) { rw64[k] = m.rule_W[k]; for (int d = 0; d < 3; ++d) rl64[3 * k + d] = m.rule_L[k][d]; }
    UP(rule_w64, rw64); UP(rule_l64, rl64);
    std::vector<double> la, lb;
    std::vector<int> loff(NCLASS + 1, 0);
    for (int c = 0; c < NCLASS; ++c) {
        la.insert(la.end(), A->lag_a[c].begin(), A->lag_a[c].end());
        lb.insert(lb.end(), A->lag_b[c].begin(), A->lag_b[c].end());
        loff[c + 1] = (int)la.size();
    }
    UP(lagA, la); UP(lagB, lb);
    std::vector<int> cdlo(A->cls_dlo, A->cls_dlo + NCLASS), cdhi(A->cls_dhi, A->cls_dhi + NCLASS);
    UP(cls_dlo_d, cdlo); UP(cls_dhi_d, cdhi); UP(blk_of_lag_d, A->blk_of_lag); UP(lag_base_d, A->lag_base);
    UP(blk_of_spec_d, A->blk_of_spec);
    // psi table jobs: every panel of every class at 1 (FP32) and S64 (FP64) sub-panels
    {
        std::vector<int> kb, ib;
        std::vector<double> r0;
        const int64_t N = tg->N;
        for (int S : {1, A->S64}) {
            for (int c = 0; c < NCLASS; ++c) {
                int rk, ri, dr;
                switch (c) {
                    case C1: rk = 2; ri = 0; dr = 2; break;
                    case C2: rk = 3; ri = 1; dr = 2; break;
                    case C3: rk = (int)N - 1; ri = (int)N - 3; dr = 2; break;
                    case S00: rk = 0; ri = 0; dr = 0; break;
                    case S01: rk = 0; ri = 1; dr = 0; break;
                    case SN0: rk = (int)N - 1; ri = 0; dr = 0; break;
                    case SNN: rk = (int)N - 1; ri = (int)N - 1; dr = 0; break;
                    default: rk = (int)N - 2; ri = (int)N - 1; dr = 0; break;
                }
                for (int j = 0; j < A->cls_P[c]; ++j)
                    for (int sb = 0; sb < S; ++sb) {
                        kb.push_back(rk);
                        ib.push_back(ri);
                        r0.push_back((dr + A->cls_rho[c] + j + (double)sb / S) * dt);
                    }
            }
        }
        UP(tab_kb, kb); UP(tab_ib, ib); UP(tab_r0, r0);
        std::vector<double> gx, gw;
        gauss_legendre01(24, gx, gw);
        UP(gl_x, gx); UP(gl_w, gw);
        if ((s = dev_alloc(A->tab_samples, kb.size() * NCHEB * 2 * sizeof(double), st))) return bail(s);
        if ((s = dev_alloc(A->tab_coef1, TOTAL_PANELS * NCHEB * 2 * sizeof(double), st))) return bail(s);
        if ((s = dev_alloc(A->tab_coef4, (size_t)TOTAL_PANELS * A->S64 * NCHEB * 2 * sizeof(double), st))) return bail(s);
    }
    for (int k = 1; k <= 3; ++k) {
        std::vector<double> r = sauter_schwab(k, o.near_order);
        A->ss_npp[k] = (int)(r.size() / 5);
        UP(ss[k], r);
    }
    std::vector<double> dummy(5, 0.0);
    UP(ss[0], dummy);
#undef UP
    const int64_t M = m.M, E = m.E;
    const size_t MM = (size_t)M * M;
    const size_t rs = A->fp64 ? 8 : 4;
    if ((s = dev_alloc(A->rec, (size_t)E * E * sizeof(PairRec), st))) return bail(s);
    // pairs whose FP32 lag decision is not certain, decided by a dense FP64 pass
    A->pb_cap = std::min<int64_t>(std::max<int64_t>(PB_LIST_MIN, E * E / 64), std::max<int64_t>(E * E, 1));
    if ((s = dev_alloc(A->pb_list, (size_t)A->pb_cap * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->pb_cnt, 16, st))) return bail(s);
    if ((s = dev_alloc(A->wdlo, 3 * MM * sizeof(int16_t), st))) return bail(s);
    if ((s = dev_alloc(A->wdhi, 3 * MM * sizeof(int16_t), st))) return bail(s);
    if ((s = dev_alloc(A->wsmask, MM, st))) return bail(s);
    if ((s = dev_alloc(A->dense, 3 * MM * A->KW * sizeof(double), st))) return bail(s);
    if ((s = dev_alloc(A->dense_spec, NSPEC * MM * sizeof(double), st))) return bail(s);
    (void)rs;
    if ((s = dev_alloc(A->ndense, (size_t)3 * M * m.NB * A->KW * sizeof(double), st))) return bail(s);
    if ((s = dev_alloc(A->ndense_spec, (size_t)NSPEC * M * m.NB * sizeof(double), st))) return bail(s);
    if ((s = dev_alloc(A->status, 16, st))) return bail(s);
    const size_t nb = A->blocks.size();
    {
        bool has_c2 = false;
        for (const Block &b : A->blocks) has_c2 |= b.cls == C2;
        A->tw_on = !A->fp64 && A->only_k < 0 && has_c2 && tg->N >= 3;
        if (A->tw_on) {
            if ((s = dev_alloc(A->tw_cnt, 2 * M * sizeof(int64_t), st))) return bail(s);
            if ((s = dev_alloc(A->tw_ptr, 2 * (M + 1) * sizeof(int64_t), st))) return bail(s);
            if ((s = dev_alloc(A->tw_tot, 4 * sizeof(int64_t), st))) return bail(s);
        }
    }
    if ((s = dev_alloc(A->cnt_far, nb * M * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->cnt_near, nb * M * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->rp_far, nb * (M + 1) * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->rp_near, nb * (M + 1) * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->tot_far, nb * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->tot_near, nb * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->off_far_d, nb * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->off_near_d, nb * sizeof(int64_t), st))) return bail(s);
    if ((s = dev_alloc(A->quad_partial, 1024 * sizeof(int64_t), st))) return bail(s);
    CUDA_TRY(cudaStreamSynchronize(st));
    A->nnz_far.assign(nb, -1);
    A->nnz_near.assign(nb, -1);
    *out = A;
    return TDBEM_OK;
}

tdbem_status tdbem_num_blocks(const tdbem_asm *a, int64_t *n) {
    if (!a || !n) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    *n = (int64_t)a->blocks.size();
    return TDBEM_OK;
}

tdbem_status tdbem_block_info(const tdbem_asm *a, int64_t b, int32_t *k, int32_t *i, int32_t *m2, int32_t *m1,
                              int64_t *nf, int64_t *nn) {
    if (!a) return fail(TDBEM_E_INVALID_ARG, "NULL assembler");
    if (b == TDBEM_LAST_BLOCK) {
        if (!a->single || !a->single->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_block first");
        return tdbem_block_info(a->single, 0, k, i, m2, m1, nf, nn);
    }
    if (b < 0 || b >= (int64_t)a->blocks.size()) return fail(TDBEM_E_INVALID_ARG, "block index out of range");
    if (k) *k = a->blocks[b].kb;
    if (i) *i = a->blocks[b].ib;
    if (m2) *m2 = a->blocks[b].m2;
    if (m1) *m1 = a->blocks[b].m1;
    if (nf) *nf = a->nnz_far[b];
    if (nn) *nn = a->nnz_near[b];
    return TDBEM_OK;
}

static Geo make_geo(tdbem_asm *A) {
    Geo g;
    g.M = A->mesh->M; g.E = A->mesh->E;
    g.F = (const int32_t *)A->F.p; g.cen = (const double *)A->cen.p; g.dq = (const double *)A->dq.p;
    g.dq32 = (const float *)A->dq32.p; g.V = (const double *)A->V.p; g.geo32 = (const float *)A->geo32.p;
    g.geo64 = (const double *)A->geo64.p; g.vt_ptr = (const int64_t *)A->vt_ptr.p; g.vt_tri = (const int32_t *)A->vt_tri.p;
    return g;
}

static LagTables make_lt(tdbem_asm *A) {
    LagTables lt;
    int off = 0;
    for (int c = 0; c < NCLASS; ++c) {
        lt.a[c] = (const double *)A->lagA.p + off;
        lt.b[c] = (const double *)A->lagB.p + off;
        off += (int)A->lag_a[c].size();
        lt.dlo[c] = A->cls_dlo[c];
        lt.dhi[c] = A->cls_dhi[c];
        lt.rho[c] = A->cls_rho[c];
        lt.P[c] = A->cls_P[c];
    }
    lt.dt = A->tg->dt;
    lt.inv_dt = 1.0 / A->tg->dt;
    lt.tie = 1e-12 * A->tg->T;
    // FP32 squared distances of points with |coordinate| <= L carry an absolute
    // error of a few ulp(L^2); take 64 ulps of 4 L^2 as the band
    lt.tol2 = 64.0 * 4.0 * A->mesh->coord_scale * A->mesh->coord_scale * 1.1920928955078125e-07;
    return lt;
}

// Diagonal run of block positions that unique block (k, i) stands for
// (0-based; Eq. relationAtildeBlock holds for 1 <= k, i <= N-2): the inner
// blocks of the second block column repeat down their diagonal, block (1, 2)
// along the superdiagonal, every other listed block is used once.
static void block_run(int64_t k, int64_t i, int64_t N, int32_t &k0, int32_t &i0, int32_t &cnt) {
    k0 = (int32_t)k;
    i0 = (int32_t)i;
    cnt = 1;
    if (i == 1 && k >= 1 && k <= N - 2) cnt = (int32_t)(N - 1 - k);
    else if (k == 1 && i == 2) cnt = (int32_t)(N - 3);
}

// widest lag range of a lag class: the CSR fill keeps one position per lag
static int fill_lag_span(const tdbem_asm *A) {
    int n = 1;
    for (int c = 0; c < NLAG; ++c) n = std::max(n, A->lag_base[c + 1] - A->lag_base[c]);
    return n;
}

static tdbem_status plan_matvec(tdbem_asm &A, cudaStream_t st) {
    const int64_t N = A.tg->N, M = A.mesh->M, P1 = A.tg->p + 1, L = N * P1;
    const size_t nb = A.blocks.size();
    A.mv_host.assign(nb, MvBlock{});
    for (size_t b = 0; b < nb; ++b) {
        MvBlock &d = A.mv_host[b];
        d.rp_far = (const int64_t *)A.rp_far.p + b * (M + 1);
        d.col_far = (const int32_t *)A.col_far.p + A.off_far[b];
        d.val_far = (const char *)A.val_far.p + A.off_far[b] * (A.fp64 ? 8 : 4);
        d.rp_near = (const int64_t *)A.rp_near.p + b * (M + 1);
        d.col_near = (const int32_t *)A.col_near.p + A.off_near[b];
        d.val_near = (const double *)A.val_near.p + A.off_near[b];
        block_run(A.blocks[b].kb, A.blocks[b].ib, N, d.k0, d.i0, d.cnt);
        if (A.graded) {
            // every block stands only for itself, at row k (p + 1) + m2 and
            // column i (p + 1) + m1 of the time functions
            d.k0 = (int32_t)(A.blocks[b].kb * P1 + A.blocks[b].m2);
            d.i0 = (int32_t)(A.blocks[b].ib * P1 + A.blocks[b].m1);
            d.cnt = 1;
        }
    }
    A.mv_rest_host.clear();
    if (A.tw_on)
        for (size_t b = 0; b < nb; ++b)
            if (A.blocks[b].cls != C2) A.mv_rest_host.push_back(A.mv_host[b]);
    tdbem_status s;
    if ((s = upload(A.mv_blk, A.mv_host, st))) return s;
    if (A.tw_on && !A.mv_rest_host.empty())
        if ((s = upload(A.mv_rest, A.mv_rest_host, st))) return s;
    const size_t xbytes = std::max((size_t)(L * M) * sizeof(double), (size_t)(A.tw_on ? 4 * M * A.tw_S : 0) * sizeof(float));
    if (A.mv_xT.n < xbytes)
        if ((s = dev_alloc(A.mv_xT, xbytes, st))) return s;
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDBEM_OK;
}

// The whole device sequence of one assembly. Eager (capture == false): with
// the host steps between its parts (FP32 copy of the psi coefficients, CSR
// sizes, allocation and offsets, status word, statistics). capture == true:
// the device work only, to be recorded into a CUDA graph; everything the host
// computed is then known from the eager run (same mesh and time grid give the
// same tables, pattern and sizes).
// Per-pair lag windows of the Toeplitz class for the mixed matvec, from the
// window bounds and the far (FP32 pairs) and near (FP64) windows the assembly
// has just accumulated. Eager: counts, scan, sizes and the widest window to
// the host (which fix the lags per entry and the x-copy geometry), buffers
// grown if needed, fill. capture: the device work with the sizes of the
// eager run.
static tdbem_status build_toeplitz(tdbem_asm *A, bool capture, cudaStream_t st) {
    if (!A->tw_on) return TDBEM_OK;
    const int64_t M = A->mesh->M, NB = A->mesh->NB;
    const size_t MM = (size_t)M * M;
    const int16_t *dlo = (const int16_t *)A->wdlo.p + C2 * MM, *dhi = (const int16_t *)A->wdhi.p + C2 * MM;
    int64_t *tot = (int64_t *)A->tw_tot.p;
    CUDA_TRY(cudaMemsetAsync(tot + 2, 0, sizeof(int64_t), st));
    launch_tw_count(M, dlo, dhi, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p, (int64_t *)A->tw_cnt.p,
                    (unsigned long long *)(tot + 2), st);
    launch_scan_rows((const int64_t *)A->tw_cnt.p, M, 2, (int64_t *)A->tw_ptr.p, tot, st);
    if (!capture) {
        int64_t h[3] = {0, 0, 0};
        CUDA_TRY(cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        A->tw_nfar = h[0];
        A->tw_nnear = h[1];
        const int TL = tw_lags((int)std::max<int64_t>(h[2], 1));
        if (TL < 0) return fail(TDBEM_E_DEVICE, "Toeplitz-class lag window wider than 16 lags");
        A->tw_TL = TL;
        tw_geometry(TL, A->cls_dhi[C2], (int)A->tg->N, &A->tw_PADL, &A->tw_S);
        const int TS = (TL + 3) / 4 * 4;
        tdbem_status s;
        if ((size_t)h[0] * TS > A->tw_cap_far || !A->tw_fhdr.p) {
            if ((s = dev_alloc(A->tw_fhdr, std::max<int64_t>(h[0], 1) * sizeof(int2), st))) return s;
            if ((s = dev_alloc(A->tw_fval, std::max<int64_t>(h[0], 1) * TS * sizeof(float), st))) return s;
            A->tw_cap_far = (size_t)h[0] * TS;
        }
        if ((size_t)h[1] * TS > A->tw_cap_near || !A->tw_nhdr.p) {
            if ((s = dev_alloc(A->tw_nhdr, std::max<int64_t>(h[1], 1) * sizeof(int2), st))) return s;
            if ((s = dev_alloc(A->tw_nval, std::max<int64_t>(h[1], 1) * TS * sizeof(double), st))) return s;
            A->tw_cap_near = (size_t)h[1] * TS;
        }
    }
    launch_tw_fill(M, dlo, dhi, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p, A->tw_TL,
                   (const int64_t *)A->tw_ptr.p, (const float2 *)A->dense.p + C2 * MM * A->KW,
                   (const double *)A->ndense.p + (size_t)C2 * M * NB * A->KW, A->KW, (int)NB, (int2 *)A->tw_fhdr.p,
                   (float *)A->tw_fval.p, (int2 *)A->tw_nhdr.p, (double *)A->tw_nval.p, st);
    CUDA_TRY(cudaGetLastError());
    return TDBEM_OK;
}

static tdbem_status assemble_body(tdbem_asm *A, cudaStream_t st, bool capture) {
    const tdbem_mesh &m = *A->mesh;
    const int64_t M = m.M, E = m.E;
    const size_t MM = (size_t)M * M;
    const size_t rs = A->fp64 ? 8 : 4;
    const size_t nb = A->blocks.size();
    (void)MM;
    for (auto &e : A->ev)
        if (!e) CUDA_TRY(cudaEventCreate(&e));
    cudaEvent_t *ev = A->ev;
    // phase boundaries: timing events when eager; when capturing, each phase
    // becomes its own graph so the replay can put timing events between them
    auto mark = [&](int k) -> cudaError_t {
        if (!capture) return cudaEventRecord(ev[k], st);
        cudaError_t e = cudaSuccess;
        if (k > 0) {
            cudaGraph_t gr = nullptr;
            e = cudaStreamEndCapture(st, &gr);
            if (e == cudaSuccess) e = cudaGraphInstantiate(&A->gexec[k - 1], gr, 0);
            if (gr) cudaGraphDestroy(gr);
            if (e != cudaSuccess) return e;
        }
        if (k < 4) e = cudaStreamBeginCapture(st, cudaStreamCaptureModeRelaxed);
        return e;
    };
    CUDA_TRY(mark(0));
    CUDA_TRY(cudaMemsetAsync(A->status.p, 0, 16, st));
    CUDA_TRY(cudaMemsetAsync(A->dense.p, 0, A->dense.n, st));
    CUDA_TRY(cudaMemsetAsync(A->dense_spec.p, 0, A->dense_spec.n, st));
    CUDA_TRY(cudaMemsetAsync(A->ndense.p, 0, A->ndense.n, st));
    CUDA_TRY(cudaMemsetAsync(A->ndense_spec.p, 0, A->ndense_spec.n, st));
    // ---- psi tables (FP64 samples, Chebyshev coefficients)
    const int n1 = TOTAL_PANELS, n4 = TOTAL_PANELS * A->S64;
    launch_psi_samples(A->tg->kind, (const double *)A->tgrid.p, (int)A->tg->N, nullptr, (const int *)A->tab_kb.p,
                       (const int *)A->tab_ib.p, (const double *)A->tab_r0.p, A->tg->dt, 1, n1,
                       (const double *)A->gl_x.p, (const double *)A->gl_w.p, 24, 8, (double *)A->tab_samples.p, st);
    launch_psi_dct((const double *)A->tab_samples.p, n1, (double *)A->tab_coef1.p, st);
    launch_psi_samples(A->tg->kind, (const double *)A->tgrid.p, (int)A->tg->N, nullptr, (const int *)A->tab_kb.p + n1,
                       (const int *)A->tab_ib.p + n1, (const double *)A->tab_r0.p + n1, A->tg->dt / A->S64, A->S64,
                       n4, (const double *)A->gl_x.p, (const double *)A->gl_w.p, 24, 8,
                       (double *)A->tab_samples.p + (size_t)n1 * NCHEB * 2, st);
    launch_psi_dct((const double *)A->tab_samples.p + (size_t)n1 * NCHEB * 2, n4, (double *)A->tab_coef4.p, st);
    CUDA_TRY(cudaGetLastError());
    if (!capture) {
        std::vector<double> c1((size_t)n1 * NCHEB * 2);
        CUDA_TRY(cudaMemcpyAsync(c1.data(), A->tab_coef1.p, c1.size() * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        for (int p = 0; p < n1; ++p)
            for (int n = 0; n < NCHEB; ++n)
                for (int k = 0; k < 2; ++k) {
                    const double v = c1[((size_t)p * NCHEB + n) * 2 + k];
                    A->c32.c[p][n][k] = (float)v;
                    if (n < NCHEB_LO) A->c32.lo[p][n][k] = (float)(v - (double)(float)v);
                    const float sg = (n & 2) ? -1.f : 1.f;
                    if (p < TOTAL_LAG_PANELS) {
                        A->c32s.c[n][p][k] = sg * A->c32.c[p][n][k];
                        if (n < NCHEB_LO) A->c32s.lo[n][p][k] = sg * A->c32.lo[p][n][k];
                    }
                }
    }
    // ---- element-pair bounds, vertex-pair windows
    Geo g = make_geo(A);
    LagTables lt = make_lt(A);
    {
        int dev = 0, nsm0 = 0;
        CUDA_TRY(cudaGetDevice(&dev));
        CUDA_TRY(cudaDeviceGetAttribute(&nsm0, cudaDevAttrMultiProcessorCount, dev));
        launch_pair_bounds(g, lt, (PairRec *)A->rec.p, (int64_t *)A->pb_list.p, A->pb_cap,
                           (unsigned long long *)A->pb_cnt.p, (int *)A->status.p, nsm0, st);
    }
    launch_vertex_windows(g, (const PairRec *)A->rec.p, (int16_t *)A->wdlo.p, (int16_t *)A->wdhi.p,
                          (uint8_t *)A->wsmask.p, A->KW, (int *)A->status.p, st);
    {
        const int npp[4] = {49, A->ss_npp[1], A->ss_npp[2], A->ss_npp[3]};
        launch_count_quad(g, (const PairRec *)A->rec.p, npp, (int64_t *)A->quad_partial.p, 1024, st);
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(mark(1));
    // ---- far field, one launch per colour
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    for (size_t c = 0; c + 1 < A->color_off.size(); ++c) {
        FarArgs fa;
        fa.g = g; fa.lt = lt;
        fa.dlo = (const int16_t *)A->wdlo.p; fa.dhi = (const int16_t *)A->wdhi.p; fa.smask = (const uint8_t *)A->wsmask.p;
        fa.color_tris = (const int32_t *)A->colors.p + A->color_off[c];
        fa.ncolor = A->color_off[c + 1] - A->color_off[c];
        fa.chunk_vptr = (const int32_t *)A->chunk_vptr.p; fa.chunk_vert = (const int32_t *)A->chunk_vert.p;
        fa.chunk_sptr = (const int32_t *)A->chunk_sptr.p; fa.chunk_src = (const int32_t *)A->chunk_src.p;
        fa.chunk_hdr = (const int4 *)A->chunk_hdr.p;
        fa.nchunks = m.nchunks;
        fa.max_nv = m.max_nv;
        fa.rule_w = (const float *)A->rule_w.p; fa.rule_l = (const float *)A->rule_l.p;
        fa.rule_w64 = (const double *)A->rule_w64.p; fa.rule_l64 = (const double *)A->rule_l64.p;
        fa.dense = (double *)A->dense.p; fa.dense_spec = (double *)A->dense_spec.p; fa.KW = A->KW;
        fa.status = (int *)A->status.p;
        fa.cheb64 = (const double *)A->tab_coef4.p;
        fa.cenh = (const float *)A->g_cenh.p; fa.cenl = (const float *)A->g_cenl.p;
        fa.geoh = (const float *)A->geo32.p; fa.geol = (const float *)A->g_geol.p;
        for (int k = 0; k < 7; ++k) {
            fa.rw32[k] = (float)m.rule_W[k];
            fa.wwh[k] = (float)m.rule_W[k];
            fa.wwl[k] = (float)(m.rule_W[k] - (double)fa.wwh[k]);
            if (k == 0 || k == 1 || k == 4) {
                const int o = k == 0 ? 0 : (k == 1 ? 1 : 2);
                // a = corner 1 of point k (0 on orbits 1, 2; any at the centroid) is a non-distinguished corner
                const double kk = m.rule_W[k] * m.rule_L[k][k == 0 ? 0 : 1];
                fa.okh[o] = (float)kk; fa.okl[o] = (float)(kk - (double)fa.okh[o]);
                fa.owh[o] = (float)m.rule_W[k]; fa.owl[o] = (float)(m.rule_W[k] - (double)fa.owh[o]);
                if (o > 0) {
                    const double dd = m.rule_W[k] * (m.rule_L[k][0] - m.rule_L[k][1]);
                    fa.odh[o - 1] = (float)dd; fa.odl[o - 1] = (float)(dd - (double)fa.odh[o - 1]);
                }
            }
            for (int d = 0; d < 3; ++d) {
                fa.rl32[3 * k + d] = (float)m.rule_L[k][d];
                const double gw = m.rule_W[k] * m.rule_L[k][d];
                fa.gwh[3 * k + d] = (float)gw;
                fa.gwl[3 * k + d] = (float)(gw - (double)fa.gwh[3 * k + d]);
            }
        }
        const int grid = (int)std::min<int64_t>(fa.ncolor, (int64_t)(A->fp64 ? 1 : 2) * nsm);
        if (grid > 0) {
            if (A->fp64) launch_far(fa, A->c32, true, A->OFF, A->S64, grid, st);
            else launch_far32(fa, A->c32s, far32_window(m.max_dq, A->tg->dt), grid, st);
        }
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(mark(2));
    // ---- near field, one launch per colour
    for (size_t c = 0; c + 1 < A->color_off.size(); ++c) {
        NearArgs na;
        na.g = g; na.lt = lt;
        na.dlo = (const int16_t *)A->wdlo.p; na.dhi = (const int16_t *)A->wdhi.p;
        na.color_tris = (const int32_t *)A->colors.p + A->color_off[c];
        na.ncolor = A->color_off[c + 1] - A->color_off[c];
        na.adj_ptr = (const int64_t *)A->adj_ptr.p; na.adj_tri = (const int32_t *)A->adj_tri.p;
        na.adj_perm = (const int8_t *)A->adj_perm.p; na.adj_nbr = (const int32_t *)A->adj_nbr.p;
        na.rec = (const PairRec *)A->rec.p;
        for (int k = 0; k < 4; ++k) { na.ss_xy[k] = (const double *)A->ss[k].p; na.ss_npp[k] = A->ss_npp[k]; }
        na.cheb64 = (const double *)A->tab_coef4.p;
        na.S = A->S64;
        na.ndense = (double *)A->ndense.p; na.ndense_spec = (double *)A->ndense_spec.p;
        na.NB = m.NB; na.KW = A->KW;
        na.status = (int *)A->status.p;
        na.far_spec = (double *)A->dense_spec.p;
        na.smask = (const uint8_t *)A->wsmask.p;
        na.rule_w64 = (const double *)A->rule_w64.p; na.rule_l64 = (const double *)A->rule_l64.p;
        const int grid = (int)std::min<int64_t>(na.ncolor, (int64_t)(A->fp64 ? 2 : 3) * nsm);
        if (grid > 0) {
            if (A->fp64) launch_near(na, grid, st);
            else launch_near32(na, A->c32, grid, st);
            // mixed: the far pairs of the special blocks, FP64 (the FP32 kernel skips them)
            if (!A->fp64) launch_farspec32(na, A->c32, (int)std::min<int64_t>(na.ncolor, (int64_t)8 * nsm), st);
        }
    }
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(mark(3));
    // ---- CSR: row counts, offsets, sizes, fill
    launch_row_counts2(M, (const int16_t *)A->wdlo.p, (const int16_t *)A->wdhi.p, (const uint8_t *)A->wsmask.p,
                       (const int *)A->cls_dlo_d.p, (const int *)A->cls_dhi_d.p, (const int *)A->blk_of_lag_d.p,
                       (const int *)A->lag_base_d.p, (const int *)A->blk_of_spec_d.p, (const int64_t *)A->nbr_ptr.p,
                       (const int32_t *)A->nbr.p, (int64_t *)A->cnt_far.p, (int64_t *)A->cnt_near.p, st);
    launch_scan_rows((const int64_t *)A->cnt_far.p, M, (int)nb, (int64_t *)A->rp_far.p, (int64_t *)A->tot_far.p, st);
    launch_scan_rows((const int64_t *)A->cnt_near.p, M, (int)nb, (int64_t *)A->rp_near.p, (int64_t *)A->tot_near.p, st);
    CUDA_TRY(cudaGetLastError());
    if (capture) {
        // sizes, buffers and offsets are those of the eager run
        launch_fill(M, (const int16_t *)A->wdlo.p, (const int16_t *)A->wdhi.p, (const uint8_t *)A->wsmask.p,
                    (const int *)A->cls_dlo_d.p, (const int *)A->blk_of_lag_d.p, (const int *)A->lag_base_d.p,
                    (const int *)A->blk_of_spec_d.p, nullptr, nullptr, (const int64_t *)A->rp_far.p,
                    (const int64_t *)A->off_far_d.p, (int32_t *)A->col_far.p, (const double *)A->dense.p,
                    (const double *)A->dense_spec.p, A->val_far.p, A->KW, 0, A->fp64, fill_lag_span(A), st);
        launch_fill(M, (const int16_t *)A->wdlo.p, (const int16_t *)A->wdhi.p, (const uint8_t *)A->wsmask.p,
                    (const int *)A->cls_dlo_d.p, (const int *)A->blk_of_lag_d.p, (const int *)A->lag_base_d.p,
                    (const int *)A->blk_of_spec_d.p, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p,
                    (const int64_t *)A->rp_near.p, (const int64_t *)A->off_near_d.p, (int32_t *)A->col_near.p,
                    (const double *)A->ndense.p, (const double *)A->ndense_spec.p, A->val_near.p, A->KW, m.NB, true,
                    fill_lag_span(A), st);
        CUDA_TRY(cudaGetLastError());
        tdbem_status ts = build_toeplitz(A, true, st);
        if (ts) return ts;
        CUDA_TRY(mark(4));
        return TDBEM_OK;
    }
    A->nnz_far.assign(nb, 0);
    A->nnz_near.assign(nb, 0);
    std::vector<int64_t> qp(1024);
    CUDA_TRY(cudaMemcpyAsync(A->nnz_far.data(), A->tot_far.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(A->nnz_near.data(), A->tot_near.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(qp.data(), A->quad_partial.p, 1024 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    A->off_far.assign(nb + 1, 0);
    A->off_near.assign(nb + 1, 0);
    for (size_t b = 0; b < nb; ++b) {
        A->off_far[b + 1] = A->off_far[b] + A->nnz_far[b];
        A->off_near[b + 1] = A->off_near[b] + A->nnz_near[b];
    }
    tdbem_status s;
    if ((size_t)A->off_far[nb] > A->col_far_cap || A->col_far.p == nullptr) {
        if ((s = dev_alloc(A->col_far, A->off_far[nb] * sizeof(int32_t), st))) return s;
        if ((s = dev_alloc(A->val_far, A->off_far[nb] * rs, st))) return s;
        A->col_far_cap = A->off_far[nb];
    }
    if ((size_t)A->off_near[nb] > A->col_near_cap || A->col_near.p == nullptr) {
        if ((s = dev_alloc(A->col_near, A->off_near[nb] * sizeof(int32_t), st))) return s;
        if ((s = dev_alloc(A->val_near, A->off_near[nb] * sizeof(double), st))) return s;
        A->col_near_cap = A->off_near[nb];
    }
    CUDA_TRY(cudaMemcpyAsync(A->off_far_d.p, A->off_far.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(A->off_near_d.p, A->off_near.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    launch_fill(M, (const int16_t *)A->wdlo.p, (const int16_t *)A->wdhi.p, (const uint8_t *)A->wsmask.p,
                (const int *)A->cls_dlo_d.p, (const int *)A->blk_of_lag_d.p, (const int *)A->lag_base_d.p,
                (const int *)A->blk_of_spec_d.p, nullptr, nullptr, (const int64_t *)A->rp_far.p,
                (const int64_t *)A->off_far_d.p, (int32_t *)A->col_far.p, (const double *)A->dense.p,
                (const double *)A->dense_spec.p, A->val_far.p,
                A->KW, 0, A->fp64, fill_lag_span(A), st);
    launch_fill(M, (const int16_t *)A->wdlo.p, (const int16_t *)A->wdhi.p, (const uint8_t *)A->wsmask.p,
                (const int *)A->cls_dlo_d.p, (const int *)A->blk_of_lag_d.p, (const int *)A->lag_base_d.p,
                (const int *)A->blk_of_spec_d.p, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p,
                (const int64_t *)A->rp_near.p, (const int64_t *)A->off_near_d.p, (int32_t *)A->col_near.p,
                (const double *)A->ndense.p, (const double *)A->ndense_spec.p, A->val_near.p, A->KW, m.NB, true, fill_lag_span(A), st);
    CUDA_TRY(cudaGetLastError());
    if ((s = build_toeplitz(A, false, st))) return s;
    CUDA_TRY(mark(4));
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(&status, A->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    float ms[4];
    for (int k = 0; k < 4; ++k) CUDA_TRY(cudaEventElapsedTime(&ms[k], ev[k], ev[k + 1]));
    A->stats.n_blocks = (int64_t)nb;
    A->stats.nnz = A->off_far[nb];
    A->stats.nnz_near = A->off_near[nb];
    int64_t q = 0;
    for (int64_t v : qp) q += v;
    A->stats.quad_points = q;
    A->stats.quad_points_far = -1;
    int64_t nearp = 0;
    for (int64_t t = 0; t < E; ++t) nearp += m.adj_ptr[t + 1] - m.adj_ptr[t];
    A->stats.near_pairs = nearp;
    A->stats.far_pairs = E * E - nearp;
    A->stats.ms_pattern = ms[0];
    A->stats.ms_far = ms[1];
    A->stats.ms_near = ms[2];
    A->stats.ms_extract = ms[3];
    A->stats.ms_total = ms[0] + ms[1] + ms[2] + ms[3];
    {
        // tables 4, bounds (two passes) + windows + counter 4, row counts 1, scans 2, fills 2,
        // and per colour: far, near (+ far special blocks in the mixed path)
        int64_t ncol = 0;
        for (size_t c = 0; c + 1 < A->color_off.size(); ++c) ncol += A->color_off[c + 1] > A->color_off[c];
        A->stats.kernel_launches = 13 + ncol * (A->fp64 ? 2 : 3) + (A->tw_on ? 3 : 0);
    }
    if (status) return fail(TDBEM_E_DEVICE, "kernel status word " + std::to_string(status));
    if ((s = plan_matvec(*A, st))) return s;
    A->assembled = true;
    return TDBEM_OK;
}

// Replay of the recorded assembly graph on `st`, then the checks the eager
// run makes on the host: status word and the per-block sizes (which the
// unchanged pattern must reproduce), and the phase times from the events.
static tdbem_status assemble_replay(tdbem_asm *A, cudaStream_t st) {
    const size_t nb = A->blocks.size();
    if (!A->gexec[3]) {
        if (!A->cap_stream) CUDA_TRY(cudaStreamCreateWithFlags(&A->cap_stream, cudaStreamNonBlocking));
        const tdbem_status s = assemble_body(A, A->cap_stream, true);
        if (s) {
            cudaStreamCaptureStatus cs;
            if (cudaStreamIsCapturing(A->cap_stream, &cs) == cudaSuccess && cs != cudaStreamCaptureStatusNone) {
                cudaGraph_t gr = nullptr;
                cudaStreamEndCapture(A->cap_stream, &gr);
                if (gr) cudaGraphDestroy(gr);
            }
            for (auto &g : A->gexec)
                if (g) { cudaGraphExecDestroy(g); g = nullptr; }
            return s;
        }
    }
    for (int k = 0; k < 4; ++k) {
        CUDA_TRY(cudaEventRecord(A->ev[k], st));
        CUDA_TRY(cudaGraphLaunch(A->gexec[k], st));
    }
    CUDA_TRY(cudaEventRecord(A->ev[4], st));
    std::vector<int64_t> tf(nb), tn(nb);
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(tf.data(), A->tot_far.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(tn.data(), A->tot_near.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(&status, A->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (status) return fail(TDBEM_E_DEVICE, "kernel status word " + std::to_string(status));
    if (tf != A->nnz_far || tn != A->nnz_near) return fail(TDBEM_E_DEVICE, "pattern sizes changed between assemblies");
    float ms[4];
    for (int k = 0; k < 4; ++k) CUDA_TRY(cudaEventElapsedTime(&ms[k], A->ev[k], A->ev[k + 1]));
    A->stats.ms_pattern = ms[0];
    A->stats.ms_far = ms[1];
    A->stats.ms_near = ms[2];
    A->stats.ms_extract = ms[3];
    A->stats.ms_total = ms[0] + ms[1] + ms[2] + ms[3];
    A->stats.graph_replays += 1;
    return TDBEM_OK;
}

static GradedArgs make_gargs(tdbem_asm *A) {
    const tdbem_mesh &m = *A->mesh;
    GradedArgs a{};
    a.g = make_geo(A);
    a.N = A->g_ncol;  // block columns (trial functions)
    a.tie = 1e-12 * A->tg->T;
    a.pair = (const double2 *)A->gpair.p;
    a.vmin = (const double *)A->gvmin.p;
    a.vmax = (const double *)A->gvmax.p;
    a.ga = (const double *)A->g_ga_d.p;
    a.gb = (const double *)A->g_gb_d.p;
    a.colblk = (const int *)A->g_colblk_d.p;
    a.colk0 = (const int *)A->g_colk0_d.p;
    a.pan0 = (const int *)A->g_pan0_d.p;
    a.pan64 = (const GPan64 *)A->g_pan64_d.p;
    a.pan32 = (const float4 *)A->g_pan32_d.p;
    a.coef32 = (const float *)A->g_coef32.p;
    a.coef64 = (const double *)A->g_coef.p + (size_t)A->g_njob32 * NCHEB * 2;
    a.p64 = (const int *)A->g_p64_d.p;
    a.S64 = A->S64;
    a.maxpan = A->g_maxpan;
    a.kw = (const int *)A->g_kw_d.p;
    a.dense = (double *)A->g_dense.p;
    a.ndense = (double *)A->g_ndense.p;
    a.NB = m.NB;
    a.all_tris = (const int32_t *)A->colors.p;
    a.col_off = (const int64_t *)A->g_coloff_d.p;
    a.ncol = (int)A->color_off.size() - 1;
    a.cenh = (const float *)A->g_cenh.p;
    a.cenl = (const float *)A->g_cenl.p;
    a.geoh = (const float *)A->geo32.p;
    a.geol = (const float *)A->g_geol.p;
    a.adj_ptr = (const int64_t *)A->adj_ptr.p;
    a.adj_tri = (const int32_t *)A->adj_tri.p;
    a.adj_perm = (const int8_t *)A->adj_perm.p;
    a.adj_nbr = (const int32_t *)A->adj_nbr.p;
    for (int k = 0; k < 4; ++k) { a.ss_xy[k] = (const double *)A->ss[k].p; a.ss_npp[k] = A->ss_npp[k]; }
    a.rule_w64 = (const double *)A->rule_w64.p;
    a.rule_l64 = (const double *)A->rule_l64.p;
    for (int k = 0; k < 7; ++k) {
        a.wwh[k] = (float)m.rule_W[k];
        a.wwl[k] = (float)(m.rule_W[k] - (double)a.wwh[k]);
        for (int d = 0; d < 3; ++d) {
            const double gw = m.rule_W[k] * m.rule_L[k][d];
            a.gwh[3 * k + d] = (float)gw;
            a.gwl[3 * k + d] = (float)(gw - (double)a.gwh[3 * k + d]);
        }
    }
    a.status = (int *)A->status.p;
    return a;
}

// Window lengths per column and the batches of trial columns whose FP64
// windows fit the staging budget; (re)allocates the staging buffers.
static tdbem_status plan_graded_batches(tdbem_asm &A, double smax, cudaStream_t st) {
    const int64_t N = A.g_ncol, M = A.mesh->M, NB = A.mesh->NB;  // N: block columns
    A.g_kw.assign(N, 1);
    for (int64_t i = 0; i < N; ++i) A.g_kw[i] = graded_kw(A, i, smax);
    size_t fr = 0, tot = 0;
    CUDA_TRY(cudaMemGetInfo(&fr, &tot));
    size_t cap = std::max<size_t>((size_t)256 << 20, std::min<size_t>((size_t)24 << 30, fr / 4));
    if (A.opts.staging_mb > 0) cap = (size_t)A.opts.staging_mb << 20;
    A.g_bi0.clear();
    A.g_bi1.clear();
    A.g_doff.assign(N, 0);
    A.g_ndoff.assign(N, 0);
    A.g_dense_max = A.g_ndense_max = 0;
    int64_t i = 0;
    while (i < N) {
        size_t d = 0, nd = 0;
        int64_t j = i;
        while (j < N) {
            const size_t fd = (size_t)M * M * A.g_kw[j] * sizeof(double);
            const size_t fn = (size_t)M * NB * A.g_kw[j] * sizeof(double);
            if (j > i && d + fd + nd + fn > cap) break;
            A.g_doff[j] = (int64_t)(d / sizeof(double));
            A.g_ndoff[j] = (int64_t)(nd / sizeof(double));
            d += fd;
            nd += fn;
            ++j;
        }
        A.g_bi0.push_back((int)i);
        A.g_bi1.push_back((int)j);
        A.g_dense_max = std::max(A.g_dense_max, d);
        A.g_ndense_max = std::max(A.g_ndense_max, nd);
        i = j;
    }
    tdbem_status s;
    if ((s = upload(A.g_kw_d, A.g_kw, st))) return s;
    if ((s = upload(A.g_doff_d, A.g_doff, st))) return s;
    if ((s = upload(A.g_ndoff_d, A.g_ndoff, st))) return s;
    if (A.g_dense.n < A.g_dense_max)
        if ((s = dev_alloc(A.g_dense, A.g_dense_max, st))) return s;
    if (A.g_ndense.n < A.g_ndense_max)
        if ((s = dev_alloc(A.g_ndense, A.g_ndense_max, st))) return s;
    A.g_smax = smax;
    return TDBEM_OK;
}

// One assembly on a graded grid (always eager): psi tables, element- and
// vertex-pair bounds, row counts and CSR sizes, then per batch of trial
// columns the far field (one launch per test colour), the near field and the
// CSR fill of the batch's blocks.
static tdbem_status assemble_graded(tdbem_asm *A, cudaStream_t st) {
    const tdbem_mesh &m = *A->mesh;
    const int64_t M = m.M, E = m.E;
    const size_t nb = A->blocks.size();
    for (auto &e : A->ev)
        if (!e) CUDA_TRY(cudaEventCreate(&e));
    CUDA_TRY(cudaEventRecord(A->ev[0], st));
    CUDA_TRY(cudaMemsetAsync(A->status.p, 0, 16, st));
    // ---- psi tables: FP32 set (24-point Gauss-Legendre x 4 per piece), FP64 sets (x 8), DCT
    const int nj32 = A->g_njob32, nj64 = A->g_nset64;
    launch_psi_samples_var(A->tg->kind, (const double *)A->tgrid.p, (int)A->tg->N, (const int *)A->g_tkb.p, (const int *)A->g_tib.p,
                           (const int *)A->g_tm2.p, (const int *)A->g_tm1.p, (const double *)A->g_tr0.p, (const double *)A->g_tdr.p, nj32, (const double *)A->gl_x.p,
                           (const double *)A->gl_w.p, 24, 4, (double *)A->g_samples.p, st);
    launch_psi_samples_var(A->tg->kind, (const double *)A->tgrid.p, (int)A->tg->N, (const int *)A->g_tkb.p + nj32,
                           (const int *)A->g_tib.p + nj32, (const int *)A->g_tm2.p + nj32,
                           (const int *)A->g_tm1.p + nj32, (const double *)A->g_tr0.p + nj32,
                           (const double *)A->g_tdr.p + nj32, nj64, (const double *)A->gl_x.p,
                           (const double *)A->gl_w.p, 24, 8, (double *)A->g_samples.p + (size_t)nj32 * NCHEB * 2, st);
    launch_psi_dct((const double *)A->g_samples.p, nj32 + nj64, (double *)A->g_coef.p, st);
    if (!A->fp64) launch_gcoef32((const double *)A->g_coef.p, A->g_npan, (float *)A->g_coef32.p, st);
    CUDA_TRY(cudaGetLastError());
    // ---- bounds, windows, row counts, CSR sizes
    Geo g = make_geo(A);
    launch_gpair_bounds(g, (double2 *)A->gpair.p, st);
    GradedArgs ga = make_gargs(A);
    launch_gvertex(ga, (double *)A->gvmin.p, (double *)A->gvmax.p, (double *)A->gpartial.p, 1024, st);
    launch_gcount(ga, (const int *)A->g_cb2api_d.p, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p,
                  (int64_t *)A->cnt_far.p, (int64_t *)A->cnt_near.p, st);
    launch_scan_rows((const int64_t *)A->cnt_far.p, M, (int)nb, (int64_t *)A->rp_far.p, (int64_t *)A->tot_far.p, st);
    launch_scan_rows((const int64_t *)A->cnt_near.p, M, (int)nb, (int64_t *)A->rp_near.p, (int64_t *)A->tot_near.p, st);
    launch_gcount_quad(ga, 49, A->ss_npp, (int64_t *)A->quad_partial.p, 1024, st);
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaEventRecord(A->ev[1], st));
    std::vector<double> part(1024);
    std::vector<int64_t> qp(2048);
    A->nnz_far.assign(nb, 0);
    A->nnz_near.assign(nb, 0);
    CUDA_TRY(cudaMemcpyAsync(part.data(), A->gpartial.p, 1024 * sizeof(double), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(qp.data(), A->quad_partial.p, 2048 * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(A->nnz_far.data(), A->tot_far.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaMemcpyAsync(A->nnz_near.data(), A->tot_near.p, nb * sizeof(int64_t), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    double smax = 0.0;
    for (double v : part) smax = std::max(smax, v);
    tdbem_status s;
    if (smax != A->g_smax)
        if ((s = plan_graded_batches(*A, smax, st))) return s;
    A->off_far.assign(nb + 1, 0);
    A->off_near.assign(nb + 1, 0);
    for (size_t b = 0; b < nb; ++b) {
        A->off_far[b + 1] = A->off_far[b] + A->nnz_far[b];
        A->off_near[b + 1] = A->off_near[b] + A->nnz_near[b];
    }
    const size_t rs = A->fp64 ? 8 : 4;
    if ((size_t)A->off_far[nb] > A->col_far_cap || A->col_far.p == nullptr) {
        if ((s = dev_alloc(A->col_far, A->off_far[nb] * sizeof(int32_t), st))) return s;
        if ((s = dev_alloc(A->val_far, A->off_far[nb] * rs, st))) return s;
        A->col_far_cap = A->off_far[nb];
    }
    if ((size_t)A->off_near[nb] > A->col_near_cap || A->col_near.p == nullptr) {
        if ((s = dev_alloc(A->col_near, A->off_near[nb] * sizeof(int32_t), st))) return s;
        if ((s = dev_alloc(A->val_near, A->off_near[nb] * sizeof(double), st))) return s;
        A->col_near_cap = A->off_near[nb];
    }
    CUDA_TRY(cudaMemcpyAsync(A->off_far_d.p, A->off_far.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    CUDA_TRY(cudaMemcpyAsync(A->off_near_d.p, A->off_near.data(), nb * sizeof(int64_t), cudaMemcpyHostToDevice, st));
    // ---- per batch of trial columns: far, near, fill
    ga = make_gargs(A);
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    const size_t nbt = A->g_bi0.size();
    const size_t nev = 3 * nbt + 1;
    while (A->g_ev.size() < nev) {
        cudaEvent_t e;
        CUDA_TRY(cudaEventCreate(&e));
        A->g_ev.push_back(e);
    }
    const size_t smem = gfar_smem(A->g_maxpan, A->fp64);
    if (smem > 227 * 1024) return fail(TDBEM_E_UNSUPPORTED, "panel tables of one block column exceed shared memory");
    const int ncol = (int)A->color_off.size() - 1;
    int64_t launches = 11;
    for (size_t bt = 0; bt < nbt; ++bt) {
        const int i0 = A->g_bi0[bt], i1 = A->g_bi1[bt];
        ga.i0 = i0;
        ga.i1 = i1;
        ga.doff = (const int64_t *)A->g_doff_d.p + i0;
        ga.ndoff = (const int64_t *)A->g_ndoff_d.p + i0;
        size_t db = 0, ndb = 0;
        for (int i = i0; i < i1; ++i) {
            db += (size_t)M * M * A->g_kw[i] * sizeof(double);
            ndb += (size_t)M * m.NB * A->g_kw[i] * sizeof(double);
        }
        CUDA_TRY(cudaMemsetAsync(A->g_dense.p, 0, db, st));
        CUDA_TRY(cudaMemsetAsync(A->g_ndense.p, 0, ndb, st));
        CUDA_TRY(cudaEventRecord(A->g_ev[3 * bt], st));
        for (int c = 0; c < ncol; ++c) {
            ga.color_tris = (const int32_t *)A->colors.p + A->color_off[c];
            ga.ncolor = A->color_off[c + 1] - A->color_off[c];
            if (ga.ncolor <= 0) continue;
            launch_gfar(ga, A->fp64, (int)std::min<int64_t>(ga.ncolor, nsm), smem, st);
            ++launches;
        }
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(A->g_ev[3 * bt + 1], st));
        for (int c = 0; c < ncol; ++c) {
            ga.color_tris = (const int32_t *)A->colors.p + A->color_off[c];
            ga.ncolor = A->color_off[c + 1] - A->color_off[c];
            if (ga.ncolor <= 0) continue;
            // mixed, p = 0: psi in FP32; p >= 1 keeps FP64 (the Legendre factors
            // left 1.2e-6 per block with FP32 on the 80-triangle sphere)
            launch_gnear(ga, !A->fp64 && A->tg->p == 0, (int)std::min<int64_t>(ga.ncolor, 4 * (int64_t)nsm), st);
            ++launches;
        }
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaEventRecord(A->g_ev[3 * bt + 2], st));
        launch_gfill(ga, (const int *)A->g_cb2api_d.p, (const int64_t *)A->nbr_ptr.p, (const int32_t *)A->nbr.p,
                     (const int64_t *)A->rp_far.p, (const int64_t *)A->off_far_d.p, (int32_t *)A->col_far.p,
                     A->val_far.p, A->fp64, (const int64_t *)A->rp_near.p, (const int64_t *)A->off_near_d.p,
                     (int32_t *)A->col_near.p, (double *)A->val_near.p, st);
        ++launches;
        CUDA_TRY(cudaGetLastError());
    }
    CUDA_TRY(cudaEventRecord(A->g_ev[3 * nbt], st));
    int status = 0;
    CUDA_TRY(cudaMemcpyAsync(&status, A->status.p, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    float ms_pat = 0.f, ms_far = 0.f, ms_near = 0.f, ms_ext = 0.f, x = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&ms_pat, A->ev[0], A->ev[1]));
    for (size_t bt = 0; bt < nbt; ++bt) {
        CUDA_TRY(cudaEventElapsedTime(&x, A->g_ev[3 * bt], A->g_ev[3 * bt + 1])); ms_far += x;
        CUDA_TRY(cudaEventElapsedTime(&x, A->g_ev[3 * bt + 1], A->g_ev[3 * bt + 2])); ms_near += x;
        CUDA_TRY(cudaEventElapsedTime(&x, A->g_ev[3 * bt + 2], A->g_ev[3 * bt + 3])); ms_ext += x;
    }
    A->stats.n_blocks = (int64_t)nb;
    A->stats.nnz = A->off_far[nb];
    A->stats.nnz_near = A->off_near[nb];
    int64_t q = 0, qf = 0;
    for (int k = 0; k < 1024; ++k) { q += qp[k]; qf += qp[1024 + k]; }
    A->stats.quad_points = q;
    A->stats.quad_points_far = qf;
    int64_t nearp = 0;
    for (int64_t t = 0; t < E; ++t) nearp += m.adj_ptr[t + 1] - m.adj_ptr[t];
    A->stats.near_pairs = nearp;
    A->stats.far_pairs = E * E - nearp;
    A->stats.ms_pattern = ms_pat;
    A->stats.ms_far = ms_far;
    A->stats.ms_near = ms_near;
    A->stats.ms_extract = ms_ext;
    A->stats.ms_total = ms_pat + ms_far + ms_near + ms_ext;
    A->stats.kernel_launches = launches;
    if (status) return fail(TDBEM_E_DEVICE, "kernel status word " + std::to_string(status));
    if ((s = plan_matvec(*A, st))) return s;
    A->assembled = true;
    return TDBEM_OK;
}

tdbem_status tdbem_assemble_all(tdbem_asm *A, void *stream) {
    if (!A) return fail(TDBEM_E_INVALID_ARG, "NULL assembler");
    cudaStream_t st = (cudaStream_t)stream;
    if (A->graded) return assemble_graded(A, st);
    if (A->assembled && A->use_graph) return assemble_replay(A, st);
    return assemble_body(A, st, false);
}

tdbem_status tdbem_assemble_block(tdbem_asm *A, int32_t k, int32_t i, void *stream) {
    if (!A) return fail(TDBEM_E_INVALID_ARG, "NULL assembler");
    if (A->tg->p > 0) return fail(TDBEM_E_UNSUPPORTED, "one block on its own takes p = 0");
    const int64_t N = A->tg->N;
    if (k < 0 || k >= N || i < 0 || i >= N) return fail(TDBEM_E_INVALID_ARG, "block index out of range");
    if (i > k + 1) return fail(TDBEM_E_INVALID_ARG, "block above the first superdiagonal is zero (i > k + 1)");
    cudaStream_t st = (cudaStream_t)stream;
    if (!A->single || A->single->only_k != k || A->single->only_i != i) {
        delete A->single;
        A->single = nullptr;
        tdbem_asm *B = new tdbem_asm();
        B->mesh = A->mesh;
        B->tg = A->tg;
        B->opts = A->opts;
        B->fp64 = A->fp64;
        B->only_k = k;
        B->only_i = i;
        tdbem_status s = create_graded(*B, st);
        if (!s && B->blocks.empty()) s = fail(TDBEM_E_INVALID_ARG, "block (k, i) is zero: its psi support starts beyond diam");
        if (s) { delete B; return s; }
        A->single = B;
    }
    return assemble_graded(A->single, st);
}

tdbem_status tdbem_block_csr(const tdbem_asm *A, int64_t b, int32_t which, const int64_t **rp, const int32_t **col,
                             const void **val, int64_t *nnz) {
    if (!A) return fail(TDBEM_E_INVALID_ARG, "NULL assembler");
    if (b == TDBEM_LAST_BLOCK) {
        if (!A->single || !A->single->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_block first");
        return tdbem_block_csr(A->single, 0, which, rp, col, val, nnz);
    }
    if (b < 0 || b >= (int64_t)A->blocks.size()) return fail(TDBEM_E_INVALID_ARG, "block index out of range");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    const int64_t M = A->mesh->M;
    if (which == TDBEM_FAR) {
        if (rp) *rp = (const int64_t *)A->rp_far.p + b * (M + 1);
        if (col) *col = (const int32_t *)A->col_far.p + A->off_far[b];
        if (val) *val = (const char *)A->val_far.p + A->off_far[b] * (A->fp64 ? 8 : 4);
        if (nnz) *nnz = A->nnz_far[b];
    } else if (which == TDBEM_NEAR) {
        if (rp) *rp = (const int64_t *)A->rp_near.p + b * (M + 1);
        if (col) *col = (const int32_t *)A->col_near.p + A->off_near[b];
        if (val) *val = (const double *)A->val_near.p + A->off_near[b];
        if (nnz) *nnz = A->nnz_near[b];
    } else {
        return fail(TDBEM_E_INVALID_ARG, "which must be TDBEM_FAR or TDBEM_NEAR");
    }
    return TDBEM_OK;
}

tdbem_status tdbem_block_csr_host(const tdbem_asm *A, int64_t b, int32_t which, int64_t *rp, int32_t *col,
                                  void *val) {
    const int64_t *drp;
    const int32_t *dcol;
    const void *dval;
    int64_t nnz;
    tdbem_status s = tdbem_block_csr(A, b, which, &drp, &dcol, &dval, &nnz);
    if (s) return s;
    const int64_t M = A->mesh->M;
    if (b == TDBEM_LAST_BLOCK) A = A->single;
    const size_t vs = (which == TDBEM_FAR && !A->fp64) ? 4 : 8;
    if (rp) CUDA_TRY(cudaMemcpy(rp, drp, (M + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost));
    if (col && nnz) CUDA_TRY(cudaMemcpy(col, dcol, nnz * sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (val && nnz) CUDA_TRY(cudaMemcpy(val, dval, nnz * vs, cudaMemcpyDeviceToHost));
    return TDBEM_OK;
}

// Matvec autotuner: on the first product of an assembler, time every launch
// shape on the caller's x and y (one warm-up and one timed run each, CUDA
// events) and keep the fastest; the choice is cached for the process per
// (device, M, N, unique blocks, precision, nnz). The last run leaves y = A x
// from the chosen shape, which the caller's launch then recomputes.
static std::mutex g_mv_mu;
static std::map<std::vector<int64_t>, int> g_mv_best;

// Kernels of one product: 3 (padded FP32 copy of x, CSR kernel on the
// blocks outside the Toeplitz class, Toeplitz kernel) where the assembler
// has the per-pair windows, else 2 (transpose, CSR kernel).
static int mv_launches(const tdbem_asm *A) { return A->tw_on ? 3 : 2; }

// The whole product y = A x; scratch: the assembler's, or the fixed array of
// the no-allocation entry point (xbytes usable bytes).
static cudaError_t mv_launch(const tdbem_asm *A, const double *x, void *scratch, size_t xbytes, double *y, int nsm,
                             int variant, cudaStream_t st) {
    const int64_t N = time_rows(A), M = A->mesh->M;
    if (A->tw_on && (size_t)(4 * M * A->tw_S) * sizeof(float) <= xbytes) {
        // variants: 3 Toeplitz shapes (outputs per lane) x 2 CSR shapes
        cudaError_t e = launch_hessenberg_rest((const MvBlock *)A->mv_rest.p, (int)A->mv_rest_host.size(), x, y, M,
                                               (int)N, nsm, variant < 3 ? 0 : 3, st);
        if (e != cudaSuccess) return e;
        TwArgs g;
        g.M = M;
        g.nin = (int)N - 2;
        g.TL = A->tw_TL;
        g.S = A->tw_S;
        g.PADL = A->tw_PADL;
        g.fptr = (const int64_t *)A->tw_ptr.p;
        g.nptr = (const int64_t *)A->tw_ptr.p + (M + 1);
        g.fhdr = (const int2 *)A->tw_fhdr.p;
        g.fval = (const float *)A->tw_fval.p;
        g.nhdr = (const int2 *)A->tw_nhdr.p;
        g.nval = (const double *)A->tw_nval.p;
        return launch_toeplitz(g, x, (float *)scratch, y, tw_variant_outputs(variant), nsm, st);
    }
    return launch_hessenberg((const MvBlock *)A->mv_blk.p, (int)A->blocks.size(), A->fp64, x, (double *)scratch, y, M,
                             (int)N, nsm, variant, st);
}

static tdbem_status tune_matvec(const tdbem_asm *A, const double *x, double *y, int nsm, cudaStream_t st) {
    int dev = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    const int64_t N = time_rows(A), M = A->mesh->M;
    const std::vector<int64_t> key = {dev, M, N, (int64_t)A->blocks.size(), A->fp64 ? 1 : 0, A->stats.nnz};
    {
        std::lock_guard<std::mutex> lock(g_mv_mu);
        auto it = g_mv_best.find(key);
        if (it != g_mv_best.end()) {
            A->mv_variant = it->second;
            return TDBEM_OK;
        }
    }
    cudaEvent_t e0, e1;
    CUDA_TRY(cudaEventCreate(&e0));
    CUDA_TRY(cudaEventCreate(&e1));
    int best = 0;
    float bt = 1e30f;
    tdbem_status s = TDBEM_OK;
    for (int v = 0; v < MV_NVARIANTS && !s; ++v) {
        float ms = 0.f;
        cudaError_t e = mv_launch(A, x, A->mv_xT.p, A->mv_xT.n, y, nsm, v, st);
        if (e == cudaSuccess) e = cudaEventRecord(e0, st);
        if (e == cudaSuccess) e = mv_launch(A, x, A->mv_xT.p, A->mv_xT.n, y, nsm, v, st);
        if (e == cudaSuccess) e = cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        if (e != cudaSuccess) s = fail(TDBEM_E_CUDA, std::string("matvec autotuner: ") + cudaGetErrorString(e));
        else if (ms < bt) { bt = ms; best = v; }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (s) return s;
    A->mv_variant = best;
    std::lock_guard<std::mutex> lock(g_mv_mu);
    g_mv_best[key] = best;
    return TDBEM_OK;
}

tdbem_status tdbem_hessenberg_apply(const tdbem_asm *A, const double *x, double *y, void *stream) {
    if (!A || !x || !y) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    const int64_t N = time_rows(A), M = A->mesh->M;
    const char *xb = (const char *)x, *yb = (const char *)y;
    const size_t bytes = (size_t)(N * M) * sizeof(double);
    if (xb < yb + bytes && yb < xb + bytes) return fail(TDBEM_E_INVALID_ARG, "x and y overlap");
    cudaStream_t st = (cudaStream_t)stream;
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (A->mv_variant < 0) {
        tdbem_status ts = tune_matvec(A, x, y, nsm, st);
        if (ts) return ts;
    }
    CUDA_TRY(mv_launch(A, x, A->mv_xT.p, A->mv_xT.n, y, nsm, A->mv_variant, st));
    return TDBEM_OK;
}

tdbem_status tdbem_hessenberg_apply_noalloc(const tdbem_asm *A, const double *x, double *y, void *stream) {
    if (!A || !x || !y) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    const int64_t N = time_rows(A), M = A->mesh->M;
    if (N * M > MV_STATIC_MAX)
        return fail(TDBEM_E_INVALID_ARG, "N*M = " + std::to_string(N * M) + " exceeds the fixed scratch of " +
                                             std::to_string(MV_STATIC_MAX) + " doubles");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    const char *xb = (const char *)x, *yb = (const char *)y;
    const size_t bytes = (size_t)(N * M) * sizeof(double);
    if (xb < yb + bytes && yb < xb + bytes) return fail(TDBEM_E_INVALID_ARG, "x and y overlap");
    double *xT = nullptr;
    CUDA_TRY(static_mv_scratch(&xT));
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    // the shape the autotuner chose for this assembler, if any (no timing here)
    CUDA_TRY(mv_launch(A, x, xT, (size_t)MV_STATIC_MAX * sizeof(double), y, nsm, A->mv_variant < 0 ? 0 : A->mv_variant,
                       (cudaStream_t)stream));
    return TDBEM_OK;
}

tdbem_status tdbem_psi_table(const tdbem_asm *A, int64_t b, int32_t which, const double *r, int64_t n, double *out,
                             void *stream) {
    if (!A || (n > 0 && (!r || !out))) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (n < 0) return fail(TDBEM_E_INVALID_ARG, "n < 0");
    if (b < 0 || b >= (int64_t)A->blocks.size()) return fail(TDBEM_E_INVALID_ARG, "block index out of range");
    if (which != 0 && which != 1) return fail(TDBEM_E_INVALID_ARG, "which must be 0 (FP64 set) or 1 (FP32 set)");
    if (A->graded) return fail(TDBEM_E_UNSUPPORTED, "per-class tables exist on equidistant grids only");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "the tables are built by tdbem_assemble_all");
    const Block &B = A->blocks[b];
    int panel0 = 0;
    for (int c = 0; c < B.cls; ++c) panel0 += A->cls_P[c];
    launch_psi_table(r, n, 1.0 / A->tg->dt, B.lag, A->cls_rho[B.cls], A->cls_P[B.cls], panel0, A->S64,
                     (const double *)A->tab_coef4.p, A->c32, which, out, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return TDBEM_OK;
}

tdbem_status tdbem_double_layer(const tdbem_asm *A, const double *alpha, const double *X, int64_t P,
                                const double *times, int32_t nt, int32_t n, double *u, void *stream) {
    if (!A) return fail(TDBEM_E_INVALID_ARG, "NULL assembler");
    if (P < 0 || nt < 1) return fail(TDBEM_E_INVALID_ARG, "need P >= 0 points and nt >= 1 times");
    if (n < 1 || n > 32) return fail(TDBEM_E_INVALID_ARG, "n (Gauss points per direction) must be in 1..32");
    if (!alpha || !times || (P > 0 && (!X || !u))) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (A->tg->p != 0) return fail(TDBEM_E_UNSUPPORTED, "the potential takes temporal degree p = 0");
    if (P == 0) return TDBEM_OK;
    cudaStream_t st = (cudaStream_t)stream;
    const tdbem_mesh &m = *A->mesh;
    const int N = (int)A->tg->N;
    const int64_t EQ = m.E * (int64_t)n * n;
    std::vector<double> gx, gw;
    gauss_legendre01(n, gx, gw);
    DevBuf dgx, dgw, yw, coef, tab;
    tdbem_status s;
    if ((s = upload(dgx, gx, st)) || (s = upload(dgw, gw, st))) return s;
    if ((s = dev_alloc(yw, (size_t)EQ * 2 * sizeof(double4), st))) return s;
    if ((s = dev_alloc(coef, (size_t)EQ * N * sizeof(double), st))) return s;
    if ((s = dev_alloc(tab, (size_t)DL_TABLE_NODES * sizeof(double3), st))) return s;
    Geo g = make_geo(const_cast<tdbem_asm *>(A));
    CUDA_TRY(launch_double_layer(A->tg->kind, g, (const double *)A->tgrid.p, N, A->tg->equidistant ? 1 : 0,
                                 A->tg->c, (const double *)dgx.p, (const double *)dgw.p, n, alpha, X, P, times, nt,
                                 (double4 *)yw.p, (double *)coef.p, (double3 *)tab.p, u, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDBEM_OK;
}

tdbem_status tdbem_rhs_assemble(const tdbem_asm *A, int32_t kind, const double *params, int32_t nparams,
                                double *g_dev, void *stream) {
    if (!A || !g_dev) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    RhsParams prm{};
    if (kind == TDBEM_RHS_PLANE_WAVE) {
        if (!params || nparams != 5) return fail(TDBEM_E_INVALID_ARG, "plane wave takes 5 parameters (dx, dy, dz, c0, w)");
        const double dn = sqrt(params[0] * params[0] + params[1] * params[1] + params[2] * params[2]);
        if (!(dn > 0.0) || !(params[4] > 0.0) || !std::isfinite(params[3]))
            return fail(TDBEM_E_INVALID_ARG, "plane wave needs a nonzero direction and a positive width");
        for (int k = 0; k < 3; ++k) prm.p[k] = params[k] / dn;
        prm.p[3] = params[3];
        prm.p[4] = params[4];
    } else if (kind == TDBEM_RHS_SPHERE_N0 || kind == TDBEM_RHS_SPHERE_N1) {
        if (nparams != 0) return fail(TDBEM_E_INVALID_ARG, "this kind takes no parameters");
    } else {
        return fail(TDBEM_E_INVALID_ARG, "unknown right-hand side kind");
    }
    const tdbem_asm *Ac = A;
    Geo g = make_geo(const_cast<tdbem_asm *>(Ac));
    launch_rhs(A->tg->kind, g, (const double *)A->tgrid.p, (int)A->tg->N, A->tg->p + 1, A->tg->c, (const double *)A->rule_w64.p,
               (const double *)A->rule_l64.p, (const double *)A->gl_x.p, (const double *)A->gl_w.p, 24, 4, kind, prm,
               g_dev, (cudaStream_t)stream);
    CUDA_TRY(cudaGetLastError());
    return TDBEM_OK;
}

// Restarted GMRES(m) with classical Gram-Schmidt and one reorthogonalisation;
// the Hessenberg least-squares problem is updated with Givens rotations on the
// host. Zero initial guess.
tdbem_status tdbem_solve_gmres(const tdbem_asm *A, const double *g, double *x, int32_t restart, double tol,
                               int32_t max_iter, int32_t *iters, double *rel_res, void *stream) {
    if (!A || !g || !x) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    if (restart < 1 || restart > GM_MAXV - 2) return fail(TDBEM_E_INVALID_ARG, "restart must be in 1..62");
    if (!(tol > 0.0) || max_iter < 1) return fail(TDBEM_E_INVALID_ARG, "need tol > 0 and max_iter >= 1");
    const int64_t n = time_rows(A) * A->mesh->M;
    const char *gb = (const char *)g, *xb = (const char *)x;
    if (gb < xb + n * 8 && xb < gb + n * 8) return fail(TDBEM_E_INVALID_ARG, "g and x overlap");
    cudaStream_t st = (cudaStream_t)stream;
    const int m = restart;
    DevBuf Vb, wb, pb, hb, sb;
    tdbem_status s;
    if ((s = dev_alloc(Vb, (size_t)(m + 1) * n * sizeof(double), st))) return s;
    if ((s = dev_alloc(wb, (size_t)n * sizeof(double), st))) return s;
    if ((s = dev_alloc(pb, (size_t)GM_BLOCKS * GM_MAXV * sizeof(double), st))) return s;
    if ((s = dev_alloc(hb, (size_t)2 * GM_MAXV * sizeof(double), st))) return s;
    if ((s = dev_alloc(sb, (size_t)GM_MAXV * sizeof(double), st))) return s;
    double *V = (double *)Vb.p, *w = (double *)wb.p, *part = (double *)pb.p, *hd = (double *)hb.p, *sd = (double *)sb.p;
    auto dot = [&](const double *Vv, int nv, const double *ww, double *hout) -> tdbem_status {
        launch_multi_dot(Vv, n, nv, ww, n, part, hd, st);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(hout, hd, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return TDBEM_OK;
    };
    auto upload = [&](const double *hv, int nv) -> tdbem_status {
        CUDA_TRY(cudaMemcpyAsync(sd, hv, nv * sizeof(double), cudaMemcpyHostToDevice, st));
        return TDBEM_OK;
    };
    CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    double gn2 = 0.0;
    if ((s = dot(g, 1, g, &gn2))) return s;
    const double gnorm = sqrt(gn2);
    int total = 0;
    double rr = 0.0;
    if (gnorm == 0.0) {
        if (iters) *iters = 0;
        if (rel_res) *rel_res = 0.0;
        return TDBEM_OK;
    }
    std::vector<double> H((size_t)(m + 1) * m), cs(m), sn(m), e(m + 1), y(m), hv(2 * GM_MAXV);
    for (;;) {
        // V_0 = (g - A x) / beta
        if ((s = tdbem_hessenberg_apply(A, x, w, stream))) return s;
        CUDA_TRY(cudaMemcpyAsync(V, g, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        const double one = 1.0;
        if ((s = upload(&one, 1))) return s;
        launch_multi_axpy(w, n, 1, sd, -1.0, V, n, st);
        double b2 = 0.0;
        if ((s = dot(V, 1, V, &b2))) return s;
        const double beta = sqrt(b2);
        rr = beta / gnorm;
        if (rr <= tol || total >= max_iter) break;
        if ((s = upload(&beta, 1))) return s;
        launch_scale_copy(V, sd, V, n, st);
        std::fill(e.begin(), e.end(), 0.0);
        e[0] = beta;
        int jdone = 0;
        bool stop = false;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
            if ((s = tdbem_hessenberg_apply(A, vj, w, stream))) return s;
            // w -= V h, twice (classical Gram-Schmidt with reorthogonalisation)
            for (int pass = 0; pass < 2; ++pass) {
                if ((s = dot(V, j + 1, w, hv.data() + pass * GM_MAXV))) return s;
                launch_multi_axpy(V, n, j + 1, hd, -1.0, w, n, st);
            }
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = hv[i] + hv[GM_MAXV + i];
            double w2 = 0.0;
            if ((s = dot(w, 1, w, &w2))) return s;
            const double hn = sqrt(w2);
            H[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) {
                if ((s = upload(&hn, 1))) return s;
                launch_scale_copy(w, sd, vn, n, st);
            }
            // previous rotations, then a new one that zeroes H[j+1][j]
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            const double rho = hypot(a, b);
            cs[j] = rho > 0.0 ? a / rho : 1.0;
            sn[j] = rho > 0.0 ? b / rho : 0.0;
            H[(size_t)j * m + j] = rho;
            H[(size_t)(j + 1) * m + j] = 0.0;
            e[j + 1] = -sn[j] * e[j];
            e[j] = cs[j] * e[j];
            ++total;
            jdone = j + 1;
            rr = fabs(e[j + 1]) / gnorm;
            if (rr <= tol || total >= max_iter || hn == 0.0) {
                stop = true;
                break;
            }
        }
        // x += V y with R y = e (back substitution)
        for (int i = jdone - 1; i >= 0; --i) {
            double v = e[i];
            for (int k = i + 1; k < jdone; ++k) v -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? v / H[(size_t)i * m + i] : 0.0;
        }
        if ((s = upload(y.data(), jdone))) return s;
        launch_multi_axpy(V, n, jdone, sd, 1.0, x, n, st);
        CUDA_TRY(cudaGetLastError());
        if (stop) {
            // true residual of the final iterate
            if ((s = tdbem_hessenberg_apply(A, x, w, stream))) return s;
            CUDA_TRY(cudaMemcpyAsync(V, g, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
            if ((s = upload(&one, 1))) return s;
            launch_multi_axpy(w, n, 1, sd, -1.0, V, n, st);
            if ((s = dot(V, 1, V, &b2))) return s;
            rr = sqrt(b2) / gnorm;
            break;
        }
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (iters) *iters = total;
    if (rel_res) *rel_res = rr;
    return TDBEM_OK;
}

tdbem_status tdbem_deflation_basis(const double *H, int32_t m, int32_t ldh, int32_t l, double *B, int32_t *sdim,
                                   double *lam_max) {
    if (!H || !B || !sdim || !lam_max) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (m < 1 || m > KR_MAXM) return fail(TDBEM_E_INVALID_ARG, "m must be in 1..62");
    if (ldh < m) return fail(TDBEM_E_INVALID_ARG, "ldh < m");
    if (l < 0) return fail(TDBEM_E_INVALID_ARG, "l < 0");
    int sd = 0;
    double lm = 0.0;
    if (deflation_basis(H, m, ldh, l, B, &sd, &lm)) return fail(TDBEM_E_NUMERIC, "Schur iteration did not converge");
    *sdim = sd;
    *lam_max = lm;
    return TDBEM_OK;
}

// DGMRES(m, l) of Sec. 4.1, the cycle structure of restarted GMRES above with
// the deflation preconditioner applied to each basis vector before the
// product and to the correction V y; U and A U live on the device, T^-1 on
// the host.
tdbem_status tdbem_solve_dgmres(const tdbem_asm *A, const double *g, double *x, int32_t restart, int32_t l,
                                int32_t r, double tol, int32_t max_iter, int32_t *iters, double *rel_res,
                                int32_t *deflated, void *stream) {
    if (!A || !g || !x) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    if (restart < 1 || restart > KR_MAXM) return fail(TDBEM_E_INVALID_ARG, "restart must be in 1..62");
    if (l < 0) return fail(TDBEM_E_INVALID_ARG, "l must be >= 0");
    if (r < 0 || r > KR_MAXM) return fail(TDBEM_E_INVALID_ARG, "r must be in 0..62");
    if (!(tol > 0.0) || max_iter < 1) return fail(TDBEM_E_INVALID_ARG, "need tol > 0 and max_iter >= 1");
    const int64_t n = time_rows(A) * A->mesh->M;
    const char *gb = (const char *)g, *xb = (const char *)x;
    if (gb < xb + n * 8 && xb < gb + n * 8) return fail(TDBEM_E_INVALID_ARG, "g and x overlap");
    cudaStream_t st = (cudaStream_t)stream;
    const int m = restart;
    DevBuf Vb, wb, zb, Ub, AUb, pb, hb, sb;
    tdbem_status s;
    if ((s = dev_alloc(Vb, (size_t)(m + 1) * n * sizeof(double), st))) return s;
    if ((s = dev_alloc(wb, (size_t)n * sizeof(double), st))) return s;
    if ((s = dev_alloc(zb, (size_t)n * sizeof(double), st))) return s;
    if (r > 0 && l > 0) {
        if ((s = dev_alloc(Ub, (size_t)r * n * sizeof(double), st))) return s;
        if ((s = dev_alloc(AUb, (size_t)r * n * sizeof(double), st))) return s;
    }
    if ((s = dev_alloc(pb, (size_t)GM_BLOCKS * GM_MAXV * sizeof(double), st))) return s;
    if ((s = dev_alloc(hb, (size_t)2 * GM_MAXV * sizeof(double), st))) return s;
    if ((s = dev_alloc(sb, (size_t)GM_MAXV * sizeof(double), st))) return s;
    double *V = (double *)Vb.p, *w = (double *)wb.p, *z = (double *)zb.p, *U = (double *)Ub.p,
           *AU = (double *)AUb.p, *part = (double *)pb.p, *hd = (double *)hb.p, *sd = (double *)sb.p;
    auto dot = [&](const double *Vv, int nv, const double *ww, double *hout) -> tdbem_status {
        launch_multi_dot(Vv, n, nv, ww, n, part, hd, st);
        CUDA_TRY(cudaGetLastError());
        CUDA_TRY(cudaMemcpyAsync(hout, hd, nv * sizeof(double), cudaMemcpyDeviceToHost, st));
        CUDA_TRY(cudaStreamSynchronize(st));
        return TDBEM_OK;
    };
    auto upload = [&](const double *hv, int nv) -> tdbem_status {
        CUDA_TRY(cudaMemcpyAsync(sd, hv, nv * sizeof(double), cudaMemcpyHostToDevice, st));
        return TDBEM_OK;
    };
    // deflation state: nu columns of U, T^-1 (row-major nu x nu), |lambda_max|
    int nu = 0;
    double lam = 1.0;
    std::vector<double> Tinv;
    // out = M^-1 v (out != v)
    auto prec = [&](const double *v, double *out) -> tdbem_status {
        CUDA_TRY(cudaMemcpyAsync(out, v, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if (nu == 0) return TDBEM_OK;
        std::vector<double> c(nu), d(nu);
        tdbem_status ps = dot(U, nu, v, c.data());
        if (ps) return ps;
        for (int i = 0; i < nu; ++i) {
            double t = 0.0;
            for (int k = 0; k < nu; ++k) t += Tinv[(size_t)i * nu + k] * c[k];
            d[i] = lam * t - c[i];
        }
        if ((ps = upload(d.data(), nu))) return ps;
        launch_multi_axpy(U, n, nu, sd, 1.0, out, n, st);
        CUDA_TRY(cudaGetLastError());
        return TDBEM_OK;
    };
    CUDA_TRY(cudaMemsetAsync(x, 0, n * sizeof(double), st));
    double gn2 = 0.0;
    if ((s = dot(g, 1, g, &gn2))) return s;
    const double gnorm = sqrt(gn2);
    int total = 0;
    double rr = 0.0;
    if (gnorm == 0.0) {
        if (iters) *iters = 0;
        if (rel_res) *rel_res = 0.0;
        if (deflated) *deflated = 0;
        return TDBEM_OK;
    }
    const double one = 1.0;
    std::vector<double> H((size_t)(m + 1) * m), Hr((size_t)(m + 1) * m), cs(m), sn(m), e(m + 1), y(m),
        hv(2 * GM_MAXV), Bm((size_t)m * m);
    auto true_residual = [&](double &b2) -> tdbem_status {
        tdbem_status ts = tdbem_hessenberg_apply(A, x, w, stream);
        if (ts) return ts;
        CUDA_TRY(cudaMemcpyAsync(V, g, n * sizeof(double), cudaMemcpyDeviceToDevice, st));
        if ((ts = upload(&one, 1))) return ts;
        launch_multi_axpy(w, n, 1, sd, -1.0, V, n, st);
        return dot(V, 1, V, &b2);
    };
    for (;;) {
        double b2 = 0.0;
        if ((s = true_residual(b2))) return s;
        const double beta = sqrt(b2);
        rr = beta / gnorm;
        if (rr <= tol || total >= max_iter) break;
        if ((s = upload(&beta, 1))) return s;
        launch_scale_copy(V, sd, V, n, st);
        std::fill(e.begin(), e.end(), 0.0);
        std::fill(Hr.begin(), Hr.end(), 0.0);
        e[0] = beta;
        int jdone = 0;
        bool stop = false;
        for (int j = 0; j < m; ++j) {
            double *vj = V + (int64_t)j * n, *vn = V + (int64_t)(j + 1) * n;
            if ((s = prec(vj, z))) return s;
            if ((s = tdbem_hessenberg_apply(A, z, w, stream))) return s;
            for (int pass = 0; pass < 2; ++pass) {
                if ((s = dot(V, j + 1, w, hv.data() + pass * GM_MAXV))) return s;
                launch_multi_axpy(V, n, j + 1, hd, -1.0, w, n, st);
            }
            for (int i = 0; i <= j; ++i) H[(size_t)i * m + j] = Hr[(size_t)i * m + j] = hv[i] + hv[GM_MAXV + i];
            double w2 = 0.0;
            if ((s = dot(w, 1, w, &w2))) return s;
            const double hn = sqrt(w2);
            H[(size_t)(j + 1) * m + j] = Hr[(size_t)(j + 1) * m + j] = hn;
            if (hn > 0.0) {
                if ((s = upload(&hn, 1))) return s;
                launch_scale_copy(w, sd, vn, n, st);
            }
            for (int i = 0; i < j; ++i) {
                const double a = H[(size_t)i * m + j], b = H[(size_t)(i + 1) * m + j];
                H[(size_t)i * m + j] = cs[i] * a + sn[i] * b;
                H[(size_t)(i + 1) * m + j] = -sn[i] * a + cs[i] * b;
            }
            const double a = H[(size_t)j * m + j], b = H[(size_t)(j + 1) * m + j];
            const double rho = hypot(a, b);
            cs[j] = rho > 0.0 ? a / rho : 1.0;
            sn[j] = rho > 0.0 ? b / rho : 0.0;
            H[(size_t)j * m + j] = rho;
            H[(size_t)(j + 1) * m + j] = 0.0;
            e[j + 1] = -sn[j] * e[j];
            e[j] = cs[j] * e[j];
            ++total;
            jdone = j + 1;
            rr = fabs(e[j + 1]) / gnorm;
            if (rr <= tol || total >= max_iter || hn == 0.0) {
                stop = true;
                break;
            }
        }
        for (int i = jdone - 1; i >= 0; --i) {
            double v = e[i];
            for (int k = i + 1; k < jdone; ++k) v -= H[(size_t)i * m + k] * y[k];
            y[i] = H[(size_t)i * m + i] != 0.0 ? v / H[(size_t)i * m + i] : 0.0;
        }
        // x += M^-1 (V y)
        CUDA_TRY(cudaMemsetAsync(w, 0, n * sizeof(double), st));
        if ((s = upload(y.data(), jdone))) return s;
        launch_multi_axpy(V, n, jdone, sd, -1.0, w, n, st);  // w = -V y
        if ((s = prec(w, z))) return s;
        if ((s = upload(&one, 1))) return s;
        launch_multi_axpy(z, n, 1, sd, -1.0, x, n, st);  // x -= M^-1 (-V y)
        CUDA_TRY(cudaGetLastError());
        if (stop) {
            if ((s = true_residual(b2))) return s;
            rr = sqrt(b2) / gnorm;
            break;
        }
        if (l == 0 || nu >= r) continue;
        // deflation: invariant subspace of H_m for its smallest eigenvalues
        int ns = 0;
        double lmax = 0.0;
        if (deflation_basis(Hr.data(), m, m, l, Bm.data(), &ns, &lmax))
            return fail(TDBEM_E_NUMERIC, "DGMRES: Schur iteration of H_m did not converge");
        lam = lmax;
        const int nu0 = nu;
        std::vector<double> bk(m), cU(std::max(nu + ns, 1));
        for (int k = 0; k < ns && nu < r; ++k) {
            // u = V_m B[:, k] into U column nu, then two Gram-Schmidt passes against U
            double *u = U + (int64_t)nu * n;
            for (int i = 0; i < m; ++i) bk[i] = -Bm[(size_t)i * m + k];
            CUDA_TRY(cudaMemsetAsync(u, 0, n * sizeof(double), st));
            if ((s = upload(bk.data(), m))) return s;
            launch_multi_axpy(V, n, m, sd, -1.0, u, n, st);
            double w0 = 0.0;
            if ((s = dot(u, 1, u, &w0))) return s;
            for (int pass = 0; pass < 2 && nu > 0; ++pass) {
                if ((s = dot(U, nu, u, cU.data()))) return s;
                launch_multi_axpy(U, n, nu, hd, -1.0, u, n, st);
            }
            double w1 = 0.0;
            if ((s = dot(u, 1, u, &w1))) return s;
            if (!(sqrt(w1) > 1e-10 * sqrt(w0))) continue;
            const double nrm = sqrt(w1);
            if ((s = upload(&nrm, 1))) return s;
            launch_scale_copy(u, sd, u, n, st);
            ++nu;
        }
        if (nu == nu0) continue;
        // A U for the new columns, then T = U^T A U and its inverse
        for (int k = nu0; k < nu; ++k)
            if ((s = tdbem_hessenberg_apply(A, U + (int64_t)k * n, AU + (int64_t)k * n, stream))) return s;
        std::vector<double> T((size_t)nu * nu), col(nu);
        for (int k = 0; k < nu; ++k) {
            if ((s = dot(U, nu, AU + (int64_t)k * n, col.data()))) return s;
            for (int i = 0; i < nu; ++i) T[(size_t)i * nu + k] = col[i];
        }
        // Gauss-Jordan with partial pivoting
        Tinv.assign((size_t)nu * nu, 0.0);
        for (int i = 0; i < nu; ++i) Tinv[(size_t)i * nu + i] = 1.0;
        for (int c = 0; c < nu; ++c) {
            int p = c;
            for (int i = c + 1; i < nu; ++i)
                if (fabs(T[(size_t)i * nu + c]) > fabs(T[(size_t)p * nu + c])) p = i;
            if (T[(size_t)p * nu + c] == 0.0) return fail(TDBEM_E_NUMERIC, "DGMRES: T = U^T A U is singular");
            for (int k = 0; k < nu; ++k) {
                std::swap(T[(size_t)c * nu + k], T[(size_t)p * nu + k]);
                std::swap(Tinv[(size_t)c * nu + k], Tinv[(size_t)p * nu + k]);
            }
            const double piv = T[(size_t)c * nu + c];
            for (int k = 0; k < nu; ++k) {
                T[(size_t)c * nu + k] /= piv;
                Tinv[(size_t)c * nu + k] /= piv;
            }
            for (int i = 0; i < nu; ++i) {
                if (i == c) continue;
                const double f = T[(size_t)i * nu + c];
                if (f == 0.0) continue;
                for (int k = 0; k < nu; ++k) {
                    T[(size_t)i * nu + k] -= f * T[(size_t)c * nu + k];
                    Tinv[(size_t)i * nu + k] -= f * Tinv[(size_t)c * nu + k];
                }
            }
        }
    }
    CUDA_TRY(cudaStreamSynchronize(st));
    if (iters) *iters = total;
    if (rel_res) *rel_res = rr;
    if (deflated) *deflated = nu;
    return TDBEM_OK;
}

// shared checks and set-up of tdbem_solve_fgmres and tdbem_precond_apply:
// validates the arguments, tunes the product if needed (on x, y), fills the
// solver plan and allocates its workspace
static tdbem_status krylov_setup(const tdbem_asm *A, int32_t restart, double tol, int32_t levels,
                                 const int32_t *inner, const double *x, double *y, KrylovSolver &K, DevBuf &ws,
                                 cudaStream_t st) {
    if (!A || !x || !y) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    if (!A->assembled) return fail(TDBEM_E_NOT_ASSEMBLED, "call tdbem_assemble_all first");
    if (restart < 1 || restart > KR_MAXM) return fail(TDBEM_E_INVALID_ARG, "restart must be in 1..62");
    if (!(tol > 0.0 && tol < 1.0)) return fail(TDBEM_E_INVALID_ARG, "tol must be in (0, 1)");
    if (levels < 0 || levels > KR_MAXLEVELS) return fail(TDBEM_E_INVALID_ARG, "levels must be in 0..24");
    if (levels > 0 && !inner) return fail(TDBEM_E_INVALID_ARG, "inner_iters is NULL");
    for (int l = 0; l < levels; ++l)
        if (inner[l] < 1 || inner[l] > KR_MAXM) return fail(TDBEM_E_INVALID_ARG, "inner iterations must be in 1..62");
    if (A->tg->p > 0) return fail(TDBEM_E_UNSUPPORTED, "the block-Hessenberg preconditioner takes p = 0");
    const int64_t N = A->tg->N, M = A->mesh->M;
    const size_t bytes = (size_t)(N * M) * sizeof(double);
    const char *xb = (const char *)x, *yb = (const char *)y;
    if (xb < yb + bytes && yb < xb + bytes) return fail(TDBEM_E_INVALID_ARG, "arrays overlap");
    int dev = 0, nsm = 0;
    CUDA_TRY(cudaGetDevice(&dev));
    CUDA_TRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
    if (A->mv_variant < 0) {
        tdbem_status ts = tune_matvec(A, x, y, nsm, st);
        if (ts) return ts;
    }
    K.op = MvOp{(const MvBlock *)A->mv_blk.p, (int)A->blocks.size(), A->fp64, (double *)A->mv_xT.p, M, (int)N, nsm,
                A->mv_variant};
    K.levels = levels;
    K.m[0] = restart;
    for (int l = 1; l <= levels; ++l) K.m[l] = inner[l - 1];
    K.tol = tol;
    size_t need = 0;
    K.layout(nullptr, &need);
    tdbem_status s = dev_alloc(ws, need, st);
    if (s) return s;
    CUDA_TRY(cudaMemsetAsync(ws.p, 0, need, st));
    K.layout(ws.p, &need);
    return TDBEM_OK;
}

tdbem_status tdbem_solve_fgmres(const tdbem_asm *A, const double *g, double *x, int32_t restart, double tol,
                                int32_t max_iter, int32_t levels, const int32_t *inner_iters, int32_t *iters,
                                double *rel_res, void *stream) {
    if (max_iter < 1) return fail(TDBEM_E_INVALID_ARG, "max_iter must be >= 1");
    cudaStream_t st = (cudaStream_t)stream;
    KrylovSolver K;
    DevBuf ws;
    tdbem_status s = krylov_setup(A, restart, tol, levels, inner_iters, g, x, K, ws, st);
    if (s) return s;
    cudaStream_t cap = nullptr;
    CUDA_TRY(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking));
    int it = 0;
    double rr = 0.0;
    const cudaError_t e = K.solve(g, x, max_iter, st, cap, &it, &rr);
    cudaStreamDestroy(cap);
    if (e != cudaSuccess) return fail(TDBEM_E_CUDA, std::string("FGMRES: ") + cudaGetErrorString(e));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (iters) *iters = it;
    if (rel_res) *rel_res = rr;
    return TDBEM_OK;
}

tdbem_status tdbem_precond_apply(const tdbem_asm *A, int32_t levels, const int32_t *inner_iters, double tol,
                                 const double *r, double *z, void *stream) {
    if (levels < 1) return fail(TDBEM_E_INVALID_ARG, "levels must be in 1..24");
    cudaStream_t st = (cudaStream_t)stream;
    KrylovSolver K;
    DevBuf ws;
    tdbem_status s = krylov_setup(A, 1, tol, levels, inner_iters, r, z, K, ws, st);
    if (s) return s;
    const cudaError_t e = K.apply_preconditioner(r, z, st);
    if (e != cudaSuccess) return fail(TDBEM_E_CUDA, std::string("preconditioner: ") + cudaGetErrorString(e));
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaStreamSynchronize(st));
    return TDBEM_OK;
}

tdbem_status tdbem_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops, void *stream) {
    CUDA_TRY(measure_fma_peaks(fp32_tflops, fp64_tflops, (cudaStream_t)stream));
    return TDBEM_OK;
}

tdbem_status tdbem_stats(const tdbem_asm *A, tdbem_stats_t *out) {
    if (!A || !out) return fail(TDBEM_E_INVALID_ARG, "NULL argument");
    *out = A->stats;
    out->matvec_variant = A->mv_variant;
    out->matvec_launches = mv_launches(A);
    return TDBEM_OK;
}

}  // extern "C"
