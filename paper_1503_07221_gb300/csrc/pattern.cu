// Culling and sparsity pattern (paper Sec. 3.2, Eq. SparsitySmallBlock):
// element-pair distance bounds and kept lag ranges, vertex-pair lag windows,
// per-block row counts, row offsets, and the CSR fill that gathers the
// assembled values into per-block CSR.
#include <math.h>

#include <type_traits>

#include <algorithm>
#include <cstddef>

#include "tdbem_internal.h"

namespace tdbem {

// ------------------------------------------------------------------ geometry
struct d3 { double x, y, z; };
__device__ static inline d3 ld3(const double *p) { return {p[0], p[1], p[2]}; }
__device__ static inline d3 sub(d3 a, d3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ static inline d3 add(d3 a, d3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ static inline d3 mul(d3 a, double s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ static inline double dot(d3 a, d3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }

__device__ static inline double clamp01(double x) { return x < 0.0 ? 0.0 : (x > 1.0 ? 1.0 : x); }

// The squared distance of a point to a triangle uses the seven Voronoi
// regions of the triangle (vertices, edges, interior); that of two segments
// minimises over [0,1]^2 by clamping the unconstrained minimiser and
// re-solving for the other parameter. Both are templated on the precision.
// ----------------------------------------------------------- bounds pass
// Lowest lag in [lo, hi] with b_d > x (b increasing in d); hi + 1 if none.
__device__ static int first_b_above(const double *b, int lo, int hi, double x) {
    int L = lo, H = hi + 1;
    while (L < H) {
        const int m = (L + H) >> 1;
        if (b[m - lo] > x) H = m; else L = m + 1;
    }
    return L;
}
// Highest lag in [lo, hi] with a_d < x (a increasing in d); lo - 1 if none.
__device__ static int last_a_below(const double *a, int lo, int hi, double x) {
    int L = lo - 1, H = hi;
    while (L < H) {
        const int m = (L + H + 1) >> 1;
        if (a[m - lo] < x) L = m; else H = m - 1;
    }
    return L;
}

// FP32 copies of the geometry helpers for the prefilter
struct f3 { float x, y, z; };
__device__ static inline f3 sub(f3 a, f3 b) { return {a.x - b.x, a.y - b.y, a.z - b.z}; }
__device__ static inline f3 add(f3 a, f3 b) { return {a.x + b.x, a.y + b.y, a.z + b.z}; }
__device__ static inline f3 mul(f3 a, float s) { return {a.x * s, a.y * s, a.z * s}; }
__device__ static inline float dot(f3 a, f3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ static inline float clamp01(float x) { return x < 0.f ? 0.f : (x > 1.f ? 1.f : x); }

template <typename V, typename T>
__device__ static T point_triangle_d2t(V p, V a, V b, V c) {
    const V ab = sub(b, a), ac = sub(c, a), ap = sub(p, a);
    const T d1 = dot(ab, ap), d2 = dot(ac, ap);
    if (d1 <= T(0) && d2 <= T(0)) return dot(ap, ap);
    const V bp = sub(p, b);
    const T d3_ = dot(ab, bp), d4 = dot(ac, bp);
    if (d3_ >= T(0) && d4 <= d3_) return dot(bp, bp);
    const T vc = d1 * d4 - d3_ * d2;
    if (vc <= T(0) && d1 >= T(0) && d3_ <= T(0)) {
        const V e = sub(p, add(a, mul(ab, d1 / (d1 - d3_))));
        return dot(e, e);
    }
    const V cp = sub(p, c);
    const T d5 = dot(ab, cp), d6 = dot(ac, cp);
    if (d6 >= T(0) && d5 <= d6) return dot(cp, cp);
    const T vb = d5 * d2 - d1 * d6;
    if (vb <= T(0) && d2 >= T(0) && d6 <= T(0)) {
        const V e = sub(p, add(a, mul(ac, d2 / (d2 - d6))));
        return dot(e, e);
    }
    const T va = d3_ * d6 - d5 * d4;
    if (va <= T(0) && (d4 - d3_) >= T(0) && (d5 - d6) >= T(0)) {
        const V e = sub(p, add(b, mul(sub(c, b), (d4 - d3_) / ((d4 - d3_) + (d5 - d6)))));
        return dot(e, e);
    }
    const T den = T(1) / (va + vb + vc);
    const V e = sub(p, add(a, add(mul(ab, vb * den), mul(ac, vc * den))));
    return dot(e, e);
}

template <typename V, typename T>
__device__ static T segment_segment_d2t(V p0, V p1, V q0, V q1) {
    const V d1 = sub(p1, p0), d2 = sub(q1, q0), r = sub(p0, q0);
    const T a = dot(d1, d1), e = dot(d2, d2), f = dot(d2, r);
    const T c = dot(d1, r), b = dot(d1, d2);
    const T den = a * e - b * b;
    T s = den > T(0) ? clamp01((b * f - c * e) / den) : T(0);
    T u = (b * s + f) / e;
    if (u < T(0)) { u = T(0); s = clamp01(-c / a); }
    else if (u > T(1)) { u = T(1); s = clamp01((b - c) / a); }
    const V w = sub(add(p0, mul(d1, s)), add(q0, mul(d2, u)));
    return dot(w, w);
}

// squared minimum and maximum distance of two triangles (dmin = 0 when
// they share a vertex: closed surfaces, touching triangles never intersect)
template <typename V, typename T>
__device__ static void tri_bounds2(const V *a, const V *b, bool shared, T &dmin2, T &dmax2) {
    T mx = T(0);
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) { const V d = sub(a[i], b[j]); mx = fmax(mx, dot(d, d)); }
    dmax2 = mx;
    if (shared) { dmin2 = T(0); return; }
    T m2 = T(1e30);
    for (int i = 0; i < 3; ++i) {
        m2 = fmin(m2, point_triangle_d2t<V, T>(a[i], b[0], b[1], b[2]));
        m2 = fmin(m2, point_triangle_d2t<V, T>(b[i], a[0], a[1], a[2]));
    }
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) m2 = fmin(m2, segment_segment_d2t<V, T>(a[i], a[(i + 1) % 3], b[j], b[(j + 1) % 3]));
    dmin2 = m2;
}

// Kept lag range of each lag class and kept special blocks from distance
// bounds (exact FP64 decisions: dmin < b_d - tie, dmax > a_d + tie).
__device__ static void decide(const LagTables &lt, double dmin, double dmax, PairRec &r) {
    for (int c = 0; c < NLAG; ++c) {
        r.lo[c] = 0; r.cnt[c] = 0;
        if (lt.dlo[c] > lt.dhi[c]) continue;
        const int lo = first_b_above(lt.b[c], lt.dlo[c], lt.dhi[c], dmin + lt.tie);
        const int hi = last_a_below(lt.a[c], lt.dlo[c], lt.dhi[c], dmax - lt.tie);
        if (lo <= hi) { r.lo[c] = (int16_t)lo; r.cnt[c] = (uint8_t)(hi - lo + 1); }
    }
    uint8_t sm = 0;
    for (int c = NLAG; c < NCLASS; ++c) {
        if (lt.dlo[c] > lt.dhi[c]) continue;
        if (dmin < lt.b[c][0] - lt.tie && dmax > lt.a[c][0] + lt.tie) sm |= (uint8_t)(1u << (c - NLAG));
    }
    r.smask = sm;
}

// The decisions of `decide` in FP32: thr holds, per class c from off[c],
// the thresholds b_d - tie (n_c of them) then a_d + tie, rounded to FP32.
__device__ static void decide32(const float *thr, const int *off, const LagTables &lt, float dmin, float dmax,
                                PairRec &r) {
    for (int c = 0; c < NLAG; ++c) {
        r.lo[c] = 0; r.cnt[c] = 0;
        const int n = lt.dhi[c] - lt.dlo[c] + 1;
        if (n <= 0) continue;
        const float *tb = thr + off[c], *ta = tb + n;
        int L = 0, H = n;  // first index with tb > dmin
        while (L < H) {
            const int m = (L + H) >> 1;
            if (tb[m] > dmin) H = m; else L = m + 1;
        }
        const int lo = L;
        L = -1; H = n - 1;  // last index with ta < dmax
        while (L < H) {
            const int m = (L + H + 1) >> 1;
            if (ta[m] < dmax) L = m; else H = m - 1;
        }
        const int hi = L;
        if (lo <= hi) { r.lo[c] = (int16_t)(lt.dlo[c] + lo); r.cnt[c] = (uint8_t)(hi - lo + 1); }
    }
    uint8_t sm = 0;
    for (int c = NLAG; c < NCLASS; ++c) {
        if (lt.dlo[c] > lt.dhi[c]) continue;
        if (dmin < thr[off[c]] && dmax > thr[off[c] + 1]) sm |= (uint8_t)(1u << (c - NLAG));
    }
    r.smask = sm;
}

// One thread per element pair. The bounds are first computed in FP32, and
// the lag decisions are taken in FP32 at both ends of a band around them:
// the squared distances +-2 tol2 (tol2 covers their FP32 rounding with a
// wide margin, the second tol2 the rounding of the band ends and square
// roots), widened by 2^-20 max(T, d) for the FP32 rounding of the
// thresholds. Where both ends give the same decisions, no threshold lies
// between them and the exact FP64 distance decides the same; only where they
// differ is the pair recomputed exactly in FP64 and decided in FP64. The
// decisions are therefore those of the FP64 computation.
// FP32 pass for one pair: writes the record when the two ends agree and
// returns false; returns true when the pair needs the FP64 decision.
__device__ static bool pair_bounds_one(const Geo &g, const LagTables &lt, PairRec *rec, int64_t q, int64_t s,
                                       const float *pb_thr, const int *pb_off, float tmax) {
    const int32_t *A = g.F + 3 * q, *B = g.F + 3 * s;
    int shared = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) shared += (A[i] == B[j]);
    f3 a[3], b[3];
    for (int i = 0; i < 3; ++i) {
        const double *pa = g.V + 3 * A[i], *pb = g.V + 3 * B[i];
        a[i] = {(float)pa[0], (float)pa[1], (float)pa[2]};
        b[i] = {(float)pb[0], (float)pb[1], (float)pb[2]};
    }
    float mn2, mx2;
    tri_bounds2<f3, float>(a, b, shared != 0, mn2, mx2);
    PairRec r0, r1;
    const float t2 = 2.0f * (float)lt.tol2;
    const float hx = sqrtf(mx2 + t2);
    const float mg = 9.5367431640625e-07f * fmaxf(tmax, hx);  // 2^-20 max(|threshold|, d)
    const float lx = sqrtf(fmaxf(mx2 - t2, 0.f)) - mg;
    const float ln = shared ? 0.f : sqrtf(fmaxf(mn2 - t2, 0.f)) - mg, hn = shared ? 0.f : sqrtf(mn2 + t2) + mg;
    decide32(pb_thr, pb_off, lt, ln, lx, r0);
    decide32(pb_thr, pb_off, lt, hn, hx + mg, r1);
    bool same = r0.smask == r1.smask;
    for (int c = 0; c < NLAG; ++c) same = same && r0.lo[c] == r1.lo[c] && r0.cnt[c] == r1.cnt[c];
    if (!same) return true;
    PairRec r = r0;
    r.adj = (uint8_t)shared;
    for (int k = 0; k < 5; ++k) r.pad[k] = 0;
    rec[q * g.E + s] = r;
    return false;
}

// FP64 decision of one pair (exact bounds, FP64 decide)
__device__ static void pair_bounds_fp64(const Geo &g, const LagTables &lt, PairRec *rec, int64_t q, int64_t s) {
    const int32_t *A = g.F + 3 * q, *B = g.F + 3 * s;
    int shared = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) shared += (A[i] == B[j]);
    d3 ad[3], bd[3];
    for (int i = 0; i < 3; ++i) { ad[i] = ld3(g.V + 3 * A[i]); bd[i] = ld3(g.V + 3 * B[i]); }
    double dn2, dx2;
    tri_bounds2<d3, double>(ad, bd, shared != 0, dn2, dx2);
    PairRec r;
    decide(lt, shared ? 0.0 : sqrt(dn2), sqrt(dx2), r);
    r.adj = (uint8_t)shared;
    for (int k = 0; k < 5; ++k) r.pad[k] = 0;
    rec[q * g.E + s] = r;
}

// One CTA per test triangle q, its threads over the trial triangles.
__global__ void __launch_bounds__(256, 4) pair_bounds_kernel(Geo g, LagTables lt, PairRec *rec, int64_t *list, int64_t cap,
                                   unsigned long long *cnt, int *status) {
    extern __shared__ float pb_thr[];
    __shared__ int pb_off[NCLASS + 1];
    __shared__ float pb_tmax;
    if (threadIdx.x == 0) {
        int o = 0;
        for (int c = 0; c < NCLASS; ++c) {
            pb_off[c] = o;
            o += 2 * max(lt.dhi[c] - lt.dlo[c] + 1, 0);
        }
        pb_off[NCLASS] = o;
    }
    __syncthreads();
    for (int c = 0; c < NCLASS; ++c) {
        const int n = max(lt.dhi[c] - lt.dlo[c] + 1, 0);
        for (int i = threadIdx.x; i < n; i += blockDim.x) {
            pb_thr[pb_off[c] + i] = (float)(lt.b[c][i] - lt.tie);
            pb_thr[pb_off[c] + n + i] = (float)(lt.a[c][i] + lt.tie);
        }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        float t = 0.f;
        for (int i = 0; i < pb_off[NCLASS]; ++i) t = fmaxf(t, fabsf(pb_thr[i]));
        pb_tmax = t;
    }
    __syncthreads();
    const int64_t q = blockIdx.x;  // test
    const int lane = threadIdx.x & 31;
    for (int64_t s0 = 0; s0 < g.E; s0 += blockDim.x) {  // trial
        const int64_t s = s0 + threadIdx.x;
        const bool need = s < g.E && pair_bounds_one(g, lt, rec, q, s, pb_thr, pb_off, pb_tmax);
        // the pairs that need FP64 go to a list for a dense second pass (one
        // atomic per warp; the FP64 code stays out of this kernel, which keeps
        // its registers low); past the list's capacity the status flags it
        const unsigned bal = __ballot_sync(0xffffffffu, need);
        if (!bal) continue;
        unsigned long long base = 0;
        if (lane == __ffs(bal) - 1) base = atomicAdd(cnt, (unsigned long long)__popc(bal));
        base = __shfl_sync(0xffffffffu, base, __ffs(bal) - 1);
        if (need) {
            const unsigned long long idx = base + __popc(bal & ((1u << lane) - 1u));
            if (idx < (unsigned long long)cap) list[idx] = q * g.E + s;
            else *status |= ST_PBLIST;
        }
    }
}

// the listed pairs, one thread each
__global__ void pair_bounds_list_kernel(Geo g, LagTables lt, PairRec *rec, const int64_t *list, int64_t cap,
                                        const unsigned long long *cnt) {
    const int64_t n = min((int64_t)*cnt, cap);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const int64_t id = list[i];
        pair_bounds_fp64(g, lt, rec, id / g.E, id % g.E);
    }
}


void launch_pair_bounds(const Geo &g, const LagTables &lt, PairRec *rec, int64_t *list, int64_t cap,
                        unsigned long long *cnt, int *status, int nsm, cudaStream_t st) {
    int nthr = 0;
    for (int c = 0; c < NCLASS; ++c) nthr += 2 * std::max(lt.dhi[c] - lt.dlo[c] + 1, 0);
    cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st);
    pair_bounds_kernel<<<(unsigned)g.E, 256, (size_t)nthr * sizeof(float), st>>>(g, lt, rec, list, cap, cnt, status);
    pair_bounds_list_kernel<<<nsm * 8, 128, 0, st>>>(g, lt, rec, list, cap, cnt);
}

// Graded grids: exact FP64 bounds (dmin, dmax) of every element pair (dmin
// = 0 when the triangles share a vertex); the kept blocks follow from them
// per trial column (Sec. 3.2).
__global__ void gpair_bounds_kernel(Geo g, double2 *out) {
    const int64_t s = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;  // trial
    const int64_t q = blockIdx.y;                                       // test
    if (s >= g.E) return;
    const int32_t *A = g.F + 3 * q, *B = g.F + 3 * s;
    int shared = 0;
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) shared += (A[i] == B[j]);
    d3 ad[3], bd[3];
    for (int i = 0; i < 3; ++i) { ad[i] = ld3(g.V + 3 * A[i]); bd[i] = ld3(g.V + 3 * B[i]); }
    double dn2, dx2;
    tri_bounds2<d3, double>(ad, bd, shared != 0, dn2, dx2);
    out[q * g.E + s] = make_double2(sqrt(dn2), sqrt(dx2));
}

void launch_gpair_bounds(const Geo &g, double2 *out, cudaStream_t st) {
    dim3 grid((unsigned)((g.E + 127) / 128), (unsigned)g.E);
    gpair_bounds_kernel<<<grid, 128, 0, st>>>(g, out);
}

// --------------------------------------------------- vertex-pair windows
// Window of vertex pair (l, j): union over tau in star(l), sigma in star(j)
// of the element-pair lag ranges (an interval, since both stars are
// connected). Layout [c][l][j]; an empty window has dlo > dhi. A thread
// keeps the first VW_STAR triangles of star(j) in registers and reads each
// record as one aligned 16-byte load, all loads of one tau issued together;
// stars with more triangles finish in a loop.
constexpr int VW_STAR = 8;
static_assert(offsetof(PairRec, lo) == 0 && offsetof(PairRec, cnt) == 6 && offsetof(PairRec, smask) == 9,
              "vw_add unpacks PairRec by these offsets");

__device__ __forceinline__ void vw_add(const int4 v, int (&lo)[3], int (&hi)[3], unsigned &sm) {
    // PairRec: lo[3] (int16), cnt[3] (uint8), smask, adj, pad
    const int l0 = (int)(short)(v.x & 0xffff), l1 = (int)(short)((unsigned)v.x >> 16);
    const int l2 = (int)(short)(v.y & 0xffff);
    const int c0 = ((unsigned)v.y >> 16) & 0xff, c1 = ((unsigned)v.y >> 24) & 0xff, c2 = v.z & 0xff;
    if (c0) { lo[0] = min(lo[0], l0); hi[0] = max(hi[0], l0 + c0 - 1); }
    if (c1) { lo[1] = min(lo[1], l1); hi[1] = max(hi[1], l1 + c1 - 1); }
    if (c2) { lo[2] = min(lo[2], l2); hi[2] = max(hi[2], l2 + c2 - 1); }
    sm |= ((unsigned)v.z >> 8) & 0xff;
}

__global__ void vertex_windows_kernel(Geo g, const PairRec *rec, int16_t *dlo, int16_t *dhi,
                                      uint8_t *smask, int KW, int *status) {
    const int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t l = blockIdx.y;
    if (j >= g.M) return;
    int lo[3] = {32767, 32767, 32767}, hi[3] = {-32768, -32768, -32768};
    unsigned sm = 0;
    const int64_t y0 = g.vt_ptr[j], ny = g.vt_ptr[j + 1] - y0;
    int sig[VW_STAR];
#pragma unroll
    for (int y = 0; y < VW_STAR; ++y) sig[y] = y < ny ? g.vt_tri[y0 + y] : 0;
    const int4 *R = reinterpret_cast<const int4 *>(rec);
    for (int64_t x = g.vt_ptr[l]; x < g.vt_ptr[l + 1]; ++x) {
        const int4 *row = R + (int64_t)g.vt_tri[x] * g.E;
        int4 v[VW_STAR];
#pragma unroll
        for (int y = 0; y < VW_STAR; ++y) v[y] = y < ny ? __ldg(row + sig[y]) : make_int4(0, 0, 0, 0);
#pragma unroll
        for (int y = 0; y < VW_STAR; ++y) vw_add(v[y], lo, hi, sm);  // an empty record adds nothing
        for (int64_t y = VW_STAR; y < ny; ++y) vw_add(__ldg(row + g.vt_tri[y0 + y]), lo, hi, sm);
    }
    const int64_t MM = g.M * g.M;
    for (int c = 0; c < 3; ++c) {
        if (lo[c] <= hi[c] && hi[c] - lo[c] + 1 > KW) status[0] = ST_WINDOW;
        dlo[c * MM + l * g.M + j] = (int16_t)lo[c];
        dhi[c * MM + l * g.M + j] = (int16_t)hi[c];
    }
    smask[l * g.M + j] = (uint8_t)sm;
}

void launch_vertex_windows(const Geo &g, const PairRec *rec, int16_t *dlo, int16_t *dhi,
                           uint8_t *smask, int KW, int *status, cudaStream_t st) {
    dim3 grid((unsigned)((g.M + 127) / 128), (unsigned)g.M);
    vertex_windows_kernel<<<grid, 128, 0, st>>>(g, rec, dlo, dhi, smask, KW, status);
}

// ------------------------------------------ quadrature point-pair counter
// sum over element pairs of (point pairs of its rule) x (kept blocks);
// per-CTA partial sums, added up on the host (no atomics).
__global__ void count_quad_kernel(Geo g, const PairRec *rec, int npp0, int npp1, int npp2,
                                  int npp3, int64_t *partial) {
    __shared__ int64_t red[256];
    const int64_t n = g.E * g.E;
    int64_t acc = 0;
    for (int64_t x = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; x < n;
         x += (int64_t)gridDim.x * blockDim.x) {
        const PairRec r = rec[x];
        const int k = r.cnt[0] + r.cnt[1] + r.cnt[2] + __popc(r.smask);
        const int npp = r.adj == 0 ? npp0 : (r.adj == 1 ? npp1 : (r.adj == 2 ? npp2 : npp3));
        acc += (int64_t)k * npp;
    }
    red[threadIdx.x] = acc;
    __syncthreads();
    for (int s = 128; s > 0; s >>= 1) {
        if (threadIdx.x < s) red[threadIdx.x] += red[threadIdx.x + s];
        __syncthreads();
    }
    if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

void launch_count_quad(const Geo &g, const PairRec *rec, const int *npp, int64_t *partial,
                       int nblocks_grid, cudaStream_t st) {
    count_quad_kernel<<<nblocks_grid, 256, 0, st>>>(g, rec, npp[0], npp[1], npp[2], npp[3], partial);
}

// ------------------------------------------------------------ row counts
// One warp per (class, row). blockIdx.y = 0: far pattern over all columns,
// 1: near sub-pattern over the row's neighbour list. Lag classes histogram
// their window lags in shared memory; specials count their mask bits.
constexpr int RC_WARPS = 8;
constexpr int MAXLAG = 1024;

__global__ void row_counts_kernel(int64_t M, const int16_t *dlo, const int16_t *dhi,
                                  const uint8_t *smask, const int *cls_dlo, const int *cls_dhi,
                                  const int *blk_of_lag, const int *lag_base, const int *blk_of_spec,
                                  const int64_t *nbr_ptr, const int32_t *nbr, int64_t *cnt_far,
                                  int64_t *cnt_near) {
    __shared__ int hist[RC_WARPS][MAXLAG];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int64_t item = blockIdx.x * (int64_t)RC_WARPS + w;  // (c, l) with c in 0..3 (3 = specials)
    const bool nearp = blockIdx.y == 1;
    int64_t *cnt = nearp ? cnt_near : cnt_far;
    if (item >= 4 * M) return;
    const int c = (int)(item / M);
    const int64_t l = item % M;
    const int64_t MM = M * M;
    const int64_t k0 = nearp ? nbr_ptr[l] : 0, k1 = nearp ? nbr_ptr[l + 1] : M;
    if (c < 3) {
        const int nl = cls_dhi[c] - cls_dlo[c] + 1;
        if (nl <= 0) return;
        for (int x = lane; x < nl; x += 32) hist[w][x] = 0;
        __syncwarp();
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            const int64_t j = nearp ? nbr[k] : k;
            const int a = dlo[c * MM + l * M + j], b = dhi[c * MM + l * M + j];
            for (int d = a; d <= b; ++d) atomicAdd(&hist[w][d - cls_dlo[c]], 1);
        }
        __syncwarp();
        for (int x = lane; x < nl; x += 32) {
            const int blk = blk_of_lag[lag_base[c] + x];
            cnt[(int64_t)blk * M + l] = hist[w][x];
        }
    } else {
        int n[NSPEC] = {0, 0, 0, 0, 0};
        for (int64_t k = k0 + lane; k < k1; k += 32) {
            const int64_t j = nearp ? nbr[k] : k;
            const unsigned m = smask[l * M + j];
            for (int s = 0; s < NSPEC; ++s) n[s] += (m >> s) & 1u;
        }
        for (int s = 0; s < NSPEC; ++s) {
            int v = n[s];
            for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
            if (lane == 0 && blk_of_spec[s] >= 0) cnt[(int64_t)blk_of_spec[s] * M + l] = v;
        }
    }
}

void launch_row_counts2(int64_t M, const int16_t *dlo, const int16_t *dhi, const uint8_t *smask,
                        const int *cls_dlo, const int *cls_dhi, const int *blk_of_lag,
                        const int *lag_base, const int *blk_of_spec, const int64_t *nbr_ptr,
                        const int32_t *nbr, int64_t *cnt_far, int64_t *cnt_near, cudaStream_t st) {
    dim3 grid((unsigned)((4 * M + RC_WARPS - 1) / RC_WARPS), 2);
    row_counts_kernel<<<grid, RC_WARPS * 32, 0, st>>>(M, dlo, dhi, smask, cls_dlo, cls_dhi,
                                                     blk_of_lag, lag_base, blk_of_spec, nbr_ptr,
                                                     nbr, cnt_far, cnt_near);
}

// --------------------------------------------------------- row offset scan
// One CTA per block: row_ptr[b][0..M] = exclusive scan of cnt[b][0..M-1].
__global__ void scan_rows_kernel(const int64_t *cnt, int64_t M, int64_t *row_ptr, int64_t *totals) {
    __shared__ int64_t sh[1024];
    const int64_t b = blockIdx.x;
    const int64_t *c = cnt + b * M;
    int64_t *rp = row_ptr + b * (M + 1);
    int64_t carry = 0;
    for (int64_t base = 0; base < M; base += 1024) {
        const int64_t i = base + threadIdx.x;
        const int64_t v = i < M ? c[i] : 0;
        sh[threadIdx.x] = v;
        __syncthreads();
        for (int o = 1; o < 1024; o <<= 1) {
            const int64_t add = threadIdx.x >= o ? sh[threadIdx.x - o] : 0;
            __syncthreads();
            sh[threadIdx.x] += add;
            __syncthreads();
        }
        if (i < M) rp[i] = carry + sh[threadIdx.x] - v;
        const int64_t tot = sh[1023];
        __syncthreads();
        carry += tot;
    }
    if (threadIdx.x == 0) { rp[M] = carry; totals[b] = carry; }
}

void launch_scan_rows(const int64_t *cnt, int64_t M, int nsets, int64_t *row_ptr, int64_t *totals,
                      cudaStream_t st) {
    if (nsets <= 0) return;
    scan_rows_kernel<<<nsets, 1024, 0, st>>>(cnt, M, row_ptr, totals);
}

// ---------------------------------------------------------------- CSR fill
// One warp per (class, row); columns are visited in increasing order in
// chunks of 32, and for every lag present in the chunk a ballot assigns the
// positions, so each row comes out sorted by column.
template <typename T>
__global__ void fill_kernel(int64_t M, const int16_t *dlo, const int16_t *dhi, const uint8_t *smask,
                            const int *cls_dlo, const int *blk_of_lag, const int *lag_base,
                            const int *blk_of_spec, const int64_t *nbr_ptr, const int32_t *nbr,
                            const int64_t *row_ptr, const int64_t *blk_off, int32_t *col,
                            const double *dense, const double *dense_spec, T *val, int KW, int NB, int nxmax) {
    // per warp: the next CSR position of row l in the block of every lag of
    // the class (block offset + row start + entries written so far)
    extern __shared__ int64_t fill_pos[];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    int64_t *cur = fill_pos + (size_t)w * nxmax;
    const int64_t item = blockIdx.x * (int64_t)RC_WARPS + w;
    if (item >= 4 * M) return;
    const bool nearp = nbr_ptr != nullptr;
    const int c = (int)(item / M);
    const int64_t l = item % M;
    const int64_t MM = M * M;
    const int64_t k0 = nearp ? nbr_ptr[l] : 0, k1 = nearp ? nbr_ptr[l + 1] : M;
    const unsigned lt_mask = (1u << lane) - 1u;
    if (c < 3) {
        const int nx = lag_base[c + 1] - lag_base[c];
        for (int x = lane; x < nx; x += 32) {
            const int blk = blk_of_lag[lag_base[c] + x];
            cur[x] = blk >= 0 ? blk_off[blk] + row_ptr[(int64_t)blk * (M + 1) + l] : 0;
        }
        __syncwarp();
        for (int64_t kb = k0; kb < k1; kb += 32) {
            const int64_t k = kb + lane;
            const bool ok = k < k1;
            const int64_t j = ok ? (nearp ? nbr[k] : k) : 0;
            int a = 32767, b = -32768;
            if (ok) { a = dlo[c * MM + l * M + j]; b = dhi[c * MM + l * M + j]; }
            int ca = a, cb = b;
            for (int o = 16; o > 0; o >>= 1) {
                ca = min(ca, __shfl_xor_sync(0xffffffffu, ca, o));
                cb = max(cb, __shfl_xor_sync(0xffffffffu, cb, o));
            }
            for (int d = ca; d <= cb; ++d) {
                const bool in = a <= d && d <= b;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (!bal) continue;
                const int x = d - cls_dlo[c];
                if (in) {
                    const int64_t pos = cur[x] + __popc(bal & lt_mask);
                    col[pos] = (int32_t)j;
                    const int64_t src = nearp ? ((c * M + l) * NB + (k - k0)) : (c * MM + l * M + j);
                    if constexpr (std::is_same<T, float>::value) {
                        // mixed far windows hold FP32 pairs (hi, lo)
                        const float2 pr = reinterpret_cast<const float2 *>(dense)[src * KW + (d - a)];
                        val[pos] = pr.x + pr.y;
                    } else {
                        val[pos] = (T)dense[src * KW + (d - a)];
                    }
                }
                __syncwarp();
                if (lane == 0) cur[x] += __popc(bal);
                __syncwarp();
            }
        }
    } else {
        int64_t sc[NSPEC];
#pragma unroll
        for (int s = 0; s < NSPEC; ++s) {
            const int blk = blk_of_spec[s];
            sc[s] = blk >= 0 ? blk_off[blk] + row_ptr[(int64_t)blk * (M + 1) + l] : 0;
        }
        for (int64_t kb = k0; kb < k1; kb += 32) {
            const int64_t k = kb + lane;
            const bool ok = k < k1;
            const int64_t j = ok ? (nearp ? nbr[k] : k) : 0;
            const unsigned m = ok ? smask[l * M + j] : 0u;
            for (int s = 0; s < NSPEC; ++s) {
                const bool in = (m >> s) & 1u;
                const unsigned bal = __ballot_sync(0xffffffffu, in);
                if (!bal) continue;
                const int blk = blk_of_spec[s];
                if (in && blk >= 0) {
                    const int64_t pos = sc[s] + __popc(bal & lt_mask);
                    col[pos] = (int32_t)j;
                    const int64_t src = nearp ? ((s * M + l) * NB + (k - k0)) : (s * MM + l * M + j);
                    val[pos] = (T)dense_spec[src];
                }
                sc[s] += __popc(bal);
            }
        }
    }
}

void launch_fill(int64_t M, const int16_t *dlo, const int16_t *dhi, const uint8_t *smask,
                 const int *cls_dlo, const int *blk_of_lag, const int *lag_base,
                 const int *blk_of_spec, const int64_t *nbr_ptr, const int32_t *nbr,
                 const int64_t *row_ptr, const int64_t *blk_off, int32_t *col, const double *dense,
                 const double *dense_spec, void *val, int KW, int NB, bool fp64, int nxmax, cudaStream_t st) {
    const unsigned grid = (unsigned)((4 * M + RC_WARPS - 1) / RC_WARPS);
    nxmax = std::max(nxmax, 1);
    const size_t smem = (size_t)RC_WARPS * nxmax * sizeof(int64_t);
    if (fp64) {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(fill_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fill_kernel<double><<<grid, RC_WARPS * 32, smem, st>>>(
            M, dlo, dhi, smask, cls_dlo, blk_of_lag, lag_base, blk_of_spec, nbr_ptr, nbr, row_ptr,
            blk_off, col, dense, dense_spec, (double *)val, KW, NB, nxmax);
    } else {
        if (smem > 48 * 1024)
            cudaFuncSetAttribute(fill_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        fill_kernel<float><<<grid, RC_WARPS * 32, smem, st>>>(
            M, dlo, dhi, smask, cls_dlo, blk_of_lag, lag_base, blk_of_spec, nbr_ptr, nbr, row_ptr,
            blk_off, col, dense, dense_spec, (float *)val, KW, NB, nxmax);
    }
}

}  // namespace tdbem
