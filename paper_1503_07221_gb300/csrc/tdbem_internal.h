// Internal declarations of libtdbem: data layouts shared by the host planner
// (api.cu) and the kernels (table.cu, pattern.cu, far.cu, near.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/tdbem.h"

namespace tdbem {

// ---------------------------------------------------------------------------
// Classes of unique blocks on an equidistant grid.
//
// Write F / I / L for the first, an inner and the last time basis function
// (b_1, b_2..b_{N-1}, b_N in the paper's 1-based numbering). On an
// equidistant grid psi_{k,i}(r) depends only on r - (k - i) dt for every
// (test kind, trial kind) combination (Sec. 3.1, Eq. psiTildeRed and its
// analogues for the boundary functions), so each combination is one class
// with one prototype function Phi_c(q), q = r / dt, and the block of lag d
// evaluates Phi_c(q - d). Its support is q - d in (rho_c, rho_c + P_c), cut
// into P_c panels of unit width at the breakpoints of psi.
//
//   C1 (I test, F trial): blocks (d, 0),           d = 1..N-2, rho = -2, P = 3
//   C2 (I, I):            blocks (i + d, i),       d = -1..N-3, rho = -2, P = 4
//   C3 (L, I):            blocks (N-1, N-1-d),     d = 1..N-2, rho = -2, P = 3
//   specials, one block each, lag 0:
//   S00 (F,F) (0,0) rho 0 P 1;  S01 (F,I) (0,1) rho 0 P 1;
//   SN0 (L,F) (N-1,0) rho N-3 P 2;  SNN (L,L) (N-1,N-1) rho 0 P 1;
//   SN1N (I,L) (N-2,N-1) rho 0 P 1.
// ---------------------------------------------------------------------------
enum { C1 = 0, C2 = 1, C3 = 2, S00 = 3, S01 = 4, SN0 = 5, SNN = 6, SN1N = 7, NCLASS = 8 };
constexpr int NLAG = 3;   // classes C1..C3 carry a range of lags
constexpr int NSPEC = 5;  // the rest carry lag 0 only
constexpr int NCHEB = 33; // Chebyshev coefficients per panel (degree 32)
constexpr int MAXPANEL = 4;
constexpr int TOTAL_PANELS = 3 + 4 + 3 + 1 + 1 + 2 + 1 + 1;  // sum of P_c = 16
constexpr int TOTAL_LAG_PANELS = 3 + 4 + 3;                   // panels of C1..C3

struct ClassDesc {
    int rho;      // first panel starts at q - d = rho
    int P;        // panels
    int dlo, dhi; // lags of the blocks that exist (after the diam cut); dlo > dhi: none
    int kb_rep, ib_rep, d_rep;  // block used to sample the prototype
    int panel0;   // index of the class's first panel in the panel list
};

// Device-side view of everything the kernels read. Plain pointers only.
struct Geo {
    int64_t M, E;
    const int32_t *F;       // E x 3
    const double *cen;      // E x 3 centroids
    const double *dq;       // E x 7 x 3 quadrature points minus centroid (FP64)
    const float *dq32;      // same, FP32
    const double *V;        // M x 3
    const float *geo32;     // E x 16: n(3), area, curls(9), pad
    const double *geo64;    // E x 16: same in FP64
    const int64_t *vt_ptr;  // M + 1
    const int32_t *vt_tri;  // triangles around a vertex
};

// Status word bits written by kernels (plain stores; any nonzero value fails the call)
enum {
    ST_OFF_RANGE = 1,      // a point pair fell outside the accumulator window
    ST_WINDOW = 2,         // a vertex-pair lag window exceeded its storage
    ST_NEAR_ORDER = 4,     // near rule too large for shared memory
    ST_NBR = 8,            // near neighbour lookup failed
    ST_WAIT = 16,          // a bounded wait inside a kernel gave up
    ST_PBLIST = 32,        // the list of element pairs for the FP64 bound decisions overflowed
};

// Element-pair record of the bounds pass: kept lag range per lag class and a
// bit mask of kept special blocks. cnt = 0 means no lag of that class.
struct PairRec {
    int16_t lo[3];
    uint8_t cnt[3];
    uint8_t smask;
    uint8_t adj;   // number of shared vertices (0 far, 1 vertex, 2 edge, 3 same)
    uint8_t pad[5];
};
static_assert(sizeof(PairRec) == 16, "PairRec is 16 bytes");

// Per-class lag tables for the culling decisions (support endpoints computed
// on the host from the time grid exactly as Sec. 3.2 states them).
struct LagTables {
    const double *a[NCLASS];  // a_d for d = dlo..dhi (index d - dlo)
    const double *b[NCLASS];
    int dlo[NCLASS], dhi[NCLASS];
    int rho[NCLASS], P[NCLASS];
    double dt, inv_dt;
    double tie;  // support endpoints: bounds within tie of an endpoint count as equal (culled)
    double tol2; // band around FP32 squared distances inside which the FP64 bounds decide
};

// FP32 Chebyshev coefficients of all 16 panels (one sub-panel per unit),
// passed by value so kernels read them from the constant bank.
constexpr int NCHEB_LO = 4;  // leading coefficients carried as a hi + lo float pair
struct alignas(8) ChebF32 {  // 8-aligned: read as packed pairs
    float c[TOTAL_PANELS][NCHEB][2];      // (psi, psi~), rounded to FP32
    float lo[TOTAL_PANELS][NCHEB_LO][2];  // c - (double)(float)c of the leading ones
};

// The lag-class panels (C1: 0-2, C2: 3-6, C3: 7-9) for the mixed far kernel,
// term-major (the 10 coefficient pairs of one term are adjacent in the
// constant bank), with the sign pattern of its Chebyshev recurrence folded
// in: s_n c_n, s_n = +1, +1, -1, -1, ... by n mod 4.
struct alignas(8) ChebLag32 {
    float c[NCHEB][TOTAL_LAG_PANELS][2];
    float lo[NCHEB_LO][TOTAL_LAG_PANELS][2];
};

// ---- launchers (defined in the .cu files) --------------------------------
// table.cu
// bkind: step function of the time basis (0 erf(2 artanh), 1 exp(-1/s))
void launch_psi_samples(int bkind, const double *t, int N, const int *panel_class, const int *panel_kb,
                        const int *panel_ib, const double *panel_r0, double panel_dr, int S,
                        int total_sub, const double *gl_x, const double *gl_w, int gl_n, int gl_sub,
                        double *samples, cudaStream_t st);
void launch_psi_dct(const double *samples, int total_sub, double *coef, cudaStream_t st);
// evaluation of one block's table (lag, class panels) at n distances: out n x 2
void launch_psi_table(const double *r, int64_t n, double inv_dt, int lag, int rho, int P, int panel0, int S,
                      const double *c64, const ChebF32 &c32, int use32, double *out, cudaStream_t st);
// sub-panel p covers [r0[p], r0[p] + dr[p]] (uneven panels)
// (panel_m2, panel_m1: temporal orders of each panel's block, or null for 0)
void launch_psi_samples_var(int bkind, const double *t, int N, const int *panel_kb, const int *panel_ib,
                            const int *panel_m2, const int *panel_m1, const double *panel_r0, const double *panel_dr,
                            int total_sub, const double *gl_x, const double *gl_w, int gl_n, int gl_sub,
                            double *samples, cudaStream_t st);

// pattern.cu
// FP32 pass over all element pairs, then a dense FP64 pass over the pairs
// whose FP32 decision was not certain (list of capacity cap, count in cnt;
// capacity max(2^24, E^2 / 64), several times the uncertain share seen; an
// overflow sets ST_PBLIST in status)
constexpr int64_t PB_LIST_MIN = (int64_t)1 << 24;
void launch_pair_bounds(const Geo &g, const LagTables &lt, PairRec *rec, int64_t *list, int64_t cap,
                        unsigned long long *cnt, int *status, int nsm, cudaStream_t st);
// graded grids: exact (dmin, dmax) of every element pair, E x E
void launch_gpair_bounds(const Geo &g, double2 *out, cudaStream_t st);
void launch_vertex_windows(const Geo &g, const PairRec *rec, int16_t *dlo, int16_t *dhi,
                           uint8_t *smask, int KW, int *status, cudaStream_t st);
void launch_count_quad(const Geo &g, const PairRec *rec, const int *npp, int64_t *partial,
                       int nblocks_grid, cudaStream_t st);
void launch_row_counts2(int64_t M, const int16_t *dlo, const int16_t *dhi, const uint8_t *smask,
                        const int *cls_dlo, const int *cls_dhi, const int *blk_of_lag,
                        const int *lag_base, const int *blk_of_spec, const int64_t *nbr_ptr,
                        const int32_t *nbr, int64_t *cnt_far, int64_t *cnt_near, cudaStream_t st);
void launch_scan_rows(const int64_t *cnt, int64_t M, int nsets, int64_t *row_ptr, int64_t *totals,
                      cudaStream_t st);
void launch_fill(int64_t M, const int16_t *dlo, const int16_t *dhi, const uint8_t *smask,
                 const int *cls_dlo, const int *blk_of_lag, const int *lag_base,
                 const int *blk_of_spec, const int64_t *nbr_ptr, const int32_t *nbr,
                 const int64_t *row_ptr, const int64_t *blk_off, int32_t *col, const double *dense,
                 const double *dense_spec, void *val, int KW, int NB, bool fp64, int nxmax, cudaStream_t st);

// far.cu
struct FarArgs {
    Geo g;
    LagTables lt;
    const int16_t *dlo;        // 3 x M x M vertex-pair window starts
    const int16_t *dhi;
    const uint8_t *smask;      // M x M special masks
    const int32_t *color_tris; // triangles of the current colour
    int64_t ncolor;
    const int32_t *chunk_vptr; // per chunk of 32 triangles: vertex list offsets
    const int32_t *chunk_vert;
    const int32_t *chunk_sptr;
    const int32_t *chunk_src;  // sigma_local * 3 + corner
    const int4 *chunk_hdr;     // per chunk: first vertex, vertices, first source, sources
    int64_t nchunks;
    const float *rule_w;       // 7 weights
    const float *rule_l;       // 7 x 3 barycentrics
    const double *rule_w64;    // same in FP64
    const double *rule_l64;
    float rw32[7];             // 7-point rule weights and barycentrics by value
    float rl32[21];            // (constant bank in the FP32 kernel)
    int max_nv;                // most trial vertices in one chunk
    float gwh[21], gwl[21];    // w_k lambda_a(p_k) as FP32 pairs (hi, lo), index 3k + a
    float wwh[7], wwl[7];      // w_k as FP32 pairs
    // the 7-point rule by its orbits (centroid; points 1+k and 4+k with the
    // distinguished barycentric at corner k), FP32 pairs: w_0 / 3, w_1 a_1,
    // w_2 a_2 (kh, kl); w_0, w_1, w_2 (wh, wl); w_1 (b_1 - a_1), w_2 (b_2 - a_2)
    // (dh, dl), so that w_x lambda_a(x) = k_o + [a = k] d_o on orbit o
    float okh[3], okl[3], owh[3], owl[3], odh[2], odl[2];
    double *dense;             // 3 x M x M x KW lag windows, FP64 accumulation
    double *dense_spec;        // 5 x M x M
    int KW;
    int *status;
    const double *cheb64;      // TOTAL_PANELS * S * NCHEB * 2 (FP64 path)
    const float *cenh, *cenl;  // E x 3 centroids as FP32 pairs (mixed path)
    const float *geoh, *geol;  // E x 16 geometry (n, area, curls) as FP32 pairs
};
void launch_far(const FarArgs &a, const ChebF32 &c32, bool fp64, int off, int S, int grid,
                cudaStream_t st);
// far32.cu: W is the thread window in unit cells of r / dt,
// far32_window(max |y - c|, dt)
int far32_window(double max_dq, double dt);
size_t far32_smem(int W, int KW, int max_nv);
void launch_far32(const FarArgs &a, const ChebLag32 &c32, int W, int grid, cudaStream_t st);

// near.cu
struct NearArgs {
    Geo g;
    LagTables lt;
    const int16_t *dlo;
    const int16_t *dhi;
    const int32_t *color_tris;
    int64_t ncolor;
    const int64_t *adj_ptr;   // per triangle: adjacent-pair list offsets
    const int32_t *adj_tri;   // sigma
    const int8_t *adj_perm;   // per adjacent pair: kase, pa[3], pb[3], pad
    const int32_t *adj_nbr;   // per adjacent pair: 9 neighbour indices (a,b) of sigma's vertex in nbr(row)
    const PairRec *rec;       // element-pair records of the bounds pass
    const double *ss_xy[4];   // per kase 1..3: npp x 5 (xh0, xh1, yh0, yh1, w)
    int ss_npp[4];
    const double *cheb64;     // TOTAL_PANELS * S * NCHEB * 2
    int S;
    double *ndense;           // 3 x M x NB x KW
    double *ndense_spec;      // 5 x M x NB
    double *far_spec;         // 5 x M x M far-pair special-block values (FP64)
    const uint8_t *smask;     // M x M special masks of the vertex pairs
    const double *rule_w64;   // 7-point rule weights and barycentrics
    const double *rule_l64;
    int NB, KW;
    int *status;
};
void launch_near(const NearArgs &a, int grid, cudaStream_t st);
// near32.cu: the same near field with psi, psi~ in FP32 (mixed path)
void launch_near32(const NearArgs &a, const ChebF32 &c32, int grid, cudaStream_t st);
// far element pairs that reach a special block, 7-point rule, psi and psi~
// in FP32 with FP32-pair sums (mixed path; the FP64 far kernel handles them
// itself)
void launch_farspec32(const NearArgs &a, const ChebF32 &c32, int grid, cudaStream_t st);

// matvec.cu: one unique block and the diagonal run of block positions
// (k0 + p, i0 + p), p < cnt, that it stands for (Eq. relationAtildeBlock)
struct MvBlock {
    const int64_t *rp_far;
    const int32_t *col_far;
    const void *val_far;  // float (mixed) or double (FP64)
    const int64_t *rp_near;
    const int32_t *col_near;
    const double *val_near;
    int32_t k0, i0, cnt, pad;
};
// the blocks outside the Toeplitz class in the mixed path (no diagonal runs),
// x read in its (N, M) layout; writes every entry of y
cudaError_t launch_hessenberg_rest(const MvBlock *blk, int nb, const double *x, double *y, int64_t M, int N, int nsm,
                                   int variant, cudaStream_t st);

// toeplitz.cu: the Toeplitz class (inner blocks (k, 1) and (1, 2)) of the
// mixed path from per-pair lag windows of TL lags, added into y
struct TwArgs {
    int64_t M;
    int nin;                   // inner time indices N - 2
    int TL, S, PADL;           // lags per entry; row stride and left padding of the x copies (floats)
    const int64_t *fptr;       // far entries of row l: [fptr[l], fptr[l + 1])
    const int2 *fhdr;          // (trial vertex j, first lag)
    const float *fval;         // TL FP32 values per entry, stride TL rounded up to 4
    const int64_t *nptr;       // near entries, FP64 values
    const int2 *nhdr;
    const double *nval;
};
// lags per entry for the widest window (8, 9, 10, 12 or 16; -1 above 16)
int tw_lags(int maxw);
// outputs per lane of a matvec variant (the autotuner's index)
int tw_variant_outputs(int variant);
void tw_geometry(int TL, int max_lag, int N, int *PADL, int *S);
void launch_tw_count(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                     int64_t *cnt, unsigned long long *maxw, cudaStream_t st);
void launch_tw_fill(int64_t M, const int16_t *dlo, const int16_t *dhi, const int64_t *nbr_ptr, const int32_t *nbr,
                    int TL, const int64_t *ptr, const float2 *dense, const double *ndense, int KW, int NB, int2 *fhdr,
                    float *fval, int2 *nhdr, double *nval, cudaStream_t st);
// writes the four shifted FP32 copies of x (4 x M x S floats at xP), then
// adds the Toeplitz class into y with R outputs per lane (4, 8 or 16)
cudaError_t launch_toeplitz(const TwArgs &g, const double *x, float *xP, double *y, int R, int nsm, cudaStream_t st);

// transposes x (N, M) into xT (M, N), then y = A x; returns the launch status
// variant: one of MV_NVARIANTS launch shapes (0 = default), see matvec.cu
constexpr int MV_NVARIANTS = 6;
cudaError_t launch_hessenberg(const MvBlock *blk, int nb, bool far_fp64, const double *x, double *xT, double *y,
                              int64_t M, int N, int nsm, int variant, cudaStream_t st);
// y (nk, M) = A[ka:ka+nk, ia:ia+nx] x (nx, M) over block rows and columns;
// nothing happens when active is given and *active == 0 (device flag)
cudaError_t launch_hessenberg_range(const MvBlock *blk, int nb, bool far_fp64, const double *x, double *xT, double *y,
                                    int64_t M, int ka, int nk, int ia, int nx, const int *active, int nsm, int variant,
                                    cudaStream_t st);
// table.cu: right-hand side of the linear system (Neumann data by kind)
enum { RHS_PLANE_WAVE = 0, RHS_SPHERE_N0 = 1, RHS_SPHERE_N1 = 2 };
struct RhsParams {
    double p[5];
};
void launch_rhs(int bkind, const Geo &g, const double *t, int N, int P1, double c, const double *rule_w,
                const double *rule_l, const double *gx, const double *gw, int gn, int sub, int kind,
                const RhsParams &prm, double *out, cudaStream_t st);
// solve.cu: vector kernels of the GMRES solver
void launch_multi_dot(const double *V, int64_t ld, int nv, const double *w, int64_t n, double *partial, double *h,
                      cudaStream_t st, const int *active = nullptr);
void launch_multi_axpy(const double *V, int64_t ld, int nv, const double *h, double sign, double *w, int64_t n,
                       cudaStream_t st, const int *active = nullptr);
void launch_scale_copy(const double *w, const double *beta, double *v, int64_t n, cudaStream_t st);
// deflation.cu: basis B (m x m row-major, first *sdim columns) of the
// invariant subspace of the Hessenberg H for its l eigenvalues of smallest
// modulus, *lam_max the largest modulus; 0, or -1 if the QR iteration fails
int deflation_basis(const double *H, int m, int ldh, int l, double *B, int *sdim, double *lam_max);
constexpr int GM_BLOCKS = 256;   // blocks of the dot-product partial sums
constexpr int GM_MAXV = 64;      // most vectors in one multi_dot / multi_axpy

// fgmres.cu: flexible GMRES with the recursive block-Hessenberg
// preconditioner (Sec. 4.2, Algorithm 1), iterated on the device
constexpr int KR_MAXM = GM_MAXV - 2;  // most steps of one cycle
constexpr int KR_MAXLEVELS = 24;      // most levels of the preconditioner
// the status that the host reads after every outer step (the head of KState)
struct KHead {
    int run, stop, jdone, iters;
    double resid;
};
// one solve's scalars: run = the cycle goes on; stop = it ended converged
// (or at breakdown); resid = residual estimate / |b|; H row-major with row
// stride KR_MAXM; hc = the two Gram-Schmidt passes of the current step
struct KState {
    int run, stop, jdone, iters;
    double resid;
    int m, pad;
    double bref, inv, r2, w2;
    double hc[2 * GM_MAXV];
    double H[(KR_MAXM + 1) * KR_MAXM];
    double cs[KR_MAXM], sn[KR_MAXM], e[KR_MAXM + 1], y[KR_MAXM];
};
static_assert(offsetof(KState, resid) == offsetof(KHead, resid), "KHead is the head of KState");
// the block-Hessenberg product of one assembled matrix
struct MvOp {
    const MvBlock *blk;
    int nb;
    bool far_fp64;
    double *xT;  // scratch of N M doubles
    int64_t M;
    int N, nsm, variant;
};
class KrylovSolver {
  public:
    MvOp op{};
    int levels = 0;                   // preconditioner levels (0: none)
    int m[KR_MAXLEVELS + 1] = {};     // m[0] restart length, m[l] steps at level l
    double tol = 0.0;                 // relative tolerance, outer and inner
    int64_t graph_nodes = 0;          // nodes of the recorded preconditioner
    // sets the workspace pointers into ws (nullptr: only the size)
    cudaError_t layout(void *ws, size_t *bytes);
    // alpha with A alpha = g from zero; cap: a stream for graph capture
    cudaError_t solve(const double *g, double *x, int max_iter, cudaStream_t st, cudaStream_t cap, int *iters,
                      double *rel_res);
    // z = M^-1 r, one application of the level-1 preconditioner
    cudaError_t apply_preconditioner(const double *r, double *z, cudaStream_t st);

  private:
    int nblk[KR_MAXLEVELS + 1] = {};
    KState *states = nullptr;
    double *partial = nullptr, *pin = nullptr, *pout = nullptr;
    double *V[KR_MAXLEVELS + 1] = {}, *Z[KR_MAXLEVELS + 1] = {}, *w[KR_MAXLEVELS + 1] = {},
           *t[KR_MAXLEVELS + 1] = {};
    cudaError_t matvec(const double *x, double *y, int ka, int nk, int ia, int nx, const int *active,
                       cudaStream_t st);
    cudaError_t arnoldi(int l, int lo, int hi, int j, const double *z, cudaStream_t st);
    cudaError_t inner_solve(int l, int lo, int hi, const double *rhs, double *x, const int *parent, cudaStream_t st);
    cudaError_t precondition(int l, int lo, int hi, const double *in, double *out, const int *parent,
                             cudaStream_t st);
    cudaError_t read_head(KHead *h, cudaStream_t st);
};

// graded.cu: assembly on a non-equidistant time grid, where every nonzero
// block (k, i) with i <= k + 1 is its own unique block (no reuse along the
// diagonals). Blocks are numbered column-major internally: column i holds
// blocks k = colk0[i] .. colk0[i] + (colblk[i+1] - colblk[i]) - 1, a
// contiguous range (the supports a, b grow with k). Each block has GP_MAXPAN
// or fewer panels between the breakpoints t_{k-a} - t_{i-b} of psi.
constexpr int GP_MAXPAN = 8;
struct alignas(32) GPan64 {  // FP64 panel: start, width, S64 / width, unused
    double x, y, z, w;
};     // panels of one block
constexpr int GP_KSLOT = 4;      // blocks one far warp evaluates at a time
constexpr int GP_MAXK = 256;     // blocks of one trial column
constexpr int GF_WARPS = 16;     // warps of a far CTA
constexpr int GN_WARPS = 8;      // warps of a near CTA
constexpr int GN_TILE = 512;     // near point pairs staged at a time
struct GradedArgs {
    Geo g;
    int N;
    double tie;
    const double2 *pair;      // E x E element-pair (dmin, dmax)
    const double *vmin;       // M x M vertex-pair Dmin (min over the two stars)
    const double *vmax;       // M x M vertex-pair Dmax
    const double *ga, *gb;    // support (a, b) per column-major block
    const int *colblk;        // N + 1
    const int *colk0;         // N
    const int *pan0;          // column-major block -> first panel (nblk + 1)
    const GPan64 *pan64;     // per panel: (start, width, -, -)
    const float4 *pan32;      // per panel: (start_h, mid_h, mid_l, 2/width)
    const float *coef32;      // per panel: 34 x (psi, psi~), FP32 (entry 33 zero)
    const double *coef64;     // per FP64 coefficient set: 33 x (psi, psi~)
    const int *p64;           // per panel: first of its S64 FP64 sets (-1: none)
    int S64;
    int maxpan;               // most panels of one column
    // batch of trial columns [i0, i1) and its staging windows
    int i0, i1;
    const int64_t *doff;      // per batch column: offset (doubles) of its far windows
    const int64_t *ndoff;     // per batch column: offset of its near windows
    const int *kw;            // per column: window length KW_i
    double *dense;            // far: [l][j][KW_i] per batch column
    double *ndense;           // near: [l][nbr index][KW_i] per batch column
    int NB;
    // triangles
    const int32_t *color_tris; // test triangles of this launch (one colour)
    int64_t ncolor;
    const int32_t *all_tris;  // every triangle, grouped by colour
    const int64_t *col_off;   // colour offsets into all_tris (ncol + 1)
    int ncol;
    const float *cenh, *cenl; // E x 3 centroids as FP32 pairs
    const float *geoh, *geol; // E x 16 geometry (n, area, curls) as FP32 pairs
    // near field
    const int64_t *adj_ptr;
    const int32_t *adj_tri;
    const int8_t *adj_perm;
    const int32_t *adj_nbr;
    const double *ss_xy[4];
    int ss_npp[4];
    // 7-point rule: weights, barycentrics, w_k lambda_a(p_k) and w_k as FP32 pairs
    const double *rule_w64, *rule_l64;
    float gwh[21], gwl[21], wwh[7], wwl[7];
    int *status;
};
void launch_gfar(const GradedArgs &a, bool fp64, int grid, size_t smem, cudaStream_t st);
void launch_gnear(const GradedArgs &a, bool f32, int grid, cudaStream_t st);
// per (row, column): far and near row counts of every block of the column
void launch_gcount(const GradedArgs &a, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                   int64_t *cnt_far, int64_t *cnt_near, cudaStream_t st);
// vertex-pair Dmin / Dmax and per-CTA maxima of Dmax - Dmin (partial, nblocks entries)
void launch_gvertex(const GradedArgs &a, double *vmin, double *vmax, double *partial, int nblocks, cudaStream_t st);
// quadrature point pairs x kept blocks over all element pairs (per-CTA partial
// sums: partial[0, nblocks) all pairs, partial[nblocks, 2 nblocks) far pairs)
void launch_gcount_quad(const GradedArgs &a, int npp_far, const int *npp_near, int64_t *partial, int nblocks,
                        cudaStream_t st);
// CSR fill of the blocks of batch columns [a.i0, a.i1)
void launch_gfill(const GradedArgs &a, const int *cb2api, const int64_t *nbr_ptr, const int32_t *nbr,
                  const int64_t *rp_far, const int64_t *off_far, int32_t *col_far, void *val_far, bool fp64,
                  const int64_t *rp_near, const int64_t *off_near, int32_t *col_near, double *val_near,
                  cudaStream_t st);
size_t gfar_smem(int max_col_panels, bool fp64);
void launch_gcoef32(const double *coef, int npan, float *out, cudaStream_t st);

// potential.cu: retarded double layer potential at P points and nt times;
// workspace yw (E n^2 x 2 double4), coef (N E n^2 doubles) and the step
// table tab (DL_TABLE_NODES double3); equi: the grid is equidistant
constexpr int DL_TABLE_NODES = 1025;
cudaError_t launch_double_layer(int bkind, const Geo &g, const double *tg, int N, int equi, double c, const double *gx,
                                const double *gw, int n, const double *alpha, const double *X, int64_t P,
                                const double *times, int nt, double4 *yw, double *coef, double3 *tab, double *out,
                                cudaStream_t st);

// peaks.cu: FMA throughput of the device (roofline denominators)
cudaError_t measure_fma_peaks(double *fp32, double *fp64, cudaStream_t st);
// noalloc.cu: fixed scratch of MV_STATIC_MAX doubles for the matvec that
// allocates nothing; its address on the current device
constexpr int64_t MV_STATIC_MAX = (int64_t)1 << 21;
cudaError_t static_mv_scratch(double **ptr);

}  // namespace tdbem
