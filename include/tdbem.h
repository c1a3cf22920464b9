/*
 * tdbem.h -- C ABI of libtdbem, the GB300 (sm_103a) assembler of the
 * space-time Galerkin system of the time-domain hypersingular operator
 * (3-D wave equation, Neumann data), after Veit, Merta, Zapletal, Lukas,
 * "Efficient solution of time-domain boundary integral equations arising in
 * sound-hard scattering".
 *
 * What is assembled (paper Sec. 3, Eq. MatrixEntries):
 *
 *   A_{k,i}(l,j) = int_G int_G [ n_x.n_y phi_j(y) phi_l(x) psi_{k,i}(|x-y|)
 *                   + curl phi_j(y) . curl phi_l(x) psi~_{k,i}(|x-y|) ]
 *                  / (4 pi |x-y|) dG_y dG_x
 *
 *   psi_{k,i}(r) = int_0^T b''_i(t-r) b'_k(t) dt,
 *   psi~_{k,i}(r) = int_0^T b_i(t-r) b'_k(t) dt          (Eq. psis)
 *
 * with continuous piecewise-linear hat functions phi on a flat triangle
 * mesh and the C-infinity partition-of-unity time basis b of Sec. 3
 * (Eq. BasisFunctions; p = 0, or p = 1, 2 with the Legendre factors of
 * b_{i,m}, m = 0..p). Row = test (k, l), column = trial (i, j);
 * every block is spatially symmetric, so this is also the paper's A_{k,i}(j,l).
 *
 * Blocks (Sec. 3.2): A is block Hessenberg (Eq. Apartitioned); block (k,i)
 * vanishes when the support [a,b] of psi_{k,i} (a = max(0, t_{k-2} - t_i),
 * b = t_k - t_{i-2}, 1-based) starts at or beyond diam(Gamma). On an
 * equidistant grid only the blocks of Sec. 5.1 are assembled -- the first two
 * block columns, the last block row, A_{2,3} and A_{N-1,N} -- and every other
 * block is one of them by Eq. relationAtildeBlock. On any other grid (for
 * instance geometrically graded steps) the shift invariance is lost and
 * every nonzero block (k,i), i <= k+1, is assembled from its own psi_{k,i}
 * (Sec. 3, "O(N^2 p^2)" distinct functions); the list is k-major in both
 * cases. Within a block, entry
 * (l,j) is structural iff the open support (a,b) meets [mindist_{l,j},
 * maxdist_{l,j}] (Eq. SparsitySmallBlock); such entries stay in the pattern
 * even where they evaluate to 0.
 *
 * Quadrature: element pairs without a shared vertex use the 7-point
 * degree-5 triangle rule on both triangles (49 point pairs); pairs sharing a
 * vertex, an edge or the triangle use Sauter-Schwab regularising maps with
 * Gauss-Legendre points per direction. psi and psi~ come from piecewise
 * Chebyshev tables (Sec. 3.1) built on the device from a direct 1-D
 * Gauss-Legendre quadrature of Eq. psis.
 *
 * Indices are 0-based (the paper's are 1-based): time basis k, i in
 * 0..N-1 for N grid points t_0 = 0 < ... < t_{N-1} = T.
 *
 * Conventions for every call:
 *   - Host input arrays are copied; the caller keeps ownership.
 *   - Device pointers returned by tdbem_block_csr are borrowed: valid until
 *     the next assemble call or tdbem_asm_destroy.
 *   - Work is queued on the given CUDA stream (cudaStream_t passed as void*,
 *     NULL = legacy default stream). Calls that return data to the host
 *     synchronise that stream.
 *   - Errors are returned as status codes; no exception crosses the ABI and
 *     nothing aborts. tdbem_last_error() describes the last failure of the
 *     calling thread.
 *   - Device memory comes from the allocator registered with
 *     tdbem_set_allocator (else cudaMalloc / cudaFree).
 */
#ifndef TDBEM_H
#define TDBEM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* entry points are the only exported symbols of libtdbem.so */
#if defined(__GNUC__)
#define TDBEM_API __attribute__((visibility("default")))
#else
#define TDBEM_API
#endif

typedef int tdbem_status;
#define TDBEM_OK 0
#define TDBEM_E_INVALID_ARG 1   /* NULL pointer, size or option out of range */
#define TDBEM_E_MESH 2          /* degenerate triangle, bad index, NaN vertex */
#define TDBEM_E_TIMEGRID 3      /* N < 3, t_0 != 0, not strictly increasing */
#define TDBEM_E_OOM 4           /* device allocation failed */
#define TDBEM_E_CUDA 5          /* a CUDA runtime call failed */
#define TDBEM_E_DEVICE 6        /* a kernel reported an inconsistency (status word) */
#define TDBEM_E_NOT_ASSEMBLED 7 /* values requested before an assemble call */
#define TDBEM_E_UNSUPPORTED 8   /* configuration not supported by this build */
#define TDBEM_E_NUMERIC 9       /* a host iteration (Schur form of a small Hessenberg matrix) did not converge */

/* Precision of the far field (element pairs without a shared vertex). */
#define TDBEM_PREC_FP64 0  /* plain: everything in FP64 */
#define TDBEM_PREC_MIXED 1 /* FP32 quadrature and Chebyshev evaluation with
                              FP64 element-pair distances; near field FP64 */

/* Which values tdbem_block_csr returns. */
#define TDBEM_FAR 0  /* full block pattern, values of the element pairs without
                        a shared vertex: float (MIXED) or double (FP64) */
#define TDBEM_NEAR 1 /* sub-pattern reached by element pairs sharing a vertex,
                        their values, double */

typedef struct tdbem_mesh tdbem_mesh;
typedef struct tdbem_timegrid tdbem_timegrid;
typedef struct tdbem_asm tdbem_asm;

typedef struct {
    int32_t precision;     /* TDBEM_PREC_FP64 or TDBEM_PREC_MIXED */
    int32_t near_order;    /* Gauss-Legendre points per direction, Sauter-Schwab (default 4) */
    int32_t cheb_degree;   /* Chebyshev degree per panel (32; the only value this build takes) */
    int32_t staging_mb;    /* non-equidistant grids: cap (MiB) on the FP64 staging windows of one
                              batch of block columns; 0 = a quarter of the free memory, <= 24 GiB */
    int32_t reserved[4];
} tdbem_opts;

typedef struct {
    int64_t n_blocks;        /* unique blocks assembled */
    int64_t nnz;             /* stored entries summed over the unique blocks */
    int64_t nnz_near;        /* entries of the near sub-patterns */
    int64_t far_pairs;       /* element pairs without a shared vertex */
    int64_t near_pairs;      /* element pairs sharing a vertex */
    int64_t quad_points;     /* point pairs x blocks evaluated (far + near) */
    double ms_total;         /* device time of the last tdbem_assemble_all */
    double ms_pattern;       /* of which: bounds, windows, table build */
    double ms_far;           /* far-field quadrature */
    double ms_near;          /* near-field quadrature */
    double ms_extract;       /* CSR extraction */
    int64_t kernel_launches; /* kernels launched by the last tdbem_assemble_all */
    int64_t graph_replays;   /* assemblies replayed from the recorded CUDA graph */
    int64_t matvec_variant;  /* matvec launch shape chosen by the autotuner (-1: not tuned yet) */
    int64_t quad_points_far; /* of quad_points: far element pairs (non-equidistant grids; -1 otherwise) */
    int64_t matvec_launches; /* kernels one tdbem_hessenberg_apply launches: 3 in the mixed path on an
                                equidistant grid (padded FP32 copy of x, the blocks outside the Toeplitz
                                class, the Toeplitz class from per-pair lag windows), else 2 */
} tdbem_stats_t;

/* Thread-local description of the last failure; never NULL. */
TDBEM_API const char *tdbem_last_error(void);

/* Register device allocation callbacks (NULL, NULL restores cudaMalloc).
 * alloc(bytes, stream, ctx) returns a device pointer or NULL;
 * free_(ptr, stream, ctx) releases it. Applies to objects created later. */
TDBEM_API tdbem_status tdbem_set_allocator(void *(*alloc)(size_t, void *, void *),
                                 void (*free_)(void *, void *, void *), void *ctx);

/* Surface mesh: M vertices (host, M x 3 doubles, row-major) and E flat
 * triangles (host, E x 3 int32 vertex indices, counter-clockwise seen from
 * the side the unit normal points to). Each vertex carries one hat function
 * phi_j (Sec. 3, "piecewise linear"). Fails with TDBEM_E_MESH on an index out
 * of range, a repeated index, a zero-area triangle or a non-finite vertex. */
TDBEM_API tdbem_status tdbem_mesh_create(const double *verts_xyz, int64_t M, const int32_t *tris,
                               int64_t E, tdbem_mesh **out);

/* Time grid of N points (host): t[0] = 0 < t[1] < ... < t[N-1] = T (Sec. 3).
 * p: Legendre degree of the time basis, 0, 1 or 2 (else TDBEM_E_UNSUPPORTED):
 * the L = N (p + 1) time functions b_{k,m} of Eq. BasisFunctions, numbered
 * k (p + 1) + m (Sec. 3), the Legendre coordinate mapping each function's
 * support onto [-1, 1] (on a non-equidistant grid, the support of the inner
 * function i is [t_{i-1}, t_{i+1}]). With p >= 1 every nonzero block and
 * order pair (k, i, m2, m1) is assembled from its own psi on any grid (the
 * path of non-equidistant grids: no Toeplitz reuse), at most 256 blocks
 * times orders in one block column; the block-Hessenberg preconditioner,
 * tdbem_assemble_block, tdbem_psi_table and tdbem_double_layer take p = 0
 * only (TDBEM_E_UNSUPPORTED). basis_kind:
 * the smooth step that builds the partition of unity, TDBEM_STEP_ERF_ARTANH
 * (0) = the paper's f = erf(2 artanh x)/2 + 1/2, TDBEM_STEP_EXP_INV (1) =
 * F(s) = h(s)/(h(s) + h(1-s)), h(s) = exp(-1/s), s = (x+1)/2 (any other
 * value: TDBEM_E_INVALID_ARG); c: wave speed (> 0, r = |x-y|/c). An equidistant grid (|t_i - i T/(N-1)| <= 1e-12 T) uses the
 * Toeplitz block reuse of Sec. 5.1; any other grid assembles every nonzero
 * block on its own (the uneven steps enter the basis through the local step
 * widths: b_1 uses t_1 - t_0, inner flanks the widths of their own
 * intervals). The assembler needs 5 <= N <= 1000 and, on a non-equidistant
 * grid, at most 256 nonzero blocks in one block column. */
#define TDBEM_STEP_ERF_ARTANH 0
#define TDBEM_STEP_EXP_INV 1
TDBEM_API tdbem_status tdbem_timegrid_create(const double *t, int64_t N, int32_t p, int32_t basis_kind,
                                   double c, tdbem_timegrid **out);

/* Plan an assembler on the current CUDA device: the unique block list, the
 * device copies of the geometry and the triangle colouring. opts may be
 * NULL (defaults: MIXED, near_order 4, degree 32). */
TDBEM_API tdbem_status tdbem_assembler_create(const tdbem_mesh *mesh, const tdbem_timegrid *tg,
                                    const tdbem_opts *opts, void *stream, tdbem_asm **out);

/* Number of unique blocks, and block b's test / trial time index (0-based),
 * temporal orders and structural entry counts (after an assemble call;
 * -1 before). */
TDBEM_API tdbem_status tdbem_num_blocks(const tdbem_asm *a, int64_t *n_unique);
TDBEM_API tdbem_status tdbem_block_info(const tdbem_asm *a, int64_t b, int32_t *k, int32_t *i,
                              int32_t *m2, int32_t *m1, int64_t *nnz_far, int64_t *nnz_near);

/* Assemble every unique block: psi tables, element-pair bounds, vertex-pair
 * windows, far and near quadrature, CSR extraction. The first call runs the
 * steps with the host work between them (table copy, CSR sizes and
 * allocation); later calls on the same assembler record the whole device
 * sequence once into a CUDA graph (on an internal stream) and replay it on
 * `stream`, every step recomputed, the CSR arrays and borrowed pointers
 * unchanged. On a non-equidistant grid every call runs eagerly: the blocks
 * are assembled in batches of block columns whose FP64 staging windows fit a
 * quarter of the free device memory (at most 24 GiB), one far and one near
 * launch per triangle colour and batch. Synchronises the stream at the end
 * and returns TDBEM_E_DEVICE if a kernel flagged an inconsistency or the
 * pattern sizes changed. */
TDBEM_API tdbem_status tdbem_assemble_all(tdbem_asm *a, void *stream);

/* One block (k, i), i <= k+1, of the block-Hessenberg matrix, assembled on
 * its own from its own psi_{k,i} (Sec. 3, Eq. MatrixEntries; Eq.
 * SparsitySmallBlock for its pattern), on any time grid: psi table, element-
 * pair bounds, pattern, far and near quadrature and CSR of this block only,
 * by the kernels of the non-equidistant path. On an equidistant grid the
 * result equals the unique block that Eq. relationAtildeBlock maps (k, i) to.
 * Afterwards tdbem_block_csr, tdbem_block_csr_host and tdbem_block_info with
 * b = TDBEM_LAST_BLOCK return it (borrowed pointers valid until the next
 * tdbem_assemble_block call or tdbem_asm_destroy); the assembler's own
 * blocks are untouched. Synchronises the stream. TDBEM_E_INVALID_ARG for
 * k or i outside 0..N-1, i > k+1, or a block whose support starts beyond
 * diam(Gamma) (a zero block). */
#define TDBEM_LAST_BLOCK (-1)
TDBEM_API tdbem_status tdbem_assemble_block(tdbem_asm *a, int32_t k, int32_t i, void *stream);

/* CSR of unique block b (borrowed device pointers). which = TDBEM_FAR: M+1
 * int64 row offsets, int32 sorted columns and float (MIXED) / double (FP64)
 * values; TDBEM_NEAR: the near sub-pattern with double values. Any output
 * pointer may be NULL. */
TDBEM_API tdbem_status tdbem_block_csr(const tdbem_asm *a, int64_t b, int32_t which,
                             const int64_t **row_ptr_dev, const int32_t **col_dev,
                             const void **val_dev, int64_t *nnz);

/* Copy of block b's CSR into caller-owned host buffers: rp (M+1 int64), col
 * (nnz int32) and val (nnz float for TDBEM_FAR in MIXED mode, else double),
 * sizes as reported by tdbem_block_csr / tdbem_block_info. Any buffer may be
 * NULL. Synchronous (device-wide cudaMemcpy). */
TDBEM_API tdbem_status tdbem_block_csr_host(const tdbem_asm *a, int64_t b, int32_t which, int64_t *rp,
                                  int32_t *col, void *val);

/* y = A x for the whole block-Hessenberg space-time matrix (Sec. 5.1, Eq.
 * Apartitioned), every block taken from the unique blocks of the last
 * assembly through Eq. relationAtildeBlock; blocks cut by the diam criterion
 * are zero. x and y are caller-owned device arrays of L*M doubles (L = N (p
 * + 1) time functions), row k (p + 1) + m at [(k (p + 1) + m) M, ... + M)
 * (time function b_{k,m} of the trial / test side, vertex index within);
 * they must not overlap. FP64 mode: products and sums in FP64. MIXED mode:
 * x rounded to FP32, FP32 products of the FP32 far values, FP32 partial sums
 * accumulated as FP32 pairs, near terms in FP64. Asynchronous on
 * `stream`; uses a scratch buffer owned by the assembler (L*M doubles,
 * allocated by tdbem_assemble_all), so calls on one assembler must be
 * ordered on one stream. TDBEM_E_NOT_ASSEMBLED before an assembly,
 * TDBEM_E_INVALID_ARG for NULL or overlapping x / y, TDBEM_E_CUDA if the
 * launch fails. */
TDBEM_API tdbem_status tdbem_hessenberg_apply(const tdbem_asm *a, const double *x_dev, double *y_dev,
                                              void *stream);

/* Same product as tdbem_hessenberg_apply, without any device allocation
 * (the paper has no counterpart). For callers that cannot allocate device
 * memory where they apply the matrix: a solver loop that has committed all
 * device memory to its own pool, or code under a fixed memory budget where
 * an allocation failing halfway through a run is not acceptable. The
 * transposed x goes to a fixed scratch array of 2^21 doubles (16 MiB) in
 * device global memory; L*M above 2^21 is rejected with TDBEM_E_INVALID_ARG
 * before anything runs. The runtime reserves that array when it loads the
 * library's module on a device, which it does lazily at the first call of
 * this entry point there: a caller that commits all remaining device memory
 * to its own pool makes one call before doing so, and makes its first call
 * before any stream capture. The scratch address is looked up (with the
 * device current) on every call. Nothing has to be zeroed beforehand: every
 * scratch entry that is read is first written. The scratch is shared by all
 * calls on a device, whatever the assembler: calls that overlap in time race
 * on it and must be ordered (one stream).
 * Other arguments, ownership and errors as for tdbem_hessenberg_apply. */
TDBEM_API tdbem_status tdbem_hessenberg_apply_noalloc(const tdbem_asm *a, const double *x_dev, double *y_dev,
                                                      void *stream);

/* Right-hand side of the linear system (Sec. 3): g_k(l) = int_0^T int_Gamma
 * g(x,t) phi_l(x) bdot_k(t) dGamma dt for every time basis function k and
 * vertex l, for p >= 1 with bdot_{k,m} of every order m, written to the
 * caller-owned device array g_dev of L*M doubles (row k (p + 1) + m at
 * [(k (p + 1) + m) M, ... + M)). FP64; 7-point rule on every triangle, composite
 * Gauss-Legendre in time split at every grid point. Neumann data g by kind:
 *   TDBEM_RHS_PLANE_WAVE: sound-hard scattering of u_inc = exp(-(t - x.d -
 *     c0)^2 / (2 w^2)); params = {dx, dy, dz, c0, w} (nparams 5, d is
 *     normalised), g = -du_inc/dn;
 *   TDBEM_RHS_SPHERE_N0: g = Y_0^0 sin(3t) t^2 e^{-t} (Sec. 6.1), nparams 0;
 *   TDBEM_RHS_SPHERE_N1: g = Y_1^0(x) sin(2 pi t) t^3 e^{-2t} (Sec. 6.1).
 * Needs no assembly. Asynchronous on `stream`. TDBEM_E_INVALID_ARG for a NULL
 * pointer, an unknown kind or bad parameters. */
#define TDBEM_RHS_PLANE_WAVE 0
#define TDBEM_RHS_SPHERE_N0 1
#define TDBEM_RHS_SPHERE_N1 2
TDBEM_API tdbem_status tdbem_rhs_assemble(const tdbem_asm *a, int32_t kind, const double *params,
                                          int32_t nparams, double *g_dev, void *stream);

/* The assembler's own Chebyshev table of psi and psi~ (Sec. 3.1) for unique
 * block b of an equidistant grid, evaluated at n distances r (device array)
 * into out (device, n x 2: psi, psi~), so that the table can be compared
 * with a direct 1-D quadrature of Eq. psis. which: 0 = the FP64 set (4
 * sub-panels of degree 32 per time step, used by the near field and the
 * FP64 path), 1 = the FP32 set (one panel of degree 32 per time step with
 * the FP32 residuals of the leading coefficients, used by the mixed far
 * field; summed here in FP64). Zero outside the support. Valid after an
 * assembly; asynchronous on `stream`. TDBEM_E_UNSUPPORTED on a graded grid
 * (its tables are per block and panel), TDBEM_E_NOT_ASSEMBLED before an
 * assembly, TDBEM_E_INVALID_ARG for a bad block, `which` or pointer. */
TDBEM_API tdbem_status tdbem_psi_table(const tdbem_asm *a, int64_t b, int32_t which, const double *r_dev,
                                       int64_t n, double *out_dev, void *stream);

/* Retarded double layer potential (Sec. 2, Eq. RetardedPotential), the
 * evaluation of a solution off the surface:
 *   u(x, t) = -1/(4 pi) int_Gamma n_y.(x - y)/r [phi(y, t - r/c)/r^2
 *             + d_t phi(y, t - r/c)/(c r)] dGamma_y,   r = |x - y|,
 * for the density phi(y, s) = sum_{k, j} alpha[k M + j] b_k(s) phi_j(y)
 * (p = 0 time basis, hat functions in space). Every triangle is integrated
 * by the collapsed Gauss product rule with n points per direction (n^2 per
 * triangle); FP64. alpha: device, N*M doubles (row k at [k*M, k*M + M));
 * X: device, P x 3 doubles (points off the surface); times: device, nt
 * doubles; u: device, P x nt doubles (u[p*nt + i] = u(X_p, times_i)), all
 * caller-owned. Needs no assembly. The quadrature points and density
 * coefficients (E n^2 (8 + N) doubles) are allocated through the registered
 * allocator for the call; synchronises the stream. TDBEM_E_INVALID_ARG for
 * NULL arrays, P < 0, nt < 1 or n outside 1..32. */
TDBEM_API tdbem_status tdbem_double_layer(const tdbem_asm *a, const double *alpha_dev, const double *x_dev,
                                          int64_t P, const double *times_dev, int32_t nt, int32_t n, double *u_dev,
                                          void *stream);

/* Solve A alpha = g (the block-Hessenberg system of Eq. Apartitioned) by
 * restarted GMRES(restart) (Sec. 4) with tdbem_hessenberg_apply as the
 * product: zero initial guess, stop when ||g - A alpha|| <= tol ||g|| or after
 * max_iter iterations. g and alpha are caller-owned device arrays of L*M
 * doubles that must not overlap; the Krylov basis ((restart+1) N M doubles)
 * is allocated through the registered allocator for the call and freed
 * before it returns. On return *iters holds the iterations done and *rel_res
 * the relative residual of alpha (either may be NULL). Synchronises the
 * stream. TDBEM_E_NOT_ASSEMBLED before an assembly; TDBEM_E_INVALID_ARG for
 * restart outside 1..62, tol <= 0, max_iter < 1, NULL or overlapping
 * arrays; TDBEM_E_OOM if the basis cannot be allocated. */
TDBEM_API tdbem_status tdbem_solve_gmres(const tdbem_asm *a, const double *g_dev, double *alpha_dev,
                                         int32_t restart, double tol, int32_t max_iter, int32_t *iters,
                                         double *rel_res, void *stream);

/* Solve A alpha = g by DGMRES(restart, l) (Sec. 4.1): restarted GMRES
 * right-preconditioned by the deflation preconditioner
 *   M^-1 = I + U (|lambda_max| T^-1 - I) U^T,  T = U^T A U,
 * fixed within a cycle. After every cycle that does not converge, the
 * invariant subspace of the cycle's square Hessenberg matrix H_m (of A M^-1)
 * for its eigenvalues of modulus at most the l-th smallest (a complex pair
 * counts twice) is mapped through the Krylov basis, orthonormalised against U
 * (two Gram-Schmidt passes; a vector with less than 1e-10 of its norm left is
 * dropped) and appended, until U has r columns; the largest modulus among the
 * eigenvalues of H_m is the estimate of |lambda_max|. l = 0 or r = 0 is
 * GMRES(restart). Products, Gram-Schmidt (classical, two passes) and
 * M^-1 run on the device; the Schur decomposition of H_m, T^-1 and the
 * small least-squares problem on the host.
 * g and alpha: caller-owned device arrays of L*M doubles, not overlapping;
 * zero initial guess; stop when the residual estimate reaches tol ||g|| or a
 * restart finds the true residual there, or after max_iter iterations.
 * *iters: iterations done; *rel_res: the true relative residual of the
 * result; *deflated: columns of U at the end (each may be NULL). Work space:
 * (restart + 2 + 2 r) N M doubles. Synchronizes the stream.
 * TDBEM_E_NOT_ASSEMBLED before an assembly; TDBEM_E_INVALID_ARG for restart
 * outside 1..62, l < 0, r outside 0..62, tol <= 0, max_iter < 1, NULL or
 * overlapping arrays; TDBEM_E_NUMERIC if the Schur iteration of H_m does not
 * converge; TDBEM_E_OOM if the work space cannot be allocated. */
TDBEM_API tdbem_status tdbem_solve_dgmres(const tdbem_asm *a, const double *g_dev, double *alpha_dev,
                                          int32_t restart, int32_t l, int32_t r, double tol, int32_t max_iter,
                                          int32_t *iters, double *rel_res, int32_t *deflated, void *stream);

/* Deflation subspace of one DGMRES cycle (host only, no device work): for
 * the m x m upper Hessenberg matrix H (row-major, row stride ldh; entries
 * below the subdiagonal are ignored), an orthonormal real basis B of its
 * invariant subspace for the eigenvalues of modulus at most the l-th
 * smallest (times 1 + 1e-12), written column k at B[i * m + k], i < m
 * (B: caller-owned host array of m * m doubles); *sdim: its dimension;
 * *lam_max: the largest modulus among the eigenvalues. l = 0 returns
 * only *lam_max. TDBEM_E_INVALID_ARG for m outside 1..62, ldh < m or NULL
 * arrays; TDBEM_E_NUMERIC if the Schur iteration does not converge. */
TDBEM_API tdbem_status tdbem_deflation_basis(const double *H, int32_t m, int32_t ldh, int32_t l, double *B,
                                             int32_t *sdim, double *lam_max);

/* Solve A alpha = g by flexible GMRES FGMRES(restart, levels(inner...)) with
 * the recursive algebraic block-Hessenberg preconditioner (Sec. 4.2,
 * Algorithm 1; the notation of the solver tables of Sec. 6).
 * Preconditioner: on a diagonal range of block rows/columns [lo, hi) split at
 * h = lo + ceil((hi - lo) / 2), M equals A without the block (h - 1, h)
 * above the diagonal (0-based), and M^-1 r = (M11^-1 r1, M22^-1 (r2 -
 * M21 M11^-1 r1)). The two diagonal systems of a level-l splitting are
 * solved approximately by one FGMRES cycle of inner_iters[l - 1] steps from
 * zero with the same relative tolerance, preconditioned by the level-(l + 1)
 * splitting of that half while l < levels and the half spans two blocks or
 * more; the last level is unpreconditioned. levels = 0 runs the same
 * iteration without a preconditioner (GMRES(restart)).
 * g and alpha: caller-owned device arrays of L*M doubles, not overlapping;
 * zero initial guess; stop when the residual estimate reaches tol ||g||, or
 * when a restart finds the true residual there, or after max_iter outer
 * iterations. *iters: outer iterations done; *rel_res: the true relative
 * residual ||g - A alpha|| / ||g|| of the result (either may be NULL).
 * inner_iters: host array of `levels` counts, each 1..62 (NULL when levels
 * is 0). The Krylov bases of all levels (about (2 restart + 3) N M doubles
 * plus (2 inner_l + 3) N M / 2^l at level l) are allocated through the
 * registered allocator for the call. The preconditioner application is
 * recorded once per call as a CUDA graph on an internal stream and replayed
 * on `stream` at every outer step; the host reads one small status record
 * per outer step. Synchronises the stream. TDBEM_E_NOT_ASSEMBLED before an
 * assembly; TDBEM_E_INVALID_ARG for restart outside 1..62, tol outside
 * (0, 1), max_iter < 1, levels outside 0..24, an inner count outside 1..62,
 * NULL or overlapping arrays; TDBEM_E_OOM if the bases cannot be allocated. */
TDBEM_API tdbem_status tdbem_solve_fgmres(const tdbem_asm *a, const double *g_dev, double *alpha_dev,
                                          int32_t restart, double tol, int32_t max_iter, int32_t levels,
                                          const int32_t *inner_iters, int32_t *iters, double *rel_res,
                                          void *stream);

/* z = M^-1 r: one application of the recursive preconditioner of
 * tdbem_solve_fgmres (levels >= 1 levels, inner_iters as there, tol the
 * relative tolerance of the inner solves). r and z: caller-owned device
 * arrays of N*M doubles, not overlapping. Workspace as for
 * tdbem_solve_fgmres with restart 1, allocated for the call. Launched
 * directly (no graph); synchronises the stream. Errors as for
 * tdbem_solve_fgmres, and TDBEM_E_INVALID_ARG for levels < 1. */
TDBEM_API tdbem_status tdbem_precond_apply(const tdbem_asm *a, int32_t levels, const int32_t *inner_iters,
                                           double tol, const double *r_dev, double *z_dev, void *stream);

/* Measured FMA throughput of the current device in TFLOP/s (an FMA counts
 * two flops): packed FP32 pairs (the far kernel's arithmetic) and FP64. Not
 * part of the paper's method: the denominators of the roofline fractions,
 * taken at the clock the device runs at when called. Runs two short kernels
 * (tens of ms), allocates nothing, synchronises the stream. Either output
 * may be NULL. */
TDBEM_API tdbem_status tdbem_measure_fma_peaks(double *fp32_tflops, double *fp64_tflops, void *stream);

/* Assembly counters and the per-phase device times of the last assembly. */
TDBEM_API tdbem_status tdbem_stats(const tdbem_asm *a, tdbem_stats_t *out);

TDBEM_API void tdbem_mesh_destroy(tdbem_mesh *m);
TDBEM_API void tdbem_timegrid_destroy(tdbem_timegrid *t);
TDBEM_API void tdbem_asm_destroy(tdbem_asm *a);

#ifdef __cplusplus
}
#endif
#endif /* TDBEM_H */
