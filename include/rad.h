/*
 * librad — GB300 (sm_103a) hierarchical block low-rank cavity radiation.
 *
 * C ABI of the hot path of Baburin, Ballani, Peterson and Knezevic,
 * "Hierarchical Block Low-rank Approximation of Cavity Radiation":
 * view-factor entries (Eq. 10), cluster tree (§4.1, Algorithm 1), block tree
 * with the admissibility condition (§4.2, Algorithm 2, Eq. 28), cross
 * approximation of admissible blocks (§4.3, Eqs. 30-31), the block low-rank
 * matrix-vector product (§5.2) and a GMRES solve of the reflection system
 * (Eq. 11) that returns the facet flux (Eq. 12).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Every call returns an int status: RAD_OK (0) or one of the RAD_E* codes.
 *   rad_last_error() returns a message for the calling thread's last failure.
 *   No C++ exception crosses this interface.
 * - Array arguments may be HOST or DEVICE pointers (the library asks the CUDA
 *   runtime which one it was given).  Host arrays are copied to the device
 *   inside the call; device arrays must be on the current device.  The caller
 *   owns every array it passes; the library keeps no reference after return.
 * - All arrays are indexed in the caller's facet order; the tree permutation
 *   is internal.
 * - `stream` is a cudaStream_t (NULL = legacy default stream).  Work is
 *   ordered on it.  Calls that must size buffers from device results (tree
 *   build, compression, solve) synchronise that stream before returning;
 *   rad_hmatvec does not.
 * - The library owns the rad_htree handle and every device buffer inside it
 *   (rad_htree_free releases them).  Device memory comes from the handle's
 *   allocator (rad_tree_params.allocator: the caller's callbacks, or the
 *   library's own stream-ordered pool).  A handle is used on the device that
 *   was current when it was built.  Calls on one handle must not overlap.
 * - Floating-point facet data is double precision.  Facets must be
 *   non-degenerate (positive area) and finite, else RAD_EINVAL.
 */
#ifndef RAD_H
#define RAD_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define RAD_OK        0
#define RAD_EINVAL    1   /* bad argument or state                         */
#define RAD_ENOMEM    2   /* a device allocation failed                    */
#define RAD_ENOTCONV  3   /* GMRES did not reach the tolerance             */
#define RAD_ECUDA     4   /* a CUDA runtime call failed                    */
#define RAD_ELIMIT    5   /* a size limit of this library was exceeded     */

/* storage / vector element types */
#define RAD_F64   0
#define RAD_F32   1
#define RAD_BF16  2

/* cross-approximation pivoting (§1: the paper uses full pivoting) */
#define RAD_ACA_PARTIAL 0
#define RAD_ACA_FULL    1

typedef struct rad_htree rad_htree;

/* Device-memory callbacks (no counterpart in the paper; an interface of this
 * library).  A handle takes every device buffer it owns, and every per-call
 * workspace of the calls made on it, from its allocator, so that a caller
 * with its own memory manager (e.g. PyTorch's caching allocator) owns and
 * accounts for all of the library's device memory:
 *   alloc(ctx, bytes, stream) returns device memory of at least `bytes`
 *     bytes, 256-byte aligned, usable in the order of `stream` (a
 *     cudaStream_t; NULL = legacy default stream), or NULL on failure (the
 *     call then returns RAD_ENOMEM after returning what it already took);
 *   free(ctx, ptr, bytes, stream) takes back a pointer alloc returned, with
 *     the same byte count; work queued on `stream` before the call may still
 *     read it, so a stream-ordered allocator reuses it only after that work.
 *     Buffers owned by a handle are freed after a device synchronisation
 *     (rad_htree_free), per-call workspaces in the order of the call's stream.
 *   ctx is passed through unchanged.
 * The callbacks are called from the thread that makes the library call (for a
 * server: its worker threads) and must stay valid until the handle is freed.
 * Without an allocator (NULL), the library allocates stream-ordered
 * (cudaMallocFromPoolAsync on the call's stream) from a memory pool of its own
 * per device that keeps freed memory cached; it does not change the device's
 * default memory pool. */
typedef struct {
    void* (*alloc)(void* ctx, uint64_t bytes, void* stream);
    void  (*free)(void* ctx, void* ptr, uint64_t bytes, void* stream);
    void*  ctx;
} rad_allocator;

/* §4.1-4.2.  leaf_size = n_min of Algorithm 1 (a cluster with at most
 * leaf_size facets is a leaf, >= 1); eta_adm = c of Eq. (28), > 0.
 * allocator: device memory of the new handle (see rad_allocator; NULL = the
 * library's own pool); the struct is copied, the callbacks are not. */
typedef struct {
    int32_t leaf_size;
    int32_t reserved;
    double  eta_adm;
    const rad_allocator* allocator;
} rad_tree_params;

/* §4.3.  tol = eps_rel of Eq. (31) (>= 0); max_rank caps the rank of every
 * admissible block (<= 128; a block that would need more, or more than its
 * storage break-even rank m n / (m + n), is stored dense instead);
 * pivoting = RAD_ACA_PARTIAL or RAD_ACA_FULL; factor_dtype (RAD_F64, RAD_F32
 * or RAD_BF16) is the storage type of the U, V factors and near_dtype
 * (RAD_F64 or RAD_F32) that of the dense blocks.  near_dtype = RAD_F64
 * requires factor_dtype = RAD_F64 (the FP64 path); the other combinations
 * compute in FP32 with FP32 accumulation.
 * accurate_dtype = RAD_F32 with factor_dtype = RAD_BF16 also keeps the
 * factors in FP32: the "accurate operator" that mixed-precision iterative
 * refinement (rad_solve_params.refine) uses for its residuals; -1 keeps no
 * second copy.
 * scratch_mib bounds the device scratch of partial-pivot ACA (max_rank
 * columns of U and V per admissible block, before the ranks are known):
 * 0 = 30% of the free device memory, at most 48 GiB, at least 1 GiB; > 0 =
 * that many MiB.  Blocks beyond the bound are compressed in further chunks,
 * each compacted to its ranks before the next starts; the result does not
 * depend on the chunking.
 * recompress_tol (§4.3 postprocessing into standard form, ranks truncated
 * by the singular-value decay as in §5.1): 0 = keep every ACA cross as it
 * is; in (0, 1) = bring each cross of rank 2..64 to U = Q_U W_r diag(s_r),
 * V = Q_V Z_r from the SVD of R_U R_V^T (U = Q_U R_U, V = Q_V R_V), with the
 * smallest r >= 1 such that the dropped singular values have
 * sqrt(sum s_i^2) <= recompress_tol * ||U V^T||_F.  The dropped part adds at
 * most that relative error to each block (on top of tol). */
typedef struct {
    double  tol;
    int32_t max_rank;
    int32_t pivoting;
    int32_t factor_dtype;
    int32_t near_dtype;
    int32_t accurate_dtype;
    int32_t scratch_mib;
    double  recompress_tol;
} rad_aca_params;

/* GMRES on C y = b, C = I - diag(1 - eps) F (Eq. 11).  Stops when every
 * column's relative residual ||b - C y|| / ||b|| <= tol; restart = Krylov
 * dimension per cycle (1..64); max_iter = total Arnoldi steps per column.
 * refine = 1 (needs a handle compressed with accurate_dtype = RAD_F32):
 * mixed-precision iterative refinement - the residual r = b - C y is
 * computed with the accurate operator (FP32 factors) accumulated in FP64,
 * the correction solves C d = r by GMRES on the fast operator (BF16 factors)
 * to inner_tol, y += d, until the accurate relative residual <= tol.
 * precond: see rad_hlu_factor; factors built for other emissivities remain a
 * valid (weaker) preconditioner, the stopping test is always on C itself. */
typedef struct rad_hlu rad_hlu;

typedef struct {
    double  tol;
    int32_t restart;
    int32_t max_iter;
    int32_t refine;
    int32_t max_refine;          /* outer refinement steps (refine = 1)       */
    double  inner_tol;           /* relative tolerance of each correction     */
    const rad_hlu* precond;      /* optional right preconditioner: the block LU
                                    factors of C (rad_hlu_factor on the same
                                    handle); GMRES then iterates on C (LU)^-1
                                    and returns x = (LU)^-1 u.  NULL = none.  */
} rad_solve_params;

typedef struct {
    int32_t status;              /* RAD_OK or RAD_ENOTCONV                     */
    int32_t iters;               /* Arnoldi steps taken (max over columns)     */
    int32_t restarts;            /* restart cycles                             */
    int32_t matvecs;             /* block matrix products applied             */
    double  max_rel_residual;    /* max over columns of ||b - C y|| / ||b||,
                                    recomputed with the stored operator (the
                                    accurate one when refining)               */
    int32_t refinements;         /* outer refinement steps taken              */
    int32_t reserved;
} rad_solve_info;

typedef struct {
    int64_t n;                   /* facets                                     */
    int32_t leaf_size;
    int32_t n_nodes;             /* clusters in the tree                      */
    int32_t n_leaf_clusters;
    int32_t depth;               /* levels (root = level 0)                   */
    int64_t n_blocks;            /* leaf blocks of the block tree             */
    int64_t n_admissible;        /* admissible leaf blocks                    */
    int32_t compressed;          /* 1 after rad_compress_aca                  */
    int32_t factor_dtype;
    int32_t near_dtype;
    int32_t max_rank_used;       /* largest ACA rank stored                   */
    int64_t n_dense_fallback;    /* admissible blocks stored dense            */
    int64_t near_entries;        /* sum m n over dense blocks                 */
    int64_t far_entries;         /* sum k (m + n) over low-rank blocks         */
    int64_t sum_rank;            /* sum k over low-rank blocks                 */
    int64_t aca_entries;         /* entries evaluated by ACA                   */
    int64_t bytes_near;
    int64_t bytes_far;
    int64_t far_u_entries;       /* sum k m over low-rank blocks (U factors)   */
    int64_t far_v_entries;       /* sum k n over low-rank blocks (V factors)   */
    int64_t n_tiles;             /* row tiles of the product (<= 64 rows)      */
    int64_t bytes_accurate;      /* FP32 factor copy kept for refinement (0 if none) */
    int32_t tuned;               /* 1 after rad_htree_autotune                  */
    int32_t stream_rows;         /* rows per far-field item (1-4 columns)       */
    int32_t grid_a1, grid_b1;    /* grids of the 1-column phases (0: per item)  */
    int32_t grid_a2, grid_b2;    /* grids of the 2-4 column launches            */
    int32_t product_path;        /* >= 5 FP32 columns: 0 CUDA cores, 1 tensor cores */
    int32_t closed;              /* 1 after rad_htree_close_cavity               */
    int32_t one_column_path;     /* 1 column: 1 one fused launch, 0 two launches */
    int32_t reserved;
} rad_htree_stats;

/* -------------------------------------------------------------------------
 * rad_build_htree — A1-A3: facet geometry (§3.1), cluster tree (Algorithm 1)
 * and block tree (Algorithm 2 with Eq. 28), all on the GPU.
 *   n      facets (>= 1, < 2^31)
 *   verts  n x 3 x 3 doubles, row-major (facet, vertex, xyz), triangles wound
 *          so that (v1 - v0) x (v2 - v0) points into the cavity
 *   out    receives the new handle (NULL on failure)
 * The tree, permutation and block partition are deterministic and identical
 * bit for bit to Algorithms 1-2 evaluated in FP64 with the split rule:
 * longest bounding-box axis of the centroids (ties: lowest axis), left child
 * = the floor(n/2) facets first in (coordinate, facet index) order.
 * ------------------------------------------------------------------------- */
int rad_build_htree(int64_t n, const double* verts, const rad_tree_params* p,
                    void* stream, rad_htree** out);

/* Same as rad_build_htree from facet data (§3.1): centroids n x 3, unit
 * normals n x 3 (pointing into the cavity), areas n (all row-major). */
int rad_build_htree_facets(int64_t n, const double* centroid, const double* normal,
                           const double* area, const rad_tree_params* p,
                           void* stream, rad_htree** out);

/* Batch of independent cavities in one handle (no counterpart in the
 * paper, which treats one cavity): cavity c owns the next counts[c]
 * triangles of verts (the cavities' triangles concatenated, 9 doubles each,
 * host or device).  The cluster tree is a forest with one root per cavity
 * (Algorithm 1 applied to each cavity) and the block tree (Algorithm 2)
 * never pairs clusters of different cavities, whose mutual view factors
 * are not part of any cavity's problem.  Every other call works on the
 * batch as on one cavity: one ACA launch compresses all cavities' blocks,
 * one product applies all of them, and the solvers (rad_solve_reflection,
 * rad_solve_flux) keep Krylov subspaces, inner products and convergence
 * tests per cavity and per right-hand side, so that each cavity's result
 * is the one it would get alone up to rounding.  Vectors are the
 * concatenation of the cavities' vectors (length sum(counts)).
 *   n_cavities >= 1, counts[c] >= 1 (host array); RAD_EINVAL otherwise. */
int rad_build_htree_batch(int32_t n_cavities, const int64_t* counts, const double* verts,
                          const rad_tree_params* p, void* stream, rad_htree** out);

/* Test hook: wraps a caller's dense n x n view-factor matrix F (row-major,
 * F[i*n + j] = F_ij, §3.2) as a single dense block stored in FP64, already
 * "compressed".  Lets closed-form pins (e.g. Eq. 5) drive rad_solve_flux. */
int rad_htree_from_dense(int64_t n, const double* F, void* stream, rad_htree** out);

/* -------------------------------------------------------------------------
 * rad_compress_aca — A4-A5: dense blocks get their entries (Eq. 10, 1-point
 * centroid rule); admissible blocks are approximated by ACA (Eq. 30) until
 * ||X - U V^T||_F <= tol ||X||_F (Eq. 31; estimated for partial pivoting,
 * exact for full pivoting).  May be called again to recompress with other
 * parameters.  Full pivoting holds every admissible block densely while it
 * runs: RAD_ELIMIT if that exceeds 8 GiB.
 * ------------------------------------------------------------------------- */
int rad_compress_aca(rad_htree* h, const rad_aca_params* p, void* stream);

/* -------------------------------------------------------------------------
 * rad_hmatvec — A6: Y = F X (§5.2), F the stored block low-rank matrix.
 *   dtype  RAD_F64 or RAD_F32: element type of x and y
 *   x      column-major n x nrhs, column c at x + c*ldx (ldx >= n)
 *   y      column-major n x nrhs, column c at y + c*ldy (ldy >= n)
 *   nrhs   1 .. 4096
 * Requires a compressed handle.  Device arrays: asynchronous on `stream`.
 * Graph replay (no counterpart in the paper): with device arrays, the
 * second call with the same x, y, leading dimensions, nrhs, dtype and stream
 * captures the gather, the product and the scatter into a CUDA graph kept by
 * the handle, and later identical calls replay it (one graph launch; x and
 * y are read and written in place, so their contents may change between
 * calls).  Not while profiling, not when `stream` is itself being captured
 * (the kernels are then recorded into the caller's graph), and not for
 * overlapping calls on other streams.  Recompression or autotuning drops the
 * graph.
 * ------------------------------------------------------------------------- */
int rad_hmatvec(const rad_htree* h, int32_t dtype, const void* x, int64_t ldx,
                void* y, int64_t ldy, int64_t nrhs, void* stream);

/* Autotuner for the streaming products (1-4 columns; no counterpart in the
 * paper): times, on this handle's compressed operator, every combination of
 * far-field item rows (64, 128, 256) and grid policy (one CTA per work item,
 * or a persistent grid of 2, 4 or 8 CTAs per SM) for each launch, and keeps
 * the fastest (reported in rad_htree_stats).  The grid policy does not
 * change results (each work item is computed by one CTA in a fixed order);
 * the item rows change the order of the sums over a column group (results
 * agree to rounding).  Synchronous; takes a fraction of a second.
 * Recompression resets the choice. */
int rad_htree_autotune(rad_htree* h, void* stream);

/* Kernel family of the product with 5 or more FP32 columns (no counterpart
 * in the paper): 0 = CUDA-core register tiles (FP32 FFMA; the default for
 * FP64 operators), 1 = tensor cores (the default after rad_compress_aca for
 * FP32 and BF16 operators; tcgen05 kind::f16, computed transposed: the right-hand
 * sides are the MMA's M, a row tile's rows its N; every FP32 operand split
 * into three BF16 pieces carrying its 24 bits, six partial products per
 * k-step, the leading and the correction terms in two accumulators
 * restarted every 128 panel columns and summed in FP32 registers, so
 * results agree with path 0 to FP32 rounding).  Selecting path 1 builds the
 * split panel images once (about 1.5 times the FP32 operator's bytes, rows
 * padded to 8 and runs of columns to 8; synchronous); path 0 releases them.
 * rad_htree_autotune picks the faster path for the handle's operator;
 * recompression resets it to the default; a loaded checkpoint keeps the path and
 * rebuilds the images at its first product of 5 or more columns.  After
 * rad_compress_aca the images are built at the first rad_hmatvec,
 * rad_solve_flux or rad_solve_reflection call with 5 or more columns (one
 * synchronisation), never for one-column use; a call made while its
 * stream is being captured into a graph does not build them and runs on
 * the CUDA-core tiles.
 * RAD_EINVAL for another value, or for path 1 on an FP64 operator. */
int rad_htree_set_product_path(rad_htree* h, int32_t path);

/* Kernel family of the one-column product (§5.2, y = F x; no counterpart in
 * the paper): 1 = one fused launch (the default where the operator allows
 * it: FP32 dense panels, FP32 or BF16 factors, panels of at most 1024 rows)
 * in which every CTA streams panel chunks through a ring of shared-memory
 * stages filled by 1-D bulk copies, the products T = V^T x and the dense
 * panels first and the U panels after all of T is written; 0 = two launches
 * (phase A: T and the dense panels, phase B: the U panels).  Both compute
 * every output row in one CTA in a fixed order; they sum a row's terms in
 * different orders, so results agree to rounding.  rad_htree_autotune picks
 * the faster; compression resets it to 1.  RAD_EINVAL for another value, or
 * for path 1 on an operator that does not allow it. */
int rad_htree_set_one_column_path(rad_htree* h, int32_t path);

/* Closed-cavity treatment of the view factors (§6, Eqs. rowsum,
 * clamped_rowsum and F_closed, with the textbook F): s_i = sum_j F_ij of
 * the stored operator (the FP32 accurate copy when the factors are BF16),
 * c_i = s_i clamped to [0, 1], and every row with c_i != 0 divided by c_i,
 * in the stored dense blocks and U factors.  row_sums (may be NULL)
 * receives s in facet order (n doubles, host or device).  Requires a
 * compressed handle; call again after every rad_compress_aca (compression
 * rebuilds the unscaled operator).  Calling it twice scales twice. */
int rad_htree_close_cavity(rad_htree* h, double* row_sums, void* stream);

/* -------------------------------------------------------------------------
 * rad_solve_flux — A7-A8: for each of the m temperature fields T(:, c)
 * (Kelvin), solves C y_c = eps o eta_c and C z = eps (Eq. 11,
 * eta = T^4, Eq. 8) by batched GMRES in FP64 on the stored operator, then
 * writes the facet flux of Eq. (12) in the form
 *     q(:, c) = sigma eps o ( F y_c - eta_c o F z ),
 * the net flux into each facet (W m^-2).
 *   eps    n emissivities in (0, 1]
 *   T      column-major n x m, column c at T + c*ldT
 *   q      column-major n x m, column c at q + c*ldq (output)
 *   m      1 .. 1024 fields
 *   sigma  Stefan-Boltzmann constant (the caller's value; 5.670374419e-8)
 *   info   optional (may be NULL)
 * Returns RAD_ENOTCONV (q still written) if a column misses the tolerance.
 * RAD_EINVAL, before any solver work, if an emissivity is not finite or not
 * in (0, 1], or a temperature is not finite or negative.
 * ------------------------------------------------------------------------- */
int rad_solve_flux(const rad_htree* h, const double* eps, const double* T, int64_t ldT,
                   int64_t m, double sigma, const rad_solve_params* p,
                   double* q, int64_t ldq, rad_solve_info* info, void* stream);

/* -------------------------------------------------------------------------
 * rad_hmatvec_noalloc — the product of rad_hmatvec (same arguments, same
 * result; with 5 or more columns on the tensor-core path, once the handle's
 * tensor-core images exist — built by its first rad_hmatvec or solve with 5
 * or more columns, or by rad_htree_set_product_path — before that it runs
 * the CUDA-core tiles, which agree to FP32 rounding, since building the
 * images would allocate) for callers that cannot let the library allocate
 * device memory,
 * e.g. a serving engine that has already reserved the GPU's memory for its
 * own pool, or a latency-critical loop that must stay out of the allocator.
 * The paper has no counterpart; this is an interface convenience.
 * Its scratch is one fixed 32 MiB array in device memory per GPU (held from
 * the library's load until the process exits) instead of allocations:
 *   - x and y must be device arrays (host arrays are rejected: staging them
 *     would allocate);
 *   - it needs round256(s * n * p) + round256(s * n * nrhs)
 *     + round256(s * (max(sum_rank, 1) * p + (nrhs == 1 ? n + 16 : 0))) bytes,
 *     s = 8 for an FP64 operator and 4 otherwise, p = 1 for one column and
 *     nrhs rounded up to a multiple of 4 otherwise (sum_rank from
 *     rad_htree_get_stats), plus round256(6 (n + max(sum_rank, 1)) q) + 512
 *     bytes for 5 or more columns on the tensor-core product path
 *     (q = min(96, nrhs rounded up to a multiple of 8)); larger calls return
 *     RAD_ELIMIT;
 *   - the first call on each device looks up the array's device address
 *     (make that first call before any stream capture);
 *   - all calls on a device share the array: calls that overlap on the GPU
 *     race and must be serialised by the caller;
 *   - it returns RAD_EINVAL while rad_profile_enable is on.
 * Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int rad_hmatvec_noalloc(const rad_htree* h, int32_t dtype, const void* x, int64_t ldx,
                        void* y, int64_t ldy, int64_t nrhs, void* stream);

/* -------------------------------------------------------------------------
 * Hierarchical block LU of the reflection matrix (§5.1) and the forward and
 * backward substitution with its factors (§5.2).
 *
 * rad_hlu_factor: C = I - diag(1 - eps) F~, F~ the handle's stored operator
 * (dense blocks and U V^T of the low-rank blocks; the FP32 accurate copy
 * when the factors are BF16), is factorised C ~ L U in the block structure of
 * the handle's block tree: L unit lower and U upper triangular, each leaf
 * block dense or low rank.  The recursion runs over the diagonal cluster
 * pairs: a leaf pair gets a dense LU without pivoting; a pair with children
 * is factorised as a 2 x 2 block matrix (upper-left block recursively, the
 * off-diagonal blocks by triangular solves, the Schur complement of the
 * lower-right block recursively).  Every block the recursion produces is
 * brought back into the block format, the ranks of its admissible leaves
 * truncated at the relative accuracy tol by the singular-value decay; a leaf
 * whose truncation would need more than min(64, m n / (m + n)) terms stays
 * dense.  tol = 0 keeps every block exact (the unique LU of C without
 * pivoting, every leaf dense).
 *   eps     n emissivities in (0, 1] (facet order, host or device)
 *   out     receives the factors; they refer to h, which must outlive them
 * Works on one dense n x n matrix while factorising (n <= 46340; leaf
 * clusters of at most 128 facets, else RAD_ELIMIT).  Arithmetic is FP64 for
 * an FP64 operator (near_dtype RAD_F64), FP32 otherwise.  RAD_EINVAL for an
 * emissivity outside (0, 1] or a zero pivot.  Synchronous.
 *
 * rad_hlu_solve: X = U^-1 L^-1 B for nrhs right-hand sides (column-major,
 * facet order, host or device), by forward and backward substitution through
 * the block structure (a triangular solve per diagonal leaf, D x or U (V^T x)
 * per off-diagonal leaf).  Synchronous.
 * rad_hlu_export: the factors as one dense n x n row-major host array in
 * TREE order (rad_htree_export_tree gives the permutation), L strictly below
 * the diagonal (unit diagonal implied) and U on and above it.
 * ------------------------------------------------------------------------- */
typedef struct {
    double  tol;                 /* eps_rel of the truncation, in [0, 1)      */
    int32_t reserved0, reserved1;
} rad_hlu_params;

typedef struct {
    int64_t n;
    int64_t dense_entries;       /* entries of the dense leaves               */
    int64_t lowrank_entries;     /* sum k (m + n) over the low-rank leaves     */
    int32_t max_rank;
    int32_t n_lowrank;           /* low-rank leaves                            */
    int32_t n_dense_fallback;    /* admissible leaves kept dense               */
    int32_t precision;           /* RAD_F64 or RAD_F32                         */
    double  tol;
    double  factor_ms;           /* host wall time of rad_hlu_factor           */
    int32_t solve_launches;      /* steps of one substitution (leaf solves and
                                    region products)                           */
    int32_t reserved;
} rad_hlu_stats;

int rad_hlu_factor(const rad_htree* h, const double* eps, const rad_hlu_params* p, void* stream, rad_hlu** out);
int rad_hlu_solve(const rad_hlu* lu, const double* B, int64_t ldB, int64_t nrhs, double* X, int64_t ldX,
                  void* stream);
int rad_hlu_get_stats(const rad_hlu* lu, rad_hlu_stats* st);
int rad_hlu_export(const rad_hlu* lu, double* LU);
int rad_hlu_free(rad_hlu* lu);

/* -------------------------------------------------------------------------
 * rad_solve_reflection — A7 alone: solves C Y = B (Eq. 11, C = I -
 * diag(1 - eps) F) for nrhs arbitrary right-hand sides by the same batched
 * GMRES as rad_solve_flux (the paper applies C^-1 through its LU factors,
 * §5.2; this library iterates with the stored F instead).
 *   B, Y   column-major n x nrhs (ldB, ldY >= n); nrhs 1 .. 1024
 * Returns RAD_ENOTCONV (Y still written) if a column misses the tolerance;
 * RAD_EINVAL, before any solver work, for an emissivity that is not finite
 * or not in (0, 1], or a value of B that is not finite.
 * ------------------------------------------------------------------------- */
int rad_solve_reflection(const rad_htree* h, const double* eps, const double* B, int64_t ldB, int64_t nrhs,
                         const rad_solve_params* p, double* Y, int64_t ldY, rad_solve_info* info, void* stream);

/* ----------------------------- introspection ----------------------------- */
int rad_htree_get_stats(const rad_htree* h, rad_htree_stats* s);

/* Cluster tree, host arrays.  perm[p] = facet at tree position p (n);
 * per cluster (n_nodes, breadth-first, root first): begin, end, level,
 * child (2 ints, -1 for a leaf), bbox (lo xyz, hi xyz).  Any array may be
 * NULL. */
int rad_htree_export_tree(const rad_htree* h, int32_t* perm, int32_t* begin,
                          int32_t* end, int32_t* level, int32_t* child, double* bbox);

/* Leaf blocks, host arrays of n_blocks in (row begin, column begin) order:
 * row/column cluster ids, admissible flag, stored rank (-1 = stored dense). */
int rad_htree_export_blocks(const rad_htree* h, int32_t* row_node, int32_t* col_node,
                            int32_t* admissible, int32_t* rank);

/* One stored block (index into the export order) as FP64 host arrays:
 * dense blocks fill D (m x n, row-major); low-rank blocks fill U (m x k)
 * and V (n x k), both row-major.  Arrays may be NULL to skip them. */
int rad_htree_export_block(const rad_htree* h, int64_t block, double* D, double* U, double* V);

int rad_htree_free(rad_htree* h);

/* Checkpoint and resume (no counterpart in the paper): rad_htree_save writes
 * everything the handle holds (trees, block partition, compressed operator,
 * work lists, tuning) into buf.  With buf = NULL it only stores the size in
 * *bytes; otherwise *bytes is the buffer's size on entry (RAD_ELIMIT if too
 * small) and the bytes written on return.  Synchronises the device.
 * rad_htree_load builds an identical handle on the current device from such
 * a blob (p may be NULL; only p->allocator is used, as in rad_build_htree):
 * products and solves on it give the same results bit for bit.  A blob that
 * is truncated, from another format version or inconsistent gives RAD_EINVAL
 * before any device work.  Synchronous on `stream`. */
int rad_htree_save(const rad_htree* h, void* buf, uint64_t* bytes);
int rad_htree_load(const void* buf, uint64_t bytes, const rad_tree_params* p, void* stream, rad_htree** out);

const char* rad_last_error(void);

/* ------------------------------------------------------------ tracing
 * rad_launch_count: kernels this library has launched in this process.
 * rad_profile_enable(1) clears the record and starts timing the library's
 * kernels with CUDA events on their launch streams (0 stops it).
 * rad_profile_read aggregates the record by kernel name (synchronising the
 * events): up to max_kernels entries, names as 48-byte NUL-terminated slots,
 * launch counts and summed milliseconds; returns the number of names. */
int64_t rad_launch_count(void);
int rad_profile_enable(int32_t on);
int rad_profile_read(int32_t max_kernels, char* names, int64_t* counts, double* total_ms);

/* ------------------------------------------------------------ serving
 * A flux-solve server (no counterpart in the paper; a runtime around the
 * calls above).  Cavities are registered once; each request is a flux solve
 * (rad_solve_flux) on a registered cavity with its own emissivities and
 * temperature fields, e.g. one time step of a transient computation.
 *
 * Continuous batching: `slots` worker threads, each with its own CUDA
 * stream, take requests as they arrive; the requests in flight run
 * concurrently on the device.  A cavity's compressed operator is built on
 * its first request and stays resident in device memory for later ones.
 * Admission is by a device-memory budget: a request whose cavity is not
 * resident waits until its operator fits (estimated from the facet count,
 * corrected to the actual size once built) next to the resident ones; idle
 * resident operators are evicted least recently used first.  Requests
 * whose cavity is resident are admitted ahead of waiting ones.  Every
 * request's arithmetic is the same alone and in any mix: each runs on one
 * stream with deterministic kernels on the same operator bits.
 *
 * Requests take host arrays; the caller keeps eps, T and q alive until
 * rad_server_wait returns for the ticket. */
typedef struct rad_server rad_server;

typedef struct {
    int32_t slots;               /* concurrent requests (worker threads), >= 1 */
    int32_t reserved;
    int64_t hbm_budget_bytes;    /* resident operators + request workspaces   */
    rad_tree_params tree;        /* cluster/block tree of a new cavity; its
                                    allocator (copied at creation) serves every
                                    operator and request of the server          */
    rad_aca_params aca;          /* its compression                            */
    rad_solve_params solve;      /* every request's solve                      */
} rad_server_params;

typedef struct {
    int32_t status;              /* RAD_OK, RAD_ENOTCONV or the failing code   */
    int32_t built;               /* 1 if this request built its operator      */
    int32_t iters;               /* GMRES iterations                           */
    int32_t refinements;         /* refinement steps                           */
    double  max_rel_residual;    /* as in rad_solve_info                       */
    double  queue_ms;            /* submit -> start on a worker               */
    double  service_ms;          /* start -> done (build, compress, solve)    */
    double  latency_ms;          /* submit -> done                             */
    int32_t slot;                /* worker that ran it                         */
    int32_t reserved;
} rad_request_info;

typedef struct {
    int64_t submitted, completed, failed;
    int64_t builds, evictions;
    int64_t resident_bytes;      /* operators resident now                     */
    int64_t peak_bytes;          /* peak of resident + reserved                */
    int32_t resident_cavities, in_flight;
    double  p50_latency_ms, p99_latency_ms, max_latency_ms;
    double  mean_service_ms;
} rad_server_stats;

int rad_server_create(const rad_server_params* p, rad_server** out);
/* Registers a cavity (verts copied from host or device; n triangles as in
 * rad_build_htree); nothing is built until a request needs it. */
int rad_server_add_cavity(rad_server* s, int64_t n, const double* verts, int64_t* cavity_id);
/* Queues a flux solve of m fields on a registered cavity (arguments as in
 * rad_solve_flux, host arrays); returns at once with a ticket. */
int rad_server_submit(rad_server* s, int64_t cavity_id, const double* eps, const double* T, int64_t ldT,
                      int64_t m, double sigma, double* q, int64_t ldq, int64_t* ticket);
/* Blocks until the ticket's request is done; its q is written.  Returns the
 * request's status (info may be NULL). */
int rad_server_wait(rad_server* s, int64_t ticket, rad_request_info* info);
int rad_server_get_stats(rad_server* s, rad_server_stats* st);
/* Waits for every queued request, stops the workers, frees the operators. */
int rad_server_destroy(rad_server* s);

/* Library version: major * 10000 + minor * 100 + patch. */
int rad_version(void);

/* 1 in the bounds-checked build of this library (librad_checked.so, built
 * with RAD_CHECK_BOUNDS), 0 otherwise.  In that build every device
 * allocation carries 256 canary bytes on each side; they are verified when
 * the memory is returned and before every call returns, and a call after
 * which one was overwritten returns RAD_ECUDA ("bounds check: ...").  The
 * checks synchronise the device and are meant for testing, not speed. */
int rad_debug_bounds_checks(void);

#ifdef __cplusplus
}
#endif
#endif /* RAD_H */
