/*
 * spaqr.h — C ABI of the GB300 spaQR library (sparsified QR preconditioner).
 *
 * Method: Gnanasekaran & Darve, "Hierarchical Orthogonal Factorization:
 * Sparse Square Matrices" (arXiv 2010.06807).  The library solves A x = b for a
 * sparse, unsymmetric, full-rank A in R^{N x N} (Section 1) by
 *   1. a geometric modified nested-dissection ordering (Section 2.3),
 *   2. the spaQR factorisation Q^T A W^{-1} ~ I (Algorithm 2, Section 2.7):
 *      block Householder QR of every separator (Section 2.4), block-diagonal
 *      scaling (Section 2.5, "Scaling of Interfaces") and sparsification of
 *      every interface by a column-pivoted QR truncated at eps (Sections 2.2,
 *      2.5; rank rule of Section 4), merging interfaces level by level
 *      (Section 2.6),
 *   3. the application x = W^{-1} Q^T b of the stored factor sequence
 *      (Section 2.7), used as a right preconditioner inside GMRES that stops at
 *      ||b - A x||_2 / ||b||_2 <= tol (Section 4).
 *
 * Conventions (all entry points):
 *   - Return value 0 is SPAQR_OK; errors are negative SPAQR_ERR_* codes.  No
 *     C++ exception crosses this boundary.  spaqr_last_error() gives a
 *     thread-local message for the last failure.
 *   - Handles are opaque and owned by the library; the caller frees them with
 *     the matching *_destroy function.  Input arrays are borrowed, never freed.
 *   - Dense vectors / right-hand sides are column-major with a leading
 *     dimension; they may live in host or device memory (detected with
 *     cudaPointerGetAttributes).  Host buffers are copied through the device.
 *   - `stream` arguments are cudaStream_t values passed as void* (NULL = the
 *     legacy default stream).  Calls return after the work on `stream` has
 *     completed unless stated otherwise.
 *   - Every numeric step runs in the library's CUDA kernels on the current
 *     device; there is no CPU fallback.  The ordering is integer host work.
 */
#ifndef SPAQR_H
#define SPAQR_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define SPAQR_OK                 0
#define SPAQR_ERR_INVALID_ARG   -1   /* bad pointer, size, stride or option */
#define SPAQR_ERR_UNSUPPORTED   -2   /* e.g. unknown precision, rows too dense for the G(A^T A) ordering */
#define SPAQR_ERR_OOM           -3   /* device allocation failed */
#define SPAQR_ERR_SINGULAR      -4   /* zero diagonal in an R_ss or R_pp factor */
#define SPAQR_ERR_NOT_CONVERGED -5   /* GMRES hit maxit; X holds the last iterate */
#define SPAQR_ERR_TIMEOUT       -6   /* reserved: a bounded device wait ran out */
#define SPAQR_ERR_CUDA          -7   /* a CUDA runtime call failed */
#define SPAQR_ERR_NO_DEVICE     -8   /* no CUDA device is visible */

/* precision of the factorisation and of its application; GMRES, the column
 * scaling, the Householder scalars and the CPQR rank decisions are always
 * FP64 */
#define SPAQR_FP64 0   /* FP64 storage and arithmetic */
#define SPAQR_FP32 1   /* FP32 storage; the contractions of large fronts on the tensor
                          cores in three TF32 passes (about FP32 accuracy) */
#define SPAQR_TF32 2   /* FP32 storage; those contractions in one TF32 pass */

/* Row matchings of the ordering of a general matrix (spaqr_order_general). */
#define SPAQR_MATCH_GREEDY      0   /* largest |a_ij| first, then augmenting paths */
#define SPAQR_MATCH_MAX_PRODUCT 1   /* maximum product of the matched |a_ij| */

/* Sparse matrix in CSR form, rows sorted, N x N.  rowptr has n+1 entries,
 * colind/val have nnz entries.  If on_device != 0 the three arrays are device
 * pointers, otherwise host pointers; every call that takes a spaqr_csr checks
 * this against where the arrays are (INVALID_ARG for device memory flagged
 * as host or plain host memory flagged as device; pinned and managed memory
 * pass either way).  Borrowed for the duration of a call. */
typedef struct {
    int64_t n, nnz;
    const int64_t* rowptr;
    const int32_t* colind;
    const double*  val;
    int on_device;
} spaqr_csr;

/* Regular grid the matrix lives on (lexicographic numbering, x fastest).
 * dim = 2 uses nx, ny; dim = 3 uses nx, ny, nz.  n must equal the product. */
typedef struct {
    int dim;
    int nx, ny, nz;
} spaqr_grid;

/* Factorisation options.  eps: truncation tolerance of the rank-revealing QR
 * (|R_ii| >= eps |R_11| is kept, Section 4), eps = 0 keeps everything.
 * nlevels: 0 chooses ceil(log2(N/64)) (Section 4).  skip: number of levels
 * (from the leaves) factored before scaling/sparsification starts.
 * scaling: 1 (default) scales every interface before sparsifying it
 * (Section 2.5: A_pp -> I); 0 selects the unscaled variant of Sections
 * 2.2 / 3.2: no scaling, M_p = [A_np^T | sigma_p A_pp^T A_pn] with
 * sigma_p = 1 / sigma_min([A_pp; A_np]) (Lemma 1), then a Householder QR of
 * the fine columns of A_pp Q_p whose R_fn part is dropped.  precision:
 * SPAQR_FP64 (plain form) or SPAQR_FP32 (mixed form: factor stored and
 * applied in FP32, CPQR pivots from FP32 norms but each |R_kk| recomputed in
 * FP64 for the rank decision; GMRES around it stays FP64).
 * col_normalize: scale columns of A to unit 2-norm first (Section 2.7). */
typedef struct {
    double eps;
    int nlevels;
    int skip;
    int scaling;
    int precision;
    int col_normalize;
    void* stream;
} spaqr_opts;

/* Default options: eps 1e-2, nlevels 0, skip 2, scaling 1, FP64, normalise. */
void spaqr_opts_default(spaqr_opts* o);

typedef struct spaqr_ordering spaqr_ordering;
typedef struct spaqr_factor_s spaqr_factor_t;

/* Ordering summary (spaqr_ordering_info). */
typedef struct {
    int64_t n;          /* matrix size */
    int64_t nnz;        /* nonzeros of the pattern */
    int32_t nlevels;    /* L */
    int32_t n_atoms;    /* finest interface clusters (incl. leaves) */
    int32_t n_nodes;    /* nodes of the nested-dissection tree */
    int64_t plan_len;   /* int32 entries of the encoded symbolic plan */
} spaqr_ordering_info_t;

/* Factor summary (spaqr_factor_info). */
typedef struct {
    int64_t n;
    int32_t nlevels;
    int32_t skip;
    double  eps;
    int64_t factor_bytes;      /* device bytes held by the factor */
    int64_t solve_bytes;       /* algorithmic bytes one application reads (nrhs = 1) */
    double  factor_flops;      /* algorithmic FP64 flops of the factorisation */
    double  solve_flops;       /* algorithmic flops of one application per RHS */
    int32_t n_interfaces_sparsified;
    int64_t rank_sum;          /* sum of kept ranks over all sparsified interfaces */
    int64_t size_sum;          /* sum of interface sizes before sparsification */
    double  phase_ms[4];       /* factorize / scale / sparsify / merge, CUDA events */
    int32_t top_size;          /* size of the root separator when it was factored */
    int64_t peak_bytes;        /* most device bytes the factorisation held at once (factor + temporaries) */
    int64_t workspace_rows;    /* scratch rows per right-hand side of one application (level vectors
                                  and partial sums), in elements of the factor's precision */
    int32_t precision;         /* SPAQR_FP64 or SPAQR_FP32: storage of the factor */
    int32_t tc_levels;         /* levels whose fronts were applied on the tensor cores */
} spaqr_info;

/* Per-level diagnostics (spaqr_factor_level), level index k = 0 at the
 * leaves: the quantities the paper's profiling figures plot per level
 * (Section 4: sizes, ranks, time per phase). */
typedef struct {
    int32_t n_fronts;          /* separators factored at this level */
    int32_t max_front_rows;    /* tallest front (rows of R(s), Section 2.4) */
    int32_t max_front_cols;    /* widest front (|s|) */
    int32_t n_interfaces;      /* interfaces sparsified at this level (0 below skip) */
    int64_t front_rows;        /* sum of the front heights */
    int64_t front_cols;        /* sum of |s| */
    int32_t n_remaining;       /* clusters left after the fronts (interfaces) */
    int32_t max_interface;     /* largest of them before sparsification */
    int64_t remaining_size;    /* sum of their sizes before sparsification */
    int64_t interface_after;   /* sum after sparsification (= before when not sparsified) */
    int64_t block_entries;     /* dense entries of the level's block arena */
    int64_t factor_bytes;      /* device bytes held by the factor after this level */
    double  phase_ms[4];       /* factorize / scale / sparsify / merge of this level, CUDA events */
} spaqr_level_info;

/* Kinds of stored factor blocks (spaqr_factor_block).  Every block is a
 * dense column-major matrix; clusters are named by their first atom (the
 * finest cluster they contain), the same names at every level. */
#define SPAQR_BLK_FRONT      0  /* separator s (Section 2.4): the front panel after
                                   its Householder QR, rows R(s) stacked in
                                   ascending cluster order (s first), |s|
                                   columns: reflectors below the diagonal
                                   (unit diagonal implied), R_ss on and above */
#define SPAQR_BLK_FRONT_TAU  1  /* the |s| Householder scalars of that QR */
#define SPAQR_BLK_RSJ        2  /* R_sj: row s of the triangular factor in column
                                   cluster j (`other`), |s| x |j| */
#define SPAQR_BLK_SCALE      3  /* interface p (Section 2.5): A_pp = U_pp R_pp after
                                   its Householder QR, reflectors of U_pp below the
                                   diagonal, R_pp on and above, |p| x |p| */
#define SPAQR_BLK_SCALE_TAU  4  /* the |p| Householder scalars of U_pp */
#define SPAQR_BLK_CPQR       5  /* Q_pp of the truncated CPQR of M_p (Sections 2.2,
                                   2.5, 4): |p| x r reflectors, unit diagonal and
                                   zeros above it stored explicitly */
#define SPAQR_BLK_CPQR_TAU   6  /* the r Householder scalars of Q_pp */
#define SPAQR_BLK_FINE       7  /* unscaled form (Section 3.2): |p| x |p|, columns
                                   0..r-1 = H_p^T (A_pp Q_p)[:, :r] (R_fc on top,
                                   the new coarse diagonal block below), columns
                                   r.. = the QR of the fine columns A_pp Q_pf
                                   (reflectors of H_p below the diagonal, R_ff on
                                   and above) */
#define SPAQR_BLK_FINE_TAU   8  /* the |p| - r Householder scalars of H_p */

/* Description of one stored block (spaqr_factor_block). */
typedef struct {
    int32_t level;      /* 0 = the leaves */
    int32_t kind;       /* SPAQR_BLK_* */
    int32_t cluster;    /* s or p (first atom) */
    int32_t other;      /* column cluster j of SPAQR_BLK_RSJ, else -1 */
    int32_t rows, cols;
} spaqr_block_info;

/* Last error message of the calling thread (never NULL). */
const char* spaqr_last_error(void);

/* Geometric modified nested dissection of the matrix pattern on grid g
 * (Sections 2.1, 2.3): separators two grid planes thick (a vertex separator of
 * G(A^T A) for 5/7-point stencils), interfaces from the cuts of descendant
 * subdomains, cluster hierarchy, row order = column order.  Host-only integer
 * work (a device pattern is copied to the host; INVALID_ARG unless rowptr
 * runs from 0 to nnz without decreasing and every column index is in
 * [0, n)).  nlevels = 0 picks
 * ceil(log2(N/64)).  g == NULL orders a general sparse matrix instead
 * (Section 2.3 uses a hypergraph partitioner and MC64 there; this is our
 * restatement): nested dissection on G(A^T A) with breadth-first level sets
 * as separators (pseudo-peripheral start), interfaces from the descendant
 * subdomains each separator column is adjacent to, and rows assigned by a
 * matching that puts large |a_ij| on the diagonal (the maximum-product
 * matching of spaqr_order_general; A->val may be NULL for a pattern-only
 * matching).  SINGULAR if the
 * pattern has no perfect row matching; UNSUPPORTED if the squared row
 * lengths sum above 2^31 (G(A^T A) too large to form).  Also builds the
 * symbolic plan:
 * per level the active clusters, the block pattern with fill, the fronts and
 * their processing order.  *out is owned by the caller
 * (spaqr_ordering_destroy). */
int spaqr_order(const spaqr_csr* A, const spaqr_grid* g, int nlevels, spaqr_ordering** out);

/* The ordering of a general sparse matrix (spaqr_order with g == NULL) with a
 * choice of row matching (Section 2.3 assigns rows by a bipartite matching
 * that puts large entries on the diagonal, MC64 in the paper):
 *   SPAQR_MATCH_GREEDY: entries by decreasing |a_ij| (ties: row, column)
 *     matched greedily, then every unmatched row by an augmenting path;
 *   SPAQR_MATCH_MAX_PRODUCT (what spaqr_order uses): the perfect matching
 *     maximising the product of
 *     the matched |a_ij| (the product matching of MC64): minimum cost on
 *     c_ij = log max_k |a_kj| - log |a_ij| over the nonzero values
 *     (duplicates summed, explicit zeros dropped) by shortest augmenting
 *     paths with dual potentials; A->val NULL makes every entry 1.
 * Row r then sits with its matched column.  Errors as spaqr_order, plus
 * INVALID_ARG for another `matching` or a NaN / infinite value in A->val,
 * and SINGULAR when no perfect matching exists on the nonzero values (an
 * empty column included). */
int spaqr_order_general(const spaqr_csr* A, int nlevels, int matching, spaqr_ordering** out);

/* Ordering of a batch of independent matrices A[0..count-1] on grids
 * g[0..count-1], treated as the block-diagonal matrix diag(A_0, ..., A_{c-1})
 * (rows and columns of A_i at base_i = n_0 + ... + n_{i-1}).  Every matrix
 * gets the nested dissection spaqr_order gives it with nlevels = 0, and the
 * trees are aligned at their leaves: level k of the batch (from the leaves)
 * holds level k of every matrix with more than k levels, so a factorisation
 * with this ordering (spaqr_factor on the block-diagonal CSR) runs each
 * level's fronts of all matrices in the same launches, with one host
 * synchronisation per level for the whole batch.  The batch's level count is
 * the largest one.  Errors as spaqr_order; *out is owned by the caller.
 * (Batching independent systems is not in the paper; each matrix's
 * factorisation is the one Algorithm 2 gives it alone.) */
int spaqr_order_batch(int count, const spaqr_csr* A, const spaqr_grid* g, spaqr_ordering** out);

/* Sizes of the ordering's arrays. */
int spaqr_ordering_info(const spaqr_ordering* ord, spaqr_ordering_info_t* info);

/* Copy the ordering out: perm[new] = old index (n entries), atom_ptr
 * (n_atoms+1 entries), atom_node (n_atoms entries, preorder id of the atom's
 * nested-dissection node), node_level (n_nodes entries, 1 = root) and the
 * encoded symbolic plan (plan_len int32).  Any pointer may be NULL to skip it.
 * Plan encoding, per level k = 1..L:
 *   level, n_clusters, cluster first-atom ids...,
 *   n_fronts, then per front in processing order:
 *     front id, colour, |R|, R ids..., |C|, C ids... */
int spaqr_ordering_get(const spaqr_ordering* ord, int64_t* perm, int64_t* atom_ptr,
                       int32_t* atom_node, int32_t* node_level, int32_t* plan);

/* Row order of the ordering: rperm[new] = old row (n entries).  Equals perm
 * for grid orderings (rows ordered as columns); for a general matrix, row
 * rperm[k] is the row matched to column perm[k].
 * Errors: INVALID_ARG (null argument). */
int spaqr_ordering_rows(const spaqr_ordering* ord, int64_t* rperm);

void spaqr_ordering_destroy(spaqr_ordering* ord);

/* Numeric spaQR factorisation (Algorithm 2) of A with the ordering `ord`
 * (same pattern).  A may be on host or device.  Runs on opts->stream and
 * returns after the factor is complete.  The factor lives in device memory of
 * the current device and is immutable afterwards, so concurrent
 * spaqr_solve / spaqr_gmres calls on different streams may share it.
 * Temporaries come from the device's default memory pool (cudaMallocAsync);
 * the first call on a device raises that pool's release threshold so freed
 * memory stays with the process for reuse.
 * Errors: INVALID_ARG (scaling other than 0 / 1), UNSUPPORTED (unknown
 * precision), SINGULAR (zero column, zero diagonal of R_ss / R_pp, a rank
 * deficient A_p or R_ff of the unscaled variant), OOM, CUDA, NO_DEVICE. */
int spaqr_factor(const spaqr_ordering* ord, const spaqr_csr* A, const spaqr_opts* opts,
                 spaqr_factor_t** out);

/* One application of the preconditioner, X = W^{-1} Q^T B (Section 2.7, in
 * the original unknowns, column scaling undone).  B: n x nrhs with leading
 * dimension ldb >= n; X: n x nrhs with ldx >= n.  B and X may alias only if
 * they are the same pointer with the same leading dimension.  Host or device
 * pointers (both on the same side).  Synchronous on `stream`.
 * Errors: INVALID_ARG, SINGULAR, OOM, CUDA. */
int spaqr_solve(const spaqr_factor_t* F, int nrhs, const double* B, int64_t ldb,
                double* X, int64_t ldx, void* stream);

/* Allocation-free variant of spaqr_solve: X = M^{-1} B with the same kernels,
 * for callers that cannot allocate device memory while they run -- for
 * example code whose device memory is fully reserved by another allocator
 * (a framework's caching pool), or a control loop that must not enter the CUDA
 * allocator because cudaMalloc / cudaFree can synchronise the device and take
 * an unbounded time.  The paper has no counterpart; it is an interface
 * convenience.
 * The scratch space (one vector per level plus partial sums:
 * spaqr_info.workspace_rows x nrhs elements of the factor's precision, i.e.
 * ceil(workspace_rows x nrhs x element bytes / 8) doubles) lives in a fixed
 * array of SPAQR_NOALLOC_SCRATCH_DOUBLES doubles
 * (16 MiB) inside the library, which every GPU that loads the library holds
 * until the process exits.  Calls needing more return SPAQR_ERR_INVALID_ARG
 * (use fewer right-hand sides per call).  B and X must be device pointers
 * (n x nrhs, leading dimensions ldb, ldx >= n; same aliasing rule as
 * spaqr_solve), device memory of the factor's GPU.  The first call on a
 * device looks up the array's device
 * address (cudaGetSymbolAddress); make that first call before any stream
 * capture.  All calls share the one array, so calls that overlap on the GPU
 * (other streams, other host threads) race and must be serialised by the
 * caller.  Nothing is allocated or freed (keep spaqr_profile off: profiling
 * creates CUDA events).  Synchronous on `stream`.
 * Errors: INVALID_ARG (size, host pointers), SINGULAR, CUDA. */
#define SPAQR_NOALLOC_SCRATCH_DOUBLES (2 * 1024 * 1024)
int spaqr_solve_noalloc(const spaqr_factor_t* F, int nrhs, const double* B, int64_t ldb,
                        double* X, int64_t ldx, void* stream);

/* Right-preconditioned GMRES (Section 4) for the nrhs columns of B, each with
 * its own Krylov space, using F as preconditioner and A (CSR, host or device)
 * for products.  The flexible form is used (the preconditioned vectors
 * Z_j = M^{-1} v_j are kept and x = x0 + Z y), so an FP32 factor, whose
 * application is not exactly linear, still converges to FP64 accuracy.  X on entry is the initial guess, on exit the solution.
 * Converged when the explicitly recomputed ||b - A x||_2 / ||b||_2 <= tol.
 * iters[c] and relres[c] (host arrays of nrhs entries, may be NULL) receive
 * per-column iteration counts and final relative residuals.  maxit bounds the
 * Krylov dimension (no restart).  Returns NOT_CONVERGED if any column missed
 * tol (X holds the last iterate).  Synchronous on `stream`.
 * A must be the factored matrix: INVALID_ARG if A->nnz differs from the
 * factored pattern's, and, for a host CSR, if its rowptr does not run from 0
 * to nnz without decreasing or a column index is out of range (checked
 * before any kernel); a device CSR is trusted (its SpMV reads it as given). */
int spaqr_gmres(const spaqr_factor_t* F, const spaqr_csr* A, int nrhs, const double* B,
                int64_t ldb, double* X, int64_t ldx, double tol, int maxit, int* iters,
                double* relres, void* stream);

/* spaqr_gmres with the residual history the paper's convergence figures plot
 * (Section 4): `history` (host, nrhs * maxit doubles, not NULL) receives for
 * column c at history[c * maxit + j] the Arnoldi estimate |g_{j+1}| / ||b_c||
 * of the relative residual after iteration j + 1 (the quantity the stopping
 * test reads), for j < iters[c]; the remaining entries are NaN.  The
 * estimates are non-increasing.  Errors as spaqr_gmres, plus INVALID_ARG for
 * a NULL history. */
int spaqr_gmres_history(const spaqr_factor_t* F, const spaqr_csr* A, int nrhs, const double* B,
                        int64_t ldb, double* X, int64_t ldx, double tol, int maxit, int* iters,
                        double* relres, double* history, void* stream);

/* GMRES for a batch factorised with a spaqr_order_batch ordering: A is the
 * block-diagonal CSR diag(A_0, ..., A_{count-1}) (n = part_ptr[count]), and
 * part_ptr[0..count] (host, int64) are the row offsets of the matrices
 * (part_ptr[0] = 0, strictly increasing).  Every (matrix i, column c) pair is
 * its own Krylov process, exactly as spaqr_gmres runs it on A_i alone up to
 * rounding: its residual ||b_i - A_i x_i|| / ||b_i|| is what tol bounds, and it
 * stops on its own.  The SpMV and the factor application of an iteration are
 * one pass over the whole batch (every level's fronts of all matrices in the
 * same launches).  iters and relres hold count * nrhs entries, entry
 * c * count + i for matrix i and column c (may be NULL).  B, X as spaqr_gmres.
 * Errors as spaqr_gmres, plus INVALID_ARG for a bad part_ptr.  (The paper
 * solves one system at a time; batching is an addition.) */
int spaqr_gmres_batch(const spaqr_factor_t* F, const spaqr_csr* A, int count, const int64_t* part_ptr,
                      int nrhs, const double* B, int64_t ldb, double* X, int64_t ldx, double tol, int maxit,
                      int* iters, double* relres, void* stream);

/* Summary and timings of a factor. */
int spaqr_factor_info(const spaqr_factor_t* F, spaqr_info* out);

/* Number of stored blocks of F (every block the application reads, level by
 * level: fronts, R_sj, scaling and sparsification factors).  For inspection
 * and parity checks; not on the hot path. */
int spaqr_factor_nblocks(const spaqr_factor_t* F, int64_t* count);

/* Block `index` (0 <= index < spaqr_factor_nblocks) of F: its description in
 * *info and, when out is not NULL, a copy of its rows x cols entries in out
 * (host, column-major, leading dimension rows; FP32 factors are widened to
 * double).  Synchronous device-to-host copy on the factor's GPU.
 * Errors: INVALID_ARG (NULL F or info, index out of range), CUDA. */
int spaqr_factor_block(const spaqr_factor_t* F, int64_t index, spaqr_block_info* info, double* out);

/* Per-level interface ranks: for level index k (0 = leaves) writes up to cap
 * pairs (size before, kept rank) of the interfaces sparsified at that level,
 * in ascending cluster order, and the count in *count.  Also the CPQR pivot
 * norms |R_rr| (first rejected or last kept) and |R_11| per interface into
 * margins[2*i], margins[2*i+1] if margins != NULL. */
int spaqr_factor_ranks(const spaqr_factor_t* F, int level, int32_t* pairs, double* margins,
                       int cap, int* count);

/* Diagnostics of level k (0 = leaves) into *out.
 * Errors: INVALID_ARG (null argument, level out of range). */
int spaqr_factor_level(const spaqr_factor_t* F, int level, spaqr_level_info* out);

/* CPQR pivot norms |R_kk| (Section 4's rank rule) of every interface
 * sparsified at level k, in the order of spaqr_factor_ranks: the kept steps
 * and the first rejected one.  Interface i owns norms[offsets[i] ..
 * offsets[i+1]).  Writes up to cap norms and cap_offsets offsets (either
 * array may be NULL) and the totals into *n_norms and *n_interfaces.
 * Errors: INVALID_ARG (null counts, level out of range). */
int spaqr_factor_pivots(const spaqr_factor_t* F, int level, double* norms, int64_t cap, int32_t* offsets,
                        int cap_offsets, int64_t* n_norms, int* n_interfaces);

/* sigma_p = 1 / sigma_min(A_p) of the interfaces sparsified at level k by the
 * unscaled variant (Lemma 1), in the order of spaqr_factor_ranks; 0 for the
 * scaled variant.  Writes up to cap values into sigma (may be NULL) and the
 * count into *count.  Computed on the device in FP64: Householder QR of A_p,
 * then Lanczos with full reorthogonalisation on (R^T R)^{-1}, stopped when
 * the largest Ritz value of four consecutive steps agrees to 1e-15 relative.
 * Errors: INVALID_ARG (null F or count, level out of range). */
int spaqr_factor_sigmas(const spaqr_factor_t* F, int level, double* sigma, int cap, int* count);

void spaqr_factor_destroy(spaqr_factor_t* F);

/* Autotuner of the factor application for nrhs right-hand sides.  Every
 * unit of the application (the fronts of one colour of a level forward, the
 * scale-sparsify step of a level forward and backward, the fronts of a level
 * backward) has two launch forms: one CTA per front / interface, or one
 * thread-block cluster per front / interface (with the R_sj products as
 * separate tiles).  The tuner times both forms of every unit on this factor
 * (CUDA events, best of three runs from the same workspace snapshot, on
 * stream), keeps the faster, and times whole applications with the untuned
 * rules and with the table (*ms_rule, *ms_tuned; may be NULL).  The table is
 * stored in F and used by later spaqr_solve / spaqr_gmres calls with the
 * same nrhs (or, without a table for their nrhs, the nearest tuned count) if
 * it is faster than the rules; the results do not depend on the
 * forms chosen beyond rounding.  Must not run concurrently with another call
 * on F.  Synchronises the stream.  Errors: INVALID_ARG (profiling on, bad
 * arguments), OOM, CUDA.  (Launch-form tuning is ours; the paper has no
 * counterpart.) */
int spaqr_autotune(spaqr_factor_t* F, int nrhs, void* stream, double* ms_rule, double* ms_tuned);

/* The launch forms spaqr_autotune kept for nrhs, level by level (0 = leaves):
 * one entry per forward colour of the level, then the level's forward
 * scale-sparsify, backward scale-sparsify and backward fronts; 1 = one CTA
 * per front / interface, 2 = a cluster of 8 CTAs per front / interface,
 * 3 = the staged cluster kernels with one CTA.  Writes up to cap entries and
 * the total in *count (0: no table for nrhs, the rules apply). */
int spaqr_factor_tuning(const spaqr_factor_t* F, int nrhs, int32_t* forms, int cap, int* count);

/* Process-wide switch (default on): spaqr_gmres / spaqr_gmres_batch run on a
 * private non-blocking stream ordered after the caller's stream, and capture
 * the factor application of an iteration once per call as a CUDA graph that
 * every iteration replays (the same kernels with the same arguments, so the
 * results are identical).  Off, or while profiling is on, every iteration
 * launches the kernels directly on the caller's stream. */
void spaqr_use_graphs(int on);

/* Process-wide switch (default on): factorisations with FP32 storage
 * (SPAQR_FP32, SPAQR_TF32) apply the reflectors of the levels whose fronts
 * are large on the tensor cores (spaqr_tc_gemm's products: compact-WY form
 * Q^T B = B - V T^T (V^T B), Section 2.4).  Off, every front is applied on the
 * CUDA cores as in the FP64 form.  Read when a factorisation starts. */
void spaqr_use_tensor_cores(int on);

/* Testing aid (host-side fault injection; the paper has no counterpart):
 * after `after` more successful device allocations of the library, the next
 * one reports failure exactly as a failed cudaMallocAsync would, once; the
 * call then returns SPAQR_ERR_OOM after releasing what it allocated.
 * after < 0 switches the injection off.  Process wide. */
void spaqr_test_fail_alloc(int64_t after);

/* Kernel launch statistics (process wide).  The paper reports the runtime of
 * every level split into factorize / scale / sparsify / merge (Section 4,
 * "runtime per level" figure); these counters refine that split per kernel.
 * launches counts every kernel the library enqueues; with profiling on
 * (spaqr_profile(1)) each launch is also bracketed by CUDA events on its
 * stream and total_ms sums their durations.  flops / bytes are the
 * algorithmic FP64 flops and bytes of the counted launches (from block sizes,
 * not from hardware counters). */
typedef struct {
    char name[32];
    int64_t launches;
    double total_ms;
    double flops;
    double bytes;
    double idle_ms;     /* with spaqr_profile(1): time the stream stood idle between the
                           previous profiled launch on it and each launch of this kind
                           (the GPU waiting for the host); an upper bound, since the
                           event records add host time of their own */
} spaqr_kernel_stat;

/* Zero all counters and drop pending event records. */
void spaqr_stats_reset(void);
/* on != 0: record CUDA events around every launch from now on. */
void spaqr_profile(int on);
/* Copy up to cap per-kernel records into out (cap may be 0), set *count to
 * the number of kernel kinds and *total_launches to the launch count since the
 * last reset.  Waits for pending events.  Errors: INVALID_ARG, CUDA. */
int spaqr_stats(spaqr_kernel_stat* out, int cap, int* count, int64_t* total_launches);

/* ---- Measurement aids (the paper has no counterpart) ---- */

/* Arithmetic peak microbenchmarks of the current GPU, the denominators of
 * roofline fractions: which = SPAQR_PEAK_DFMA (FP64 fused multiply-add on
 * the CUDA cores), SPAQR_PEAK_DMMA (FP64 mma.sync m8n8k4), SPAQR_PEAK_FFMA
 * (FP32 fused multiply-add), SPAQR_PEAK_TF32 (tcgen05.mma kind::tf32,
 * M = 128, N = 256, FP32 accumulation in tensor memory).  One warm-up launch,
 * then `reps` timed launches on the legacy default stream with CUDA events;
 * *flops = flops of one launch, *ms = mean milliseconds per launch.
 * Errors: INVALID_ARG, OOM, TIMEOUT (a bounded tensor-core wait ran out),
 * CUDA. */
#define SPAQR_PEAK_DFMA 0
#define SPAQR_PEAK_DMMA 1
#define SPAQR_PEAK_FFMA 2
#define SPAQR_PEAK_TF32 3
int spaqr_peak(int which, int reps, double* flops, double* ms);

/* Latency microbenchmark: clock cycles per operation of a dependent chain,
 * in one CTA of `warps` warps (1..32) with the operation in lanes
 * 0..lanes-1 (1..32) of every warp; *cycles = the slowest warp's cycles per
 * operation.  op: SPAQR_OP_DFMA, SPAQR_OP_DADD, SPAQR_OP_DDIV,
 * SPAQR_OP_DSQRT (with one FP64 add), SPAQR_OP_FFMA, SPAQR_OP_F2F
 * (double -> float -> double and one FP64 add), SPAQR_OP_DSEL (FP64 compare,
 * then a multiply or an add).  Synchronous on the current device.  Errors:
 * INVALID_ARG, OOM, CUDA. */
#define SPAQR_OP_DFMA 0
#define SPAQR_OP_DADD 1
#define SPAQR_OP_DDIV 2
#define SPAQR_OP_DSQRT 3
#define SPAQR_OP_FFMA 4
#define SPAQR_OP_F2F 5
#define SPAQR_OP_DSEL 6
int spaqr_op_cycles(int op, int warps, int lanes, double* cycles);

/* Self-check of the tcgen05 TF32 tile the mixed-precision factorisation
 * builds on: D (128 x N, row-major) = A (128 x K, row-major) B^T (B: N x K,
 * row-major), inputs rounded to TF32, FP32 accumulation.  Device pointers;
 * 16 <= N <= 256 with N % 16 == 0, 8 <= K <= 128 with K % 8 == 0, else
 * INVALID_ARG.  Synchronous on `stream`.  Errors: INVALID_ARG, OOM,
 * TIMEOUT, CUDA. */
int spaqr_tc_tile_check(const float* A, const float* B, float* D, int N, int K, void* stream);

/* The tensor-core matrix product of the mixed-precision factorisation, for
 * one product: C = alpha A B + beta C with M x K A, K x N B and M x N C in
 * device memory, FP32, any element strides (A(i, k) = A[i a_rs + k a_cs],
 * B(k, j) = B[k b_rs + j b_cs], C(i, j) = C[i c_rs + j c_cs]).  a_reflectors:
 * A is a factored panel read as its unit lower trapezoidal reflector matrix
 * (entries below the diagonal as stored, 1 on it, 0 above it), the V of
 * Section 2.4's block Householder step.  The product runs on tcgen05.mma
 * kind::tf32 with FP32 accumulation in tensor memory: one TF32 pass, or with
 * split3 three (hi*hi + hi*lo + lo*hi of the TF32 split x = hi + lo, about
 * FP32 accuracy).  beta = 0 does not read C.  Synchronous on `stream`.
 * Errors: INVALID_ARG, OOM, TIMEOUT (a bounded tensor-core wait ran out),
 * CUDA. */
int spaqr_tc_gemm(int M, int N, int K, float alpha, const float* A, int64_t a_rs, int64_t a_cs,
                  int a_reflectors, const float* B, int64_t b_rs, int64_t b_cs, float beta, float* C,
                  int64_t c_rs, int64_t c_cs, int split3, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* SPAQR_H */
