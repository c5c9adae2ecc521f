/*
 * ca_gb300.h -- C-ABI of the GB300 (sm_103a) communication-avoiding LU and QR
 * library: tall-skinny panel factorization by reduction trees (TSLU
 * tournament pivoting, TSQR) and the trailing updates that consume each
 * panel (CALU, CAQR), plus the solves built on the factors.
 *
 * Method: Grigori, Jacquelin, Khabou, "Multilevel communication optimal LU
 * and QR factorizations for hierarchical platforms" (INRIA RR-8270, 2013).
 * Each entry point cites the passage that defines its operation.
 *
 * Common conventions
 *   - Matrices are FP64, column-major, element (i, j) at A[i + j * lda],
 *     lda >= max(1, m).  All matrix, vector and workspace pointers are DEVICE
 *     pointers owned by the caller; the library never allocates, frees or
 *     keeps them after the call returns.
 *   - Every call only enqueues work on `stream` and returns without waiting.
 *     The return value is the synchronous argument check: CA_OK (0), -i when
 *     argument i (1-based) is invalid, or a CA_ERR_* code.  On a non-zero
 *     return nothing has been enqueued and no memory has been touched.
 *   - dev_info (device, 2 ints) is written asynchronously on `stream`:
 *       dev_info[0]  LAPACK-style info: 0, or 1 + the first column whose U
 *                    diagonal is exactly zero (LU; the factorization still
 *                    completes, as in LAPACK getrf);
 *       dev_info[1]  status bits: CA_STATUS_NONFINITE when a NaN or Inf was
 *                    read from a panel.
 *     Read it after synchronizing the stream.
 *   - The reduction tree (ca_tree_t): the panel's rows are cut into leaves of
 *     `leaf_rows` consecutive rows (the last leaf may be shorter).  Level l
 *     groups consecutive nodes of the level below by fan_in[l]; inside a
 *     group, style CA_TREE_BINARY merges neighbours two by two until one node
 *     is left (an odd node is promoted unchanged) and CA_TREE_FLAT merges the
 *     whole group in one step.  The last level always merges all remaining
 *     nodes.  leaf_rows must be >= the panel width b.  (Sec. 3.1 and 3.2:
 *     Pr subsets of the panel per level, log Pr pairwise reduction steps.)
 *     The tree fixes the numerical result; where each node runs on the GPU
 *     (one CTA, a thread-block cluster sharing its rows through distributed
 *     shared memory, successive grid launches) is the library's choice.
 *   - Look-ahead (calu_factor, caqr_factor and their _mixed forms, when there
 *     is more than one panel): the next panel's tree factorization runs on a
 *     helper stream of the highest priority while the current trailing
 *     update finishes on `stream`.  The library creates one helper stream and
 *     two events per (device, caller stream) on first use (up to 64 pairs,
 *     beyond that plain stream order) and keeps them until the process exits.
 *     Every piece of work is ordered by events that start from and end on
 *     `stream`, so the caller sees ordinary stream semantics; results are
 *     bit-identical to the serial order.  Calls on one caller stream must not
 *     be enqueued from two host threads at once.
 */
#ifndef CA_GB300_H
#define CA_GB300_H

#include <stddef.h>
#include <cuda_runtime_api.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CA_MAX_LEVELS 8
#define CA_TREE_BINARY 0
#define CA_TREE_FLAT 1

typedef struct {
  int leaf_rows;              /* rows per leaf, >= panel width               */
  int nlevels;                /* 1 .. CA_MAX_LEVELS                          */
  int fan_in[CA_MAX_LEVELS];  /* nodes per group at each level (>= 2 except  */
                              /* the last level, whose value is ignored)     */
  int style[CA_MAX_LEVELS];   /* CA_TREE_BINARY or CA_TREE_FLAT              */
  /* Reduction operator of the tournament's nodes (LU only).  0: GEPP (the
   * CALU base case).  1 or 2: the 2D multilevel CALU reduction (Algorithm
   * 2D-ML-CALU, Sec. 3.2): every node -- a leaf, or the stacked candidate
   * sets of a reduction step -- is factored by CALU of the level below with
   * panel width op_b[0] over leaves of op_leaf_rows[0] rows and a binary
   * tree; its own nodes use GEPP (depth 1) or, at depth 2, CALU with
   * op_b[1] and op_leaf_rows[1] and GEPP below that.  The node's pivot rows
   * are the first rows of that factorization.  Zero-initialize for GEPP.
   * The LU entry points (calu_factor, tslu, the mixed forms, batched CALU
   * items) accept depth 1 or 2 when every tournament node (leaf_rows rows,
   * or fan-in x panel width rows) has at most 1024 rows and its tile with
   * the operator's scratch tiles fits one CTA's shared memory (about
   * 220 KB in FP64: 256 x 64 leaves, for instance); each node is then
   * factored by one CTA.  QR entry points return CA_ERR_UNSUPPORTED. */
  int op_depth;
  int op_b[2];                /* 1 <= op_b[d] <= op_leaf_rows[d]              */
  int op_leaf_rows[2];
} ca_tree_t;

/* return codes (negative small values -i name a bad argument i) */
#define CA_OK 0
#define CA_ERR_WORKSPACE -1001   /* workspace pointer null or too small      */
#define CA_ERR_UNSUPPORTED -1002 /* valid shape the library cannot run       */
#define CA_ERR_LAUNCH -1003      /* a kernel launch failed (CUDA error)      */
#define CA_ERR_TREE -1004        /* malformed tree                           */
#define CA_ERR_BATCH_ITEM -1005  /* an item of a batch is invalid            */

#define CA_STATUS_NONFINITE 1
#define CA_STATUS_SOLVE_TIMEOUT 16 /* dev_info[1] of calu_gesv_mixed: a solve gave up waiting */
#define CA_STATUS_REFACTORED 32    /* dev_info[1] of calu_gesv_mixed: the fallback refactorization ran */

/* Correction method of calu_gesv_mixed's refinement */
#define CA_REFINE_CLASSIC 0 /* x += M^-1 r, one solve with the reduced-precision factors M */
#define CA_REFINE_GMRES 1   /* x += d, (M^-1 A) d = M^-1 r solved by GMRES                 */
#define CA_REFINE_AUTO 2    /* classic while each step gains 10x, then GMRES, then a      */
                            /* refactorization with 7 exact digits if GMRES stalls too   */

/* Human-readable text for a return code (static storage). */
const char *ca_strerror(int code);

/* ------------------------------------------------------------------------ */
/* Workspace queries (host only, no GPU work).                              */
/* ------------------------------------------------------------------------ */

/* Bytes of device workspace `work` needed by calu_factor / tslu for an
 * m x n matrix with panel width b and this tree.  Also returns CA_OK or an
 * argument error exactly as calu_factor would for the same shape. */
int ca_calu_workspace(int m, int n, int b, const ca_tree_t *tree, size_t *work_bytes);

/* Bytes of the CAQR reflector store `qtree` (the T factors of every tree
 * node, see caqr_factor) and of the scratch workspace `work` for an m x n
 * matrix (m >= n) with panel width b. */
int ca_caqr_workspace(int m, int n, int b, const ca_tree_t *tree, size_t *qtree_bytes,
                      size_t *work_bytes);

/* Bytes of scratch workspace needed by caqr_geqrs (its first bytes are a
 * solve workspace, as for calu_getrs). */
int ca_geqrs_workspace(int m, int n, int nrhs, int b, const ca_tree_t *tree, size_t *work_bytes);

/* Bytes of the solve workspace of calu_getrs for order n (a few hundred
 * bytes: the ready flags of the dependency-ordered triangular solves and a
 * timeout record).  Arguments: 1 n, 2 nrhs, 3 work_bytes. */
int ca_getrs_workspace(int n, int nrhs, size_t *work_bytes);

/* ------------------------------------------------------------------------ */
/* LU with tournament pivoting                                              */
/* ------------------------------------------------------------------------ */

/* calu_factor: P A = L U of the m x n matrix A (any m, n >= 0) by CALU, the
 * one-level base case of 1D-ML-CALU (Algorithm "1D multilevel CALU", Sec. 3.2
 * and the appendix): for each panel of bk = min(b, min(m,n) - kb) columns
 *   1. tournament pivoting (TSLU) over the tree picks bk pivot rows
 *      (leaves: GEPP on each leaf; merges: GEPP on the stacked candidate rows,
 *      original values, children in order);
 *   2. the rows are swapped at left and right of the panel (full width);
 *   3. L21 = A21 U11^-1 and U12 = L11^-1 A12, with L11 U11 the root's factors;
 *   4. A22 -= L21 U12 (Schur complement).
 * Output in LAPACK getrf layout: unit L strictly below the diagonal, U on and
 * above; ipiv[i] (1-based, device, min(m,n) ints) is the row swapped with
 * row i, applied in order i = 0, 1, ....  Arguments: 1 m, 2 n, 3 A, 4 lda,
 * 5 b (>= 1), 6 tree, 7 ipiv, 8 work, 9 lwork, 10 dev_info, 11 stream. */
int calu_factor(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int *ipiv,
                void *work, size_t lwork, int *dev_info, cudaStream_t stream);

/* tslu: the panel factorization alone (TSLU, Sec. 3.2): calu_factor of an
 * m x n tall-skinny matrix with a single panel of width n (n <= 128). */
int tslu(int m, int n, double *A, int lda, const ca_tree_t *tree, int *ipiv, void *work,
         size_t lwork, int *dev_info, cudaStream_t stream);

/* tslu_noalloc: tslu for callers that cannot allocate device memory.  The
 * paper has no counterpart; this is a deployment convenience.  Some callers
 * cannot hand the library a workspace: their device memory is owned by
 * another allocator (a framework's caching allocator, a serving process that
 * reserved its HBM budget up front), or they cannot call cudaMalloc on their
 * path because it may synchronize the device and has no latency bound.  This
 * entry point takes the same inputs and outputs as tslu (arguments: 1 m,
 * 2 n, 3 A, 4 lda, 5 tree, 6 ipiv, 7 dev_info, 8 stream) and allocates
 * nothing: its scratch is one static device array of
 * CA_TSLU_NOALLOC_SCRATCH_BYTES compiled into the library, present on every
 * GPU that loads it until the process exits.
 *   - Limit: shapes whose ca_calu_workspace(m, n, n, tree) exceeds
 *     CA_TSLU_NOALLOC_SCRATCH_BYTES are rejected with CA_ERR_WORKSPACE before
 *     anything is enqueued (about 4M rows at n = 32 with 256-row leaves).
 *   - The first call on each device (with that device current) looks up the
 *     array's device address; make that first call before any stream capture.
 *   - All calls share the one array, which keeps the last call's contents
 *     (every byte a call reads is written earlier in the same call).  Calls
 *     that overlap on the GPU (different streams, or different host threads)
 *     race on it: serialize them.
 *   - Calls no cudaMalloc, cudaFree or other allocating routine (with the
 *     instrumentation below switched off). */
#define CA_TSLU_NOALLOC_SCRATCH_BYTES (16u << 20)
int tslu_noalloc(int m, int n, double *A, int lda, const ca_tree_t *tree, int *ipiv,
                 int *dev_info, cudaStream_t stream);

/* calu_getrs: solve A X = B from calu_factor's output (n x n, PA = LU):
 * apply the ipiv swaps to B, then forward substitution with the unit L and
 * back substitution with U (Sec. 3.2: PA = LU).  B is n x nrhs (ld ldb),
 * overwritten with X.  work: device memory of ca_getrs_workspace bytes, owned
 * by the caller (the triangular solves with up to 16 right-hand sides order
 * their 128-row blocks by ready flags kept there; the library allocates
 * nothing); one workspace must not be used by two solves in flight at once.
 * Arguments: 1 n, 2 nrhs, 3 LU, 4 lda, 5 ipiv, 6 B, 7 ldb, 8 work, 9 lwork,
 * 10 stream. */
int calu_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb,
               void *work, size_t lwork, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* QR by tree-based Householder reflections                                 */
/* ------------------------------------------------------------------------ */

/* caqr_factor: A = Q R of the m x n matrix A (m >= n) by CAQR, the one-level
 * base case of ML-CAQR (Algorithm ML-CAQR, Sec. 3.1): for each panel,
 *   1. TSQR: Householder QR of every leaf, then of every merge node's stacked
 *      upper-triangular R factors (the R-elimination tree);
 *   2. the trailing columns get every leaf's Q^T (UPFACT), then every merge
 *      node's Q^T bottom-up (UPELIM).
 * Q is kept in the compact Y T Y^T form (Sec. 3.1), stored in a tree
 * structure:
 *   - leaf j of panel k: Householder vectors strictly below the leaf-local
 *     diagonal of its rows (unit diagonal implied), R in its top
 *     c = min(rows, bk) rows;
 *   - merge node: the new R overwrites the first child's R rows on and above
 *     the diagonal; child i >= 1's block of Y (upper trapezoidal, c_i x bk)
 *     overwrites child i's R rows on and above the diagonal (the first
 *     child's block of Y is the identity and is not stored);
 *   - qtree (device doubles): for each panel in order, (nleaves + nmerges)
 *     blocks of b x b doubles (column-major, ld b): the leaves' T in leaf
 *     order, then the merges' T in tree order (level by level, left to
 *     right); each c x c upper-triangular T sits in the block's top-left
 *     corner, zeros elsewhere.
 * So the final R is the upper triangle of A's top n rows.  Arguments:
 * 1 m, 2 n, 3 A, 4 lda, 5 b, 6 tree, 7 qtree, 8 qtree_bytes, 9 work,
 * 10 lwork, 11 dev_info, 12 stream. */
int caqr_factor(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, double *qtree,
                size_t qtree_bytes, void *work, size_t lwork, int *dev_info, cudaStream_t stream);

/* tsqr: the panel factorization alone (TSQR, Sec. 3.1 R-elimination tree):
 * caqr_factor of an m x n tall-skinny matrix with one panel of width n
 * (n <= 128). */
int tsqr(int m, int n, double *A, int lda, const ca_tree_t *tree, double *qtree,
         size_t qtree_bytes, void *work, size_t lwork, int *dev_info, cudaStream_t stream);

/* caqr_geqrs: least-squares solve min ||A X - B|| from caqr_factor's output
 * (same m, n, b and tree): B <- Q^T B panel by panel through the tree
 * (leaves, then merges), then X = R^-1 (Q^T B)(0:n) in B's top n rows
 * (Sec. 3.1: A = QR).  B is m x nrhs (ld ldb).  Arguments: 1 m, 2 n, 3 nrhs,
 * 4 QR, 5 lda, 6 b, 7 tree, 8 qtree, 9 qtree_bytes, 10 B, 11 ldb, 12 work,
 * 13 lwork, 14 stream. */
int caqr_geqrs(int m, int n, int nrhs, const double *QR, int lda, int b, const ca_tree_t *tree,
               const double *qtree, size_t qtree_bytes, double *B, int ldb, void *work,
               size_t lwork, cudaStream_t stream);

/* ca_solve_status: the dependency-ordered triangular solves of calu_getrs
 * and caqr_geqrs wait for ready flags in their workspace; every wait is
 * bounded (about 2 s of SM clock) and a wait that gives up is recorded in the
 * workspace (the first int; each solve clears it when it starts).  This call
 * synchronizes `stream`, then sets *timed_out to 1 if the last solve that
 * used `work` gave up (its right-hand sides are then only partly solved) and
 * to 0 otherwise.  No counterpart in the paper.  Arguments: 1 work (the
 * workspace given to calu_getrs / caqr_geqrs), 2 timed_out (host), 3 stream.
 * Returns CA_OK, -1 / -2 for a NULL argument, CA_ERR_LAUNCH on a CUDA
 * error. */
int ca_solve_status(const void *work, int *timed_out, cudaStream_t stream);

/* ca_test_solve_hook: a test hook with no counterpart in the paper.  With
 * withhold = 1, the dependency-ordered triangular solves enqueued after this
 * call leave their first block's ready flag unset, so every wait on it runs
 * out after wait_cycles SM clock cycles (<= 0: the default, about 2 s) and
 * the timeout is recorded; withhold = 0 restores normal solves.  Host state
 * of the library, not thread-safe against solves being enqueued. */
void ca_test_solve_hook(long long wait_cycles, int withhold);

/* ------------------------------------------------------------------------ */
/* Reduced-precision trailing update on the tensor cores                    */
/* ------------------------------------------------------------------------ */

/* ca_gemm_minus_mixed: C -= A B, the dense contraction of the trailing update
 * (Sec. 3.2: A22 -= L21 U12), computed on the tcgen05 tensor cores.  A is
 * m x k, B is k x n, C is m x n, all FP64 column-major.  Each row of A and
 * each column of B is scaled by a power of two and cut, exactly, into
 * `slices` signed base-256 digits held in bf16; the digit products with
 * k + l <= slices + 1 are summed on the tensor cores in FP32 and applied to C
 * in FP64.
 *   exact = 0: one FP32 accumulator (digits pre-scaled); error about 2^-20
 *              relative to max|row of A| max|column of B| (slices >= 3);
 *   exact = 1: one accumulator per digit diagonal, each an exact FP32 sum of
 *              integers below 2^24 (needs k <= 128, slices <= 7); the only
 *              error is the dropped digits, about 2^(-8 slices) relative to
 *              the same scale (slices = 7: FP64-level).
 * Limits: 1 <= k <= 256, 1 <= slices <= 8.  dev_status (device int) gets a
 * bit (2, 4 or 8) if a bounded wait in the kernel timed out (the result is
 * then not applied).  Arguments: 1 m, 2 n, 3 k, 4 A, 5 lda, 6 B, 7 ldb, 8 C,
 * 9 ldc, 10 slices, 11 exact, 12 work, 13 lwork, 14 dev_status, 15 stream. */
int ca_gemm_mixed_workspace(int m, int n, int k, int slices, int exact, size_t *work_bytes);
int ca_gemm_minus_mixed(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                        double *C, int ldc, int slices, int exact, void *work, size_t lwork,
                        int *dev_status, cudaStream_t stream);

/* calu_factor_mixed: calu_factor with the Schur-complement update A22 -= L21
 * U12 on the tensor cores (ca_gemm_minus_mixed with `slices` digits and the
 * `exact` accumulation mode).  Tournament pivoting, the panel, L21 and U12
 * stay in FP64, so the pivots are chosen in FP64 on the reduced-precision
 * trailing matrix.  With exact = 1 and slices = 7 the update is FP64-accurate.
 * dev_info[1] also gets the kernel's timeout bits (2, 4, 8).  Arguments:
 * 1 m, 2 n, 3 A, 4 lda, 5 b, 6 tree, 7 slices, 8 exact, 9 ipiv, 10 work,
 * 11 lwork, 12 dev_info, 13 stream. */
int ca_calu_mixed_workspace(int m, int n, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *work_bytes);
int calu_factor_mixed(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int slices,
                      int exact, int *ipiv, void *work, size_t lwork, int *dev_info,
                      cudaStream_t stream);

/* caqr_factor_mixed: caqr_factor with the tree update of the trailing
 * columns (W = Y^T C, W = T^T W, C -= Y W for every leaf and merge node,
 * Sec. 3.1 UPFACT / UPELIM) on the tensor cores with `slices` digits and the
 * `exact` mode of ca_gemm_minus_mixed; TSQR (reflectors, norms, T) stays in
 * FP64.  Same outputs and storage as caqr_factor; with exact = 1 and
 * slices = 7 they agree with the FP64 form to FP64 rounding.  Arguments:
 * 1 m, 2 n, 3 A, 4 lda, 5 b, 6 tree, 7 slices, 8 exact, 9 qtree,
 * 10 qtree_bytes, 11 work, 12 lwork, 13 dev_info, 14 stream. */
int ca_caqr_mixed_workspace(int m, int n, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *qtree_bytes, size_t *work_bytes);
int caqr_factor_mixed(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int slices,
                      int exact, double *qtree, size_t qtree_bytes, void *work, size_t lwork,
                      int *dev_info, cudaStream_t stream);

/* calu_gesv_mixed: solve A X = B (n x n) by the mixed factorization plus
 * FP64 iterative refinement: LU <- A (copy in the caller's LU buffer),
 * calu_factor_mixed, X = U^-1 L^-1 P B, then repeat R = B - A X (FP64),
 * stop when the normwise backward error
 * max_j ||R_j||inf / (||A||inf ||X_j||inf + ||B_j||inf) <= tol, when it fails
 * to halve twice in a row, or after max_iter corrections.  The correction
 * (`refine`): CA_REFINE_CLASSIC X += (LU)^-1 R; CA_REFINE_GMRES X += D with
 * (M^-1 A) D = M^-1 R solved column by column by GMRES (FP64, at most 20
 * steps, until the preconditioned residual drops by 1e-6), M = P^T L U the
 * reduced-precision factors, which converges for matrices too ill
 * conditioned for the classic correction with the same digits; CA_REFINE_AUTO
 * three phases, each started only if the one before stopped above tol:
 * classic corrections while every step reduces the backward error at least
 * tenfold (up to max_iter); then up to 3 GMRES corrections, again while each
 * gains tenfold; then, when the
 * reduced-precision factors are too far from A for either to converge
 * (roughly cond(A) 2^(-8 slices) >= 1), A factored again with 7 exact digits
 * (FP64-accurate factors), X from those and up to 3 classic corrections, with
 * CA_STATUS_REFACTORED in dev_info[1] (dev_info[0] then describes the second
 * factorization, and ipiv / LU hold it).  The stop tests run on the device:
 * the whole procedure is enqueued and the call returns without waiting
 * (kernels of steps and phases that are not needed do nothing).
 * dev_iters (int) and dev_berr (double), device pointers or NULL, receive
 * the number of corrections and the final backward error.  dev_info[1] gets
 * CA_STATUS_SOLVE_TIMEOUT if a triangular solve gave up waiting, and the
 * tensor-core timeout bits.  Arguments: 1 n, 2 nrhs, 3 A, 4 lda, 5 b,
 * 6 tree, 7 slices, 8 exact, 9 refine, 10 LU, 11 ldlu, 12 ipiv, 13 B,
 * 14 ldb, 15 X, 16 ldx, 17 work, 18 lwork, 19 max_iter, 20 tol,
 * 21 dev_iters, 22 dev_berr, 23 dev_info, 24 stream. */
int ca_gesv_mixed_workspace(int n, int nrhs, int b, const ca_tree_t *tree, int slices, int exact, int refine,
                            size_t *work_bytes);
int calu_gesv_mixed(int n, int nrhs, const double *A, int lda, int b, const ca_tree_t *tree,
                    int slices, int exact, int refine, double *LU, int ldlu, int *ipiv, const double *B,
                    int ldb, double *X, int ldx, void *work, size_t lwork, int max_iter, double tol,
                    int *dev_iters, double *dev_berr, int *dev_info, cudaStream_t stream);

/* caqr_gels_mixed: least squares min ||A X - B|| (m x n, m >= n) by the
 * reduced-precision CAQR plus FP64 refinement: QR <- A (copy in the caller's
 * QR buffer), caqr_factor_mixed with `slices` digits and the `exact` mode
 * (TSQR in FP64, the tree update on the tensor cores), X = R^-1 (Q^T B)(0:n)
 * (as caqr_geqrs), then repeat R = B - A X (accumulated in double-double,
 * rounded once to FP64), S = A^T R in FP64 and X += R^-1 R^-T S
 * (refinement of the corrected semi-normal equations with the computed
 * triangular factor; its fixed point satisfies the least-squares condition
 * A^T (B - A X) = 0 to FP64 rounding, Sec. 3.1: A = QR), until the last
 * correction is below 4 unit roundoffs of X, fails to halve twice in a row,
 * or max_iter corrections.  Each step gains about a factor
 * cond(A) 2^(-8 slices); the stop test runs on the device and the call
 * returns without waiting.  The reported measure (dev_berr) is
 * max_j ||A^T R_j||inf / (||A||_1 (||A||inf ||X_j||inf + ||B_j||inf)) and tol
 * is its target (the least-squares solution of the FP64 problem has it at a
 * few unit roundoffs).
 * qtree receives the T factors as in caqr_factor.  dev_iters / dev_berr
 * (device, may be NULL): corrections and final value of the stop measure.
 * dev_info as calu_gesv_mixed.  Arguments: 1 m, 2 n, 3 nrhs, 4 A, 5 lda, 6 b,
 * 7 tree, 8 slices, 9 exact, 10 QR, 11 ldqr, 12 qtree, 13 qtree_bytes, 14 B,
 * 15 ldb, 16 X (n x nrhs), 17 ldx, 18 work, 19 lwork, 20 max_iter, 21 tol,
 * 22 dev_iters, 23 dev_berr, 24 dev_info, 25 stream. */
int ca_gels_mixed_workspace(int m, int n, int nrhs, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *qtree_bytes, size_t *work_bytes);
int caqr_gels_mixed(int m, int n, int nrhs, const double *A, int lda, int b, const ca_tree_t *tree, int slices,
                    int exact, double *QR, int ldqr, double *qtree, size_t qtree_bytes, const double *B, int ldb,
                    double *X, int ldx, void *work, size_t lwork, int max_iter, double tol, int *dev_iters,
                    double *dev_berr, int *dev_info, cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Batched factorizations: many small matrices of uneven shapes, each with   */
/* its own panel width and tree, in one persistent launch                    */
/* ------------------------------------------------------------------------ */

#define CA_BATCH_CALU 0
#define CA_BATCH_CAQR 1
#define CA_DTYPE_F64 0
#define CA_DTYPE_F32 1

/* One matrix of a batch.  All pointers are device pointers owned by the
 * caller; the element type (double or float) is the batch's dtype. */
typedef struct {
  int op;          /* CA_BATCH_CALU (calu_factor) or CA_BATCH_CAQR (caqr_factor) */
  int m, n, lda;   /* column-major m x n, lda >= max(1, m); CAQR needs m >= n   */
  void *A;         /* factored in place, same layout as calu_factor /           */
                   /* caqr_factor                                               */
  int *ipiv;       /* CALU: min(m, n) ints (1-based swap sequence)              */
  void *qtree;     /* CAQR: the T blocks, layout of caqr_factor in elements of  */
                   /* the batch's type (ca_caqr_workspace's qtree_bytes / 8     */
                   /* elements)                                                 */
  int *info;       /* 2 ints: [0] as calu_factor's dev_info[0] (first exactly   */
                   /* zero U diagonal), [1] CA_STATUS_NONFINITE                 */
  int b;           /* panel width, 1..128; at most 64 when n > b                */
  ca_tree_t tree;  /* leaf_rows >= min(b, min(m, n))                            */
} ca_batch_item_t;

/* ca_batched_plan: validates the batch and writes the launch plan (host
 * bytes: a header, then the items ordered by decreasing flop count, so the
 * largest start first).  plan == NULL: sizes only.  *plan_bytes: bytes of
 * the plan; *work_bytes: device workspace of ca_batched_factor.  The caller
 * copies the plan bytes to device memory of the same size (any 16-byte
 * aligned buffer) and keeps both copies until the factorization is done.
 * Each item's numerical result is the one calu_factor / caqr_factor give for
 * the same matrix, panel width and tree (Sec. 3.1 and 3.2), in the batch's
 * precision.  Errors: -1 count < 0, -2 items NULL, -3 dtype,
 * -5 / -6 size pointers NULL, CA_ERR_BATCH_ITEM for a malformed item,
 * CA_ERR_UNSUPPORTED for an item whose tree node (leaf_rows, or
 * fan-in x panel width rows) does not fit one CTA's shared memory. */
int ca_batched_plan(int count, const ca_batch_item_t *items, int dtype, void *plan, size_t *plan_bytes,
                    size_t *work_bytes);

/* ca_batched_factor: one persistent launch (one CTA per SM; each CTA takes
 * the next item from a device counter) that factors every item of the plan
 * on `stream`; plan_host and plan_dev hold the same bytes.  Nothing is
 * allocated and nothing waits on the host, so the call can be captured in a
 * CUDA graph (make one call before capturing).  Errors: -1 plan_host not a
 * plan, -2 plan_dev NULL, CA_ERR_WORKSPACE, CA_ERR_LAUNCH. */
int ca_batched_factor(const void *plan_host, const void *plan_dev, void *work, size_t lwork,
                      cudaStream_t stream);

/* ------------------------------------------------------------------------ */
/* Instrumentation (no counterpart in the paper): launch counts and device   */
/* time per kernel class, measured with CUDA events recorded on the stream   */
/* each kernel is launched on.  Classes: 0 tslu_node, 1 laswp, 2 lu_finish,  */
/* 3 trsm_u12, 4 gemm_fp64, 5 tsqr_node, 6 tree_apply, 7 solve,              */
/* 8 split_bf16, 9 gemm_tc, 10 refine, 11 batched, 12 tree_narrow (the      */
/* tree update of a few columns, or of too few column tiles to fill the GPU).*/
/* ------------------------------------------------------------------------ */

/* on = 1: create a pool of 2 * max_launches events (here, not during a
 * factorization) and start recording an event pair around every launch;
 * on = 0: stop.  Either way the recorded launches are cleared.  Launches
 * beyond the pool are counted but not timed (ca_prof_read then returns 1). */
int ca_prof_enable(int on, int max_launches);

/* Sum over the recorded launches of class `cls`: count, device time in ms
 * (waits for the recorded events) and algorithmic flops.  Host pointers;
 * any may be NULL.  Returns CA_OK, 1 if launches were dropped, -1 for a bad
 * class, CA_ERR_LAUNCH on a CUDA error. */
int ca_prof_read(int cls, long long *launches, double *ms, double *flops);

/* Kernel launches issued by the library since it was loaded: all classes
 * (cls < 0) or one class. */
long long ca_launch_count(int cls);

/* Name of a kernel class ("" when out of range). */
const char *ca_kernel_class_name(int cls);

/* ca_peak_probe: the FMA throughput of one precision on this GPU, the
 * measured denominator of the roofline fractions (no counterpart in the
 * paper).  Launches `blocks` CTAs of 256 threads; every thread does `iters`
 * rounds of 8 independent fused multiply-adds in FP64 (dtype CA_DTYPE_F64)
 * or FP32 (CA_DTYPE_F32) and writes one value to dev_out (blocks * 256
 * elements of that type, device).  The caller times it on `stream`; flops =
 * 16 * iters * blocks * 256.  Errors: -1 dtype, -2 blocks, -3 iters,
 * -4 dev_out NULL, CA_ERR_LAUNCH. */
int ca_peak_probe(int dtype, int blocks, int iters, void *dev_out, cudaStream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* CA_GB300_H */
