// api.cu -- the C-ABI: argument checks, the reduction-tree plan, workspace
// layout and the panel loops of CALU and CAQR (host side; every step runs in
// the kernels of panel_lu.cu, panel_qr.cu, gemm_fp64.cu and solve.cu).
#include <nvtx3/nvToolsExt.h>

#include <cstring>
#include <mutex>

#include "ca_internal.cuh"

namespace cagb {

// NVTX range around a host-side step (a panel of CALU / CAQR): visible in a
// timeline profiler, a null operation when none is attached.
struct NvtxRange {
  explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange &) = delete;
  NvtxRange &operator=(const NvtxRange &) = delete;
};

// Largest node tile (rows) of a panel: a leaf, or a merge of max_cnt sets.
static int max_node_rows(const Plan &p, int mk, int leaf_rows, int bk) {
  int r = leaf_rows < mk ? leaf_rows : mk;
  for (int i = 0; i < p.nrounds; ++i) {
    int m = p.r[i].max_cnt * bk;
    if (m > r) r = m;
  }
  return r;
}

bool lu_node_feasible(int rows, int bk);
bool qr_node_feasible(int rows, int bk);

}  // namespace cagb

using namespace cagb;

namespace {

constexpr int kMaxB = 128;

int check_tree(const ca_tree_t *t, int b) {
  if (!t) return 1;
  if (t->nlevels < 1 || t->nlevels > CA_MAX_LEVELS) return 1;
  if (t->leaf_rows < b || t->leaf_rows < 1) return 1;
  for (int l = 0; l < t->nlevels; ++l) {
    if (t->style[l] != CA_TREE_BINARY && t->style[l] != CA_TREE_FLAT) return 1;
    if (l < t->nlevels - 1 && t->fan_in[l] < 1) return 1;
  }
  return 0;
}

inline int nleaves_of(int mk, int L) { return (mk + L - 1) / L; }

// Shared checks of the LU shape; returns CA_OK or an error code.  The
// argument positions are those of calu_factor.
int lu_shape(int m, int n, int b, const ca_tree_t *tree, int *nl_max) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (b < 1) return -5;
  if (check_tree(tree, b)) return -6;
  if (tree->op_depth != 0 && !op_params_ok(*tree)) return -6;  // the 2D operator's levels
  int K = m < n ? m : n;
  *nl_max = 1;
  if (K == 0) return CA_OK;
  int bk = b < K ? b : K;
  if (bk > kMaxB) return CA_ERR_UNSUPPORTED;
  int nl = nleaves_of(m, tree->leaf_rows);
  Plan p;
  if (!build_plan(nl, *tree, p)) return CA_ERR_TREE;
  const int rows = max_node_rows(p, m, tree->leaf_rows, bk);
  if (tree->op_depth != 0 ? !op_node_feasible(rows, bk, *tree) : !lu_node_feasible(rows, bk))
    return CA_ERR_UNSUPPORTED;
  *nl_max = nl;
  return CA_OK;
}

// CALU panel workspace: the tournament buffers, then (2D operator) the
// operator's candidate buffers of every node of a round
size_t lu_ws_bytes(int nl, int bw, const ca_tree_t *tree) {
  return align256(lu_panel_ws_bytes(nl, bw)) + op_ws_bytes(nl, *tree);
}

int qr_shape(int m, int n, int b, const ca_tree_t *tree, int *nl_max, size_t *qbytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (b < 1) return -5;
  if (check_tree(tree, b)) return -6;
  if (tree->op_depth != 0) return CA_ERR_UNSUPPORTED;  // no pivoting in QR
  *nl_max = 1;
  *qbytes = 0;
  if (n == 0) return CA_OK;
  int bk = b < n ? b : n;
  if (bk > kMaxB) return CA_ERR_UNSUPPORTED;
  size_t q = 0;
  for (int kb = 0; kb < n; kb += b) {
    int mk = m - kb;
    int nl = nleaves_of(mk, tree->leaf_rows);
    Plan p;
    if (!build_plan(nl, *tree, p)) return CA_ERR_TREE;
    int bkk = (n - kb < b) ? n - kb : b;
    if (kb == 0) {
      if (!qr_node_feasible(max_node_rows(p, mk, tree->leaf_rows, bkk), bkk))
        return CA_ERR_UNSUPPORTED;
      *nl_max = nl;
    }
    q += (size_t)(nl + p.nmerges) * b * b * sizeof(double);
  }
  *qbytes = q;
  return CA_OK;
}

// Look-ahead: the next panel's factorization (TSLU / TSQR) runs on a helper
// stream of the highest priority as soon as the current update has reached
// its columns, while the rest of the update continues on the caller's
// stream.  One helper stream and two events per (device, caller stream),
// created on first use; they never hold memory of the caller.
struct Lookahead {
  int dev;
  cudaStream_t user, helper;
  cudaEvent_t ev_next, ev_panel;
};

Lookahead *lookahead_for(cudaStream_t user) {
  static std::mutex mu;
  static Lookahead pool[64];
  static int used = 0;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> g(mu);
  for (int i = 0; i < used; ++i)
    if (pool[i].dev == dev && pool[i].user == user) return &pool[i];
  if (used == 64) return nullptr;  // plain stream order beyond 64 caller streams
  Lookahead la;
  la.dev = dev;
  la.user = user;
  int least = 0, greatest = 0;
  if (cudaDeviceGetStreamPriorityRange(&least, &greatest) != cudaSuccess) return nullptr;
  if (cudaStreamCreateWithPriority(&la.helper, cudaStreamNonBlocking, greatest) != cudaSuccess) return nullptr;
  if (cudaEventCreateWithFlags(&la.ev_next, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  if (cudaEventCreateWithFlags(&la.ev_panel, cudaEventDisableTiming) != cudaSuccess) return nullptr;
  pool[used] = la;
  return &pool[used++];
}

// Panel loop of CALU (Algorithm "1D multilevel CALU" with one level): the
// trailing update runs in FP64 (tcws == nullptr) or on the tensor cores with
// `slices` digits (reduced precision, exact = per-diagonal accumulators).
int calu_run(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int *ipiv, void *work, int nl,
             void *tcws, int slices, int exact, int *dev_info, cudaStream_t stream, const int *skip = nullptr) {
  if (cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  const int K = m < n ? m : n;
  if (K == 0) return CA_OK;
  const int bw = b < kMaxB ? b : kMaxB;
  LuPanelWs ws;
  lu_panel_ws_carve(work, nl, bw, ws);
  int *opws = (int *)((char *)work + align256(lu_panel_ws_bytes(nl, bw)));
  const int L = tree->leaf_rows;
  Lookahead *la = (K > b) ? lookahead_for(stream) : nullptr;
  if (la && cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  auto update = [&](int mrows, int ncols, int kdim, const double *L21, const double *U12, double *C) -> cudaError_t {
    if (mrows <= 0 || ncols <= 0) return cudaSuccess;
    if (tcws)
      return gemm_minus_tc(mrows, ncols, kdim, L21, lda, U12, lda, C, lda, slices, exact, tcws, dev_info + 1, stream,
                           skip);
    return gemm_minus_f64(mrows, ncols, kdim, L21, lda, U12, lda, C, lda, stream, skip);
  };
  for (int kb = 0; kb < K; kb += b) {
    NvtxRange range("calu panel");
    const int bk = (K - kb < b) ? K - kb : b;
    const int mk = m - kb;
    Plan plan;
    if (!build_plan(nleaves_of(mk, L), *tree, plan)) return CA_ERR_TREE;
    double *P = A + kb + (size_t)kb * lda;
    cudaStream_t ps = la ? la->helper : stream;
    if (la && cudaStreamWaitEvent(ps, la->ev_next, 0) != cudaSuccess) return CA_ERR_LAUNCH;
    // 1. tournament pivoting over the tree (TSLU)
    const cudaError_t te = tree->op_depth != 0
                               ? tslu_panel_op(mk, bk, P, lda, *tree, plan, ws, opws, ipiv + kb, kb, dev_info, ps, skip)
                               : tslu_panel(mk, bk, P, lda, L, plan, ws, ipiv + kb, kb, dev_info, ps, skip);
    if (te != cudaSuccess) return CA_ERR_LAUNCH;
    if (la && (cudaEventRecord(la->ev_panel, ps) != cudaSuccess ||
               cudaStreamWaitEvent(stream, la->ev_panel, 0) != cudaSuccess))
      return CA_ERR_LAUNCH;
    // 2. swap rows at left and right of the panel
    if (laswp_apply(n, A, lda, kb, ws, bk, stream, skip) != cudaSuccess) return CA_ERR_LAUNCH;
    // 3. L11 \\ U11 into place, L21 = A21 U11^-1
    if (lu_panel_finish(mk, bk, P, lda, ws, stream, skip) != cudaSuccess) return CA_ERR_LAUNCH;
    const int nt = n - kb - bk;
    if (nt > 0) {
      double *A12 = A + kb + (size_t)(kb + bk) * lda;
      // 4. U12 = L11^-1 A12 and 5. A22 -= L21 U12: first the next panel's
      //    columns (the next tournament starts as soon as they are done),
      //    then the rest; every column's result is the same either way.  L11
      //    is read from its place in A: the workspace copy belongs to the
      //    next panel's tournament once it has started.
      const int nnext = (kb + bk < K) ? ((K - kb - bk < b) ? K - kb - bk : b) : 0;
      if (la && nnext > 0 && nnext < nt) {
        if (trsm_u12(bk, nnext, P, lda, A12, lda, stream, skip) != cudaSuccess) return CA_ERR_LAUNCH;
        if (update(mk - bk, nnext, bk, P + bk, A12, A12 + bk) != cudaSuccess) return CA_ERR_LAUNCH;
        if (cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
        double *A12r = A12 + (size_t)nnext * lda;
        if (trsm_u12(bk, nt - nnext, P, lda, A12r, lda, stream, skip) != cudaSuccess) return CA_ERR_LAUNCH;
        if (update(mk - bk, nt - nnext, bk, P + bk, A12r, A12r + bk) != cudaSuccess) return CA_ERR_LAUNCH;
      } else {
        if (trsm_u12(bk, nt, P, lda, A12, lda, stream, skip) != cudaSuccess) return CA_ERR_LAUNCH;
        if (update(mk - bk, nt, bk, P + bk, A12, A12 + bk) != cudaSuccess) return CA_ERR_LAUNCH;
        if (la && cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      }
    }
  }
  return CA_OK;
}

// Panel loop of CAQR (Algorithm ML-CAQR with one level): TSQR, then the tree
// update of the trailing columns in FP64 (tcws == nullptr) or on the tensor
// cores.  With look-ahead the per-node arrays alternate between two copies.
int caqr_run(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, double *qtree, void *work, int nl,
             void *tcws, int slices, int exact, int *dev_info, cudaStream_t stream) {
  if (cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (n == 0) return CA_OK;
  QrPanelWs wsv[2];
  qr_panel_ws_carve(work, nl, wsv[0]);
  qr_panel_ws_carve((char *)work + align256(qr_panel_ws_bytes(nl)), nl, wsv[1]);
  const int L = tree->leaf_rows;
  Lookahead *la = (n > b) ? lookahead_for(stream) : nullptr;
  if (la && cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  size_t off = 0;
  for (int kb = 0, k = 0; kb < n; kb += b, ++k) {
    NvtxRange range("caqr panel");
    const int bk = (n - kb < b) ? n - kb : b;
    const int mk = m - kb;
    Plan plan;
    if (!build_plan(nleaves_of(mk, L), *tree, plan)) return CA_ERR_TREE;
    double *P = A + kb + (size_t)kb * lda;
    double *Tp = qtree + off;
    const QrPanelWs &ws = wsv[k & 1];
    cudaStream_t ps = la ? la->helper : stream;
    if (la && cudaStreamWaitEvent(ps, la->ev_next, 0) != cudaSuccess) return CA_ERR_LAUNCH;
    // 1. TSQR: leaves, then the R-elimination tree
    if (tsqr_panel(mk, bk, b, P, lda, L, plan, Tp, ws, dev_info, ps) != cudaSuccess) return CA_ERR_LAUNCH;
    if (la && (cudaEventRecord(la->ev_panel, ps) != cudaSuccess ||
               cudaStreamWaitEvent(stream, la->ev_panel, 0) != cudaSuccess))
      return CA_ERR_LAUNCH;
    // 2. trailing columns: leaves' Q^T (UPFACT), then merges' Q^T (UPELIM);
    //    the next panel's columns first
    const int nt = n - kb - bk;
    auto apply = [&](double *C, int ncols) -> cudaError_t {
      if (ncols <= 0) return cudaSuccess;
      if (tcws)
        return tree_apply_qt_tc(mk, bk, b, P, lda, L, plan, Tp, C, lda, ncols, ws, tcws, slices, exact,
                                dev_info + 1, stream);
      return tree_apply_qt(mk, bk, b, P, lda, L, plan, Tp, C, lda, ncols, ws, stream);
    };
    if (nt > 0) {
      const int nnext = nt < b ? nt : b;
      if (la && nnext < nt) {
        if (apply(P + (size_t)bk * lda, nnext) != cudaSuccess) return CA_ERR_LAUNCH;
        if (cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
        if (apply(P + (size_t)(bk + nnext) * lda, nt - nnext) != cudaSuccess) return CA_ERR_LAUNCH;
      } else {
        if (apply(P + (size_t)bk * lda, nt) != cudaSuccess) return CA_ERR_LAUNCH;
        if (la && cudaEventRecord(la->ev_next, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      }
    }
    off += (size_t)(plan.nleaves + plan.nmerges) * b * b;
  }
  return CA_OK;
}

// P A = L U solve on `stream`: swaps, unit-lower and upper substitution.
// Given-up waits of the dependency-ordered solves go to status |= bit.
cudaError_t getrs_run(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb,
                      const SolveWs &sw, int *status, int bit, const int *skip, cudaStream_t stream) {
  cudaError_t e = getrs_swap(n, nrhs, ipiv, B, ldb, stream, skip);
  if (e != cudaSuccess) return e;
  if ((e = trsm_left(true, true, n, nrhs, LU, lda, B, ldb, sw, status, bit, skip, stream)) != cudaSuccess) return e;
  return trsm_left(false, false, n, nrhs, LU, lda, B, ldb, sw, status, bit, skip, stream);
}

size_t caqr_mixed_ws(int m, int n, int b, const ca_tree_t *tree, int nl, int slices) {
  const int bk = b < n ? b : n;
  return 2 * align256(qr_panel_ws_bytes(nl)) +
         tree_tc_ws_bytes(m, bk, n - bk > 0 ? n - bk : 1, tree->leaf_rows, nl, slices);
}

size_t calu_mixed_ws(int m, int n, int b, const ca_tree_t *tree, int nl, int slices) {
  const int bw = b < kMaxB ? b : kMaxB;
  return align256(lu_ws_bytes(nl, bw, tree)) + tc_gemm_ws_bytes(m, n, bw, slices);
}

}  // namespace

extern "C" {

const char *ca_strerror(int code) {
  switch (code) {
    case CA_OK:
      return "success";
    case CA_ERR_WORKSPACE:
      return "workspace pointer is null or smaller than the workspace query";
    case CA_ERR_UNSUPPORTED:
      return "shape not supported by the library (panel width > 128 or a tree node too large)";
    case CA_ERR_LAUNCH:
      return "a CUDA kernel launch failed";
    case CA_ERR_TREE:
      return "malformed reduction tree";
    case CA_ERR_BATCH_ITEM:
      return "an item of the batch is invalid (op, shape, lda, panel width, tree or a null pointer)";
    default:
      break;
  }
  if (code < 0 && code > -100) return "invalid argument (the negated return value is its position)";
  return "unknown error";
}

int ca_calu_workspace(int m, int n, int b, const ca_tree_t *tree, size_t *work_bytes) {
  if (!work_bytes) return -5;
  int nl;
  int rc = lu_shape(m, n, b, tree, &nl);
  if (rc == -5 || rc == -6) rc = (rc == -5) ? -3 : -4;  // positions in this call
  if (rc != CA_OK) return rc;
  *work_bytes = lu_ws_bytes(nl, b < kMaxB ? b : kMaxB, tree);
  return CA_OK;
}

int ca_caqr_workspace(int m, int n, int b, const ca_tree_t *tree, size_t *qtree_bytes,
                      size_t *work_bytes) {
  if (!qtree_bytes) return -5;
  if (!work_bytes) return -6;
  int nl;
  size_t q;
  int rc = qr_shape(m, n, b, tree, &nl, &q);
  if (rc == -5 || rc == -6) rc = (rc == -5) ? -3 : -4;
  if (rc != CA_OK) return rc;
  *qtree_bytes = q;
  *work_bytes = 2 * align256(qr_panel_ws_bytes(nl));  // two copies for look-ahead
  return CA_OK;
}

int ca_geqrs_workspace(int m, int n, int nrhs, int b, const ca_tree_t *tree, size_t *work_bytes) {
  if (!work_bytes) return -6;
  if (nrhs < 0) return -3;
  int nl;
  size_t q;
  int rc = qr_shape(m, n, b, tree, &nl, &q);
  if (rc == -5 || rc == -6) rc = (rc == -5) ? -4 : -5;
  if (rc != CA_OK) return rc;
  *work_bytes = align256(solve_ws_bytes(n)) + qr_panel_ws_bytes(nl);
  return CA_OK;
}

int ca_getrs_workspace(int n, int nrhs, size_t *work_bytes) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (!work_bytes) return -3;
  *work_bytes = solve_ws_bytes(n);
  return CA_OK;
}

int calu_factor(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int *ipiv,
                void *work, size_t lwork, int *dev_info, cudaStream_t stream) {
  int nl;
  int rc = lu_shape(m, n, b, tree, &nl);
  if (rc != CA_OK) return rc;
  if (lda < (m > 1 ? m : 1)) return -4;
  const int K = m < n ? m : n;
  if (K > 0 && !A) return -3;
  if (K > 0 && !ipiv) return -7;
  if (!dev_info) return -10;
  const int bw = b < kMaxB ? b : kMaxB;
  if (K > 0 && (!work || lwork < lu_ws_bytes(nl, bw, tree))) return CA_ERR_WORKSPACE;
  return calu_run(m, n, A, lda, b, tree, ipiv, work, nl, nullptr, 0, 0, dev_info, stream);
}

int tslu(int m, int n, double *A, int lda, const ca_tree_t *tree, int *ipiv, void *work,
         size_t lwork, int *dev_info, cudaStream_t stream) {
  if (n < 0) return -2;
  int rc = calu_factor(m, n, A, lda, n > 0 ? n : 1, tree, ipiv, work, lwork, dev_info, stream);
  // calu_factor numbers its arguments 1..11; map b (5) and later onto this call
  if (rc == -5 || rc == -6) return -5;
  if (rc == -7) return -6;
  if (rc == -10) return -9;
  return rc;
}

int calu_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb, void *work,
               size_t lwork, cudaStream_t stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !LU) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (n > 0 && !ipiv) return -5;
  if (n > 0 && nrhs > 0 && !B) return -6;
  if (ldb < (n > 1 ? n : 1)) return -7;
  if (n == 0 || nrhs == 0) return CA_OK;
  if (!work || lwork < solve_ws_bytes(n)) return CA_ERR_WORKSPACE;
  SolveWs sw;
  solve_ws_carve(work, n, sw);
  if (cudaMemsetAsync(sw.status, 0, sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (getrs_run(n, nrhs, LU, lda, ipiv, B, ldb, sw, sw.status, 1, nullptr, stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  return CA_OK;
}

int caqr_factor(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, double *qtree,
                size_t qtree_bytes, void *work, size_t lwork, int *dev_info, cudaStream_t stream) {
  int nl;
  size_t qneed;
  int rc = qr_shape(m, n, b, tree, &nl, &qneed);
  if (rc != CA_OK) return rc;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (n > 0 && !A) return -3;
  if (!dev_info) return -11;
  if (n > 0 && (!qtree || qtree_bytes < qneed)) return CA_ERR_WORKSPACE;
  if (n > 0 && (!work || lwork < 2 * align256(qr_panel_ws_bytes(nl)))) return CA_ERR_WORKSPACE;
  return caqr_run(m, n, A, lda, b, tree, qtree, work, nl, nullptr, 0, 0, dev_info, stream);
}

int tsqr(int m, int n, double *A, int lda, const ca_tree_t *tree, double *qtree,
         size_t qtree_bytes, void *work, size_t lwork, int *dev_info, cudaStream_t stream) {
  if (n < 0) return -2;
  int rc = caqr_factor(m, n, A, lda, n > 0 ? n : 1, tree, qtree, qtree_bytes, work, lwork, dev_info,
                       stream);
  if (rc == -5 || rc == -6) return -5;
  if (rc == -11) return -10;
  return rc;
}

int caqr_geqrs(int m, int n, int nrhs, const double *QR, int lda, int b, const ca_tree_t *tree,
               const double *qtree, size_t qtree_bytes, double *B, int ldb, void *work,
               size_t lwork, cudaStream_t stream) {
  if (nrhs < 0) return -3;
  int nl;
  size_t qneed;
  int rc = qr_shape(m, n, b, tree, &nl, &qneed);
  if (rc == -1 || rc == -2) return rc;
  if (rc == -5) return -6;
  if (rc == -6) return -7;
  if (rc != CA_OK) return rc;
  if (n > 0 && !QR) return -4;
  if (lda < (m > 1 ? m : 1)) return -5;
  if (ldb < (m > 1 ? m : 1)) return -11;
  if (n == 0 || nrhs == 0) return CA_OK;
  if (!B) return -10;
  if (!qtree || qtree_bytes < qneed) return CA_ERR_WORKSPACE;
  const size_t swb = align256(solve_ws_bytes(n));
  if (!work || lwork < swb + qr_panel_ws_bytes(nl)) return CA_ERR_WORKSPACE;
  SolveWs sw;
  solve_ws_carve(work, n, sw);
  if (cudaMemsetAsync(sw.status, 0, sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  QrPanelWs ws;
  qr_panel_ws_carve((char *)work + swb, nl, ws);
  const int L = tree->leaf_rows;
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    const int bk = (n - kb < b) ? n - kb : b;
    const int mk = m - kb;
    Plan plan;
    if (!build_plan(nleaves_of(mk, L), *tree, plan)) return CA_ERR_TREE;
    if (tree_apply_qt(mk, bk, b, QR + kb + (size_t)kb * lda, lda, L, plan, qtree + off, B + kb, ldb,
                      nrhs, ws, stream) != cudaSuccess)
      return CA_ERR_LAUNCH;
    off += (size_t)(plan.nleaves + plan.nmerges) * b * b;
  }
  if (trsm_left(false, false, n, nrhs, QR, lda, B, ldb, sw, sw.status, 1, nullptr, stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  return CA_OK;
}

int ca_solve_status(const void *work, int *timed_out, cudaStream_t stream) {
  if (!work) return -1;
  if (!timed_out) return -2;
  if (cudaStreamSynchronize(stream) != cudaSuccess) return CA_ERR_LAUNCH;
  int word = 0;
  if (cudaMemcpy(&word, work, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess) return CA_ERR_LAUNCH;
  *timed_out = word != 0;
  return CA_OK;
}

void ca_test_solve_hook(long long wait_cycles, int withhold) { solve_test_hook(wait_cycles, withhold ? 0 : -1); }

int ca_gemm_mixed_workspace(int m, int n, int k, int slices, int exact, size_t *work_bytes) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (k < 0) return -3;
  if (slices < 1 || slices > 8) return -4;
  if (!tc_gemm_supported(k > 0 ? k : 1, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (!work_bytes) return -6;
  *work_bytes = tc_gemm_ws_bytes(m, n, k, slices);
  return CA_OK;
}

int ca_gemm_minus_mixed(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                        double *C, int ldc, int slices, int exact, void *work, size_t lwork,
                        int *dev_status, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  if (k < 0) return -3;
  if (m > 0 && k > 0 && !A) return -4;
  if (lda < (m > 1 ? m : 1)) return -5;
  if (k > 0 && n > 0 && !B) return -6;
  if (ldb < (k > 1 ? k : 1)) return -7;
  if (m > 0 && n > 0 && !C) return -8;
  if (ldc < (m > 1 ? m : 1)) return -9;
  if (slices < 1 || slices > 8) return -10;
  if (m == 0 || n == 0 || k == 0) return CA_OK;
  if (!tc_gemm_supported(k, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (!work || lwork < tc_gemm_ws_bytes(m, n, k, slices)) return CA_ERR_WORKSPACE;
  if (!dev_status) return -14;
  if (gemm_minus_tc(m, n, k, A, lda, B, ldb, C, ldc, slices, exact, work, dev_status, stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  return CA_OK;
}

int ca_calu_mixed_workspace(int m, int n, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *work_bytes) {
  int nl;
  int rc = lu_shape(m, n, b, tree, &nl);
  if (rc == -5 || rc == -6) rc = (rc == -5) ? -3 : -4;
  if (rc != CA_OK) return rc;
  if (slices < 1 || slices > 8) return -5;
  if (!tc_gemm_supported(b < kMaxB ? b : kMaxB, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (!work_bytes) return -7;
  *work_bytes = calu_mixed_ws(m, n, b, tree, nl, slices);
  return CA_OK;
}

int calu_factor_mixed(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int slices, int exact,
                      int *ipiv, void *work, size_t lwork, int *dev_info, cudaStream_t stream) {
  int nl;
  int rc = lu_shape(m, n, b, tree, &nl);
  if (rc != CA_OK) return rc;
  if (lda < (m > 1 ? m : 1)) return -4;
  const int K = m < n ? m : n;
  if (K > 0 && !A) return -3;
  if (slices < 1 || slices > 8) return -7;
  if (!tc_gemm_supported(b < kMaxB ? b : kMaxB, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (K > 0 && !ipiv) return -9;
  if (!dev_info) return -12;
  const size_t need = calu_mixed_ws(m, n, b, tree, nl, slices);
  if (K > 0 && (!work || lwork < need)) return CA_ERR_WORKSPACE;
  const int bw = b < kMaxB ? b : kMaxB;
  char *tcws = (char *)work + align256(lu_ws_bytes(nl, bw, tree));
  return calu_run(m, n, A, lda, b, tree, ipiv, work, nl, tcws, slices, exact, dev_info, stream);
}

int ca_gesv_mixed_workspace(int n, int nrhs, int b, const ca_tree_t *tree, int slices, int exact, int refine,
                            size_t *work_bytes) {
  if (nrhs < 0) return -2;
  size_t w = 0;
  int rc = ca_calu_mixed_workspace(n, n, b, tree, slices, exact, &w);
  if (rc == -1 || rc == -2) return -1;
  if (rc != CA_OK) return rc;  // b, tree, slices are arguments 3, 4, 5 in both calls
  if (refine < CA_REFINE_CLASSIC || refine > CA_REFINE_AUTO) return -7;
  if (!work_bytes) return -8;
  if (refine == CA_REFINE_AUTO) {  // room for the fallback factorization with 7 exact digits
    size_t w7 = 0;
    if (ca_calu_mixed_workspace(n, n, b, tree, 7, 1, &w7) == CA_OK && w7 > w) w = w7;
  }
  *work_bytes = align256(w) + align256(ir_ws_bytes(n, nrhs > 0 ? nrhs : 1)) + align256(solve_ws_bytes(n)) +
                (refine != CA_REFINE_CLASSIC ? gm_ws_bytes(n) : 0);
  return CA_OK;
}

int calu_gesv_mixed(int n, int nrhs, const double *A, int lda, int b, const ca_tree_t *tree, int slices,
                    int exact, int refine, double *LU, int ldlu, int *ipiv, const double *B, int ldb, double *X,
                    int ldx, void *work, size_t lwork, int max_iter, double tol, int *dev_iters,
                    double *dev_berr, int *dev_info, cudaStream_t stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !A) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (b < 1) return -5;
  if (check_tree(tree, b)) return -6;
  if (slices < 1 || slices > 8) return -7;
  if (refine < CA_REFINE_CLASSIC || refine > CA_REFINE_AUTO) return -9;
  if (n > 0 && !LU) return -10;
  if (ldlu < (n > 1 ? n : 1)) return -11;
  if (n > 0 && !ipiv) return -12;
  if (n > 0 && nrhs > 0 && !B) return -13;
  if (ldb < (n > 1 ? n : 1)) return -14;
  if (n > 0 && nrhs > 0 && !X) return -15;
  if (ldx < (n > 1 ? n : 1)) return -16;
  if (max_iter < 0) return -19;
  if (!dev_info) return -23;
  size_t need = 0;
  int rc = ca_gesv_mixed_workspace(n, nrhs, b, tree, slices, exact, refine, &need);
  if (rc == -7) return -9;
  if (rc != CA_OK) return rc;
  if (n > 0 && (!work || lwork < need)) return CA_ERR_WORKSPACE;
  if (dev_iters && cudaMemsetAsync(dev_iters, 0, sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (dev_berr && cudaMemsetAsync(dev_berr, 0, sizeof(double), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (n == 0) return cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) == cudaSuccess ? CA_OK : CA_ERR_LAUNCH;
  size_t wf = 0, w7 = 0;
  ca_calu_mixed_workspace(n, n, b, tree, slices, exact, &wf);
  const size_t wfact = wf;  // the first factorization's part
  if (refine == CA_REFINE_AUTO && ca_calu_mixed_workspace(n, n, b, tree, 7, 1, &w7) == CA_OK && w7 > wf) wf = w7;
  const int nr = nrhs > 0 ? nrhs : 1;
  char *p = (char *)work + align256(wf);
  IrWs iw;
  ir_ws_carve(p, n, nr, iw);
  p += align256(ir_ws_bytes(n, nr));
  SolveWs sw;
  solve_ws_carve(p, n, sw);
  p += align256(solve_ws_bytes(n));
  GmWs gw{};
  if (refine != CA_REFINE_CLASSIC) gm_ws_carve(p, n, gw);
  int *status = dev_info + 1;  // given-up waits of the solves: CA_STATUS_SOLVE_TIMEOUT
  const int sbit = CA_STATUS_SOLVE_TIMEOUT;
  // 1. LU <- A, reduced-precision factorization (FP64 panels and pivots)
  if (cudaMemcpy2DAsync(LU, (size_t)ldlu * 8, A, (size_t)lda * 8, (size_t)n * 8, n, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  rc = calu_factor_mixed(n, n, LU, ldlu, b, tree, slices, exact, ipiv, work, wfact, dev_info, stream);
  if (rc != CA_OK) return rc;
  if (nrhs == 0) return CA_OK;
  // 2. X = (LU)^-1 B
  if (cudaMemcpy2DAsync(X, (size_t)ldx * 8, B, (size_t)ldb * 8, (size_t)n * 8, nrhs, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  if (getrs_run(n, nrhs, LU, ldlu, ipiv, X, ldx, sw, status, sbit, nullptr, stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  if (ir_anorm(n, A, lda, iw, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  // 3. refinement phases, enqueued in full; each step: R = B - A X in FP64,
  //    the stop test on the device, then the correction (one solve with the
  //    factors, or GMRES preconditioned by them).  The kernels of steps after
  //    a phase's stop do nothing.
  auto run_phase = [&](const IrWs &w, bool gmres, int steps) -> int {
    for (int it = 0;; ++it) {
      if (ir_residual(n, nrhs, A, lda, X, ldx, B, ldb, w, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      if (ir_berr(n, nrhs, X, ldx, B, ldb, w, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      if (ir_decide(it, steps, tol, nrhs, w, dev_berr, dev_iters, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      if (it >= steps) break;
      if (!gmres) {
        if (getrs_run(n, nrhs, LU, ldlu, ipiv, w.R, n, sw, status, sbit, &w.ctl->done, stream) != cudaSuccess)
          return CA_ERR_LAUNCH;
        if (ir_update(n, nrhs, w, X, ldx, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      } else {
        for (int j = 0; j < nrhs; ++j)
          if (ir_gmres_correction(n, A, lda, LU, ldlu, ipiv, w, gw, j, X, ldx, sw, status, sbit, stream) !=
              cudaSuccess)
            return CA_ERR_LAUNCH;
      }
    }
    return CA_OK;
  };
  constexpr double kNever = 1e308;     // no slow-step rule: stop after two non-halving steps
  constexpr double kSlowAuto = 0.1;    // AUTO: a classic step gaining less than 10x hands over to GMRES
  constexpr int kAutoGmresSteps = 3;   // AUTO: GMRES corrections before the refactorization
  constexpr int kAutoRefactorSteps = 3;
  IrWs ph[kIrPhases];
  for (int i = 0; i < kIrPhases; ++i) {
    ph[i] = iw;
    ph[i].ctl = iw.phase[i];
  }
  if (refine != CA_REFINE_AUTO) {
    if (ir_begin(ph[0], kNever, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    return run_phase(ph[0], refine == CA_REFINE_GMRES, max_iter);
  }
  // AUTO: classic corrections while each gains 10x or more
  if (ir_begin(ph[0], kSlowAuto, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if ((rc = run_phase(ph[0], false, max_iter)) != CA_OK) return rc;
  // then GMRES corrections, if the classic phase stopped above tol, while
  // each gains 10x (a GMRES correction that does not is a sign that the
  // factors are too far from A: the refactorization follows at once)
  if (ir_begin_next(ph[0].ctl, ph[1], kSlowAuto, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if ((rc = run_phase(ph[1], true, kAutoGmresSteps)) != CA_OK) return rc;
  // then, if GMRES stopped above tol too (the reduced-precision factors are
  // too far from A), A factored again with 7 exact digits (FP64-accurate
  // update), X from those factors, classic corrections
  if (ir_begin_next(ph[1].ctl, ph[2], kNever, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  const int *noref = &ph[2].ctl->done;  // set: the phase does not run
  int nl = 1;
  if (lu_shape(n, n, b, tree, &nl) != CA_OK) return CA_ERR_UNSUPPORTED;
  const int bw = b < kMaxB ? b : kMaxB;
  char *tcws = (char *)work + align256(lu_ws_bytes(nl, bw, tree));
  if (copy_matrix(n, n, A, lda, LU, ldlu, noref, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if ((rc = calu_run(n, n, LU, ldlu, b, tree, ipiv, work, nl, tcws, 7, 1, iw.info2, stream, noref)) != CA_OK)
    return rc;
  if (copy_matrix(n, nrhs, B, ldb, X, ldx, noref, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (getrs_run(n, nrhs, LU, ldlu, ipiv, X, ldx, sw, status, sbit, noref, stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  if ((rc = run_phase(ph[2], false, kAutoRefactorSteps)) != CA_OK) return rc;
  return ir_merge_info(ph[2], iw.info2, dev_info, stream) == cudaSuccess ? CA_OK : CA_ERR_LAUNCH;
}

int ca_caqr_mixed_workspace(int m, int n, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *qtree_bytes, size_t *work_bytes) {
  int nl;
  size_t q;
  int rc = qr_shape(m, n, b, tree, &nl, &q);
  if (rc == -5 || rc == -6) rc = (rc == -5) ? -3 : -4;
  if (rc != CA_OK) return rc;
  if (slices < 1 || slices > 8) return -5;
  if (!tc_gemm_supported(b < kMaxB ? b : kMaxB, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (!qtree_bytes) return -7;
  if (!work_bytes) return -8;
  *qtree_bytes = q;
  *work_bytes = n > 0 ? caqr_mixed_ws(m, n, b, tree, nl, slices) : 256;
  return CA_OK;
}

int caqr_factor_mixed(int m, int n, double *A, int lda, int b, const ca_tree_t *tree, int slices, int exact,
                      double *qtree, size_t qtree_bytes, void *work, size_t lwork, int *dev_info,
                      cudaStream_t stream) {
  int nl;
  size_t qneed;
  int rc = qr_shape(m, n, b, tree, &nl, &qneed);
  if (rc != CA_OK) return rc;
  if (lda < (m > 1 ? m : 1)) return -4;
  if (n > 0 && !A) return -3;
  if (slices < 1 || slices > 8) return -7;
  if (!tc_gemm_supported(b < kMaxB ? b : kMaxB, slices, exact)) return CA_ERR_UNSUPPORTED;
  if (!dev_info) return -13;
  if (n > 0 && (!qtree || qtree_bytes < qneed)) return CA_ERR_WORKSPACE;
  if (n > 0 && (!work || lwork < caqr_mixed_ws(m, n, b, tree, nl, slices))) return CA_ERR_WORKSPACE;
  char *tcws = n > 0 ? (char *)work + 2 * align256(qr_panel_ws_bytes(nl)) : nullptr;
  return caqr_run(m, n, A, lda, b, tree, qtree, work, nl, tcws, slices, exact, dev_info, stream);
}

int ca_gels_mixed_workspace(int m, int n, int nrhs, int b, const ca_tree_t *tree, int slices, int exact,
                            size_t *qtree_bytes, size_t *work_bytes) {
  if (nrhs < 0) return -3;
  size_t q = 0, wf = 0, wg = 0;
  int rc = ca_caqr_mixed_workspace(m, n, b, tree, slices, exact, &q, &wf);
  if (rc == -1 || rc == -2) return rc;
  if (rc == -3 || rc == -4) return rc - 1;  // b, tree are arguments 4, 5 here
  if (rc == -5) return -6;
  if (rc != CA_OK) return rc;
  rc = ca_geqrs_workspace(m, n, nrhs > 0 ? nrhs : 1, b, tree, &wg);
  if (rc != CA_OK) return rc;
  if (!qtree_bytes) return -8;
  if (!work_bytes) return -9;
  const int nr = nrhs > 0 ? nrhs : 1;
  *qtree_bytes = q;
  *work_bytes = align256(wf) + align256(wg) + align256((size_t)m * nr * 8) + align256(solve_ws_bytes(n)) +
                ls_ws_bytes(m, n, nr);
  return CA_OK;
}

int caqr_gels_mixed(int m, int n, int nrhs, const double *A, int lda, int b, const ca_tree_t *tree, int slices,
                    int exact, double *QR, int ldqr, double *qtree, size_t qtree_bytes, const double *B, int ldb,
                    double *X, int ldx, void *work, size_t lwork, int max_iter, double tol, int *dev_iters,
                    double *dev_berr, int *dev_info, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (nrhs < 0) return -3;
  if (n > 0 && !A) return -4;
  if (lda < (m > 1 ? m : 1)) return -5;
  if (b < 1) return -6;
  if (check_tree(tree, b)) return -7;
  if (slices < 1 || slices > 8) return -8;
  if (n > 0 && !QR) return -10;
  if (ldqr < (m > 1 ? m : 1)) return -11;
  if (n > 0 && nrhs > 0 && !B) return -14;
  if (ldb < (m > 1 ? m : 1)) return -15;
  if (n > 0 && nrhs > 0 && !X) return -16;
  if (ldx < (n > 1 ? n : 1)) return -17;
  if (max_iter < 0) return -20;
  if (!dev_info) return -24;
  size_t qneed = 0, need = 0;
  int rc = ca_gels_mixed_workspace(m, n, nrhs, b, tree, slices, exact, &qneed, &need);
  if (rc != CA_OK) return rc;
  if (n > 0 && (!qtree || qtree_bytes < qneed)) return CA_ERR_WORKSPACE;
  if (n > 0 && (!work || lwork < need)) return CA_ERR_WORKSPACE;
  if (dev_iters && cudaMemsetAsync(dev_iters, 0, sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (dev_berr && cudaMemsetAsync(dev_berr, 0, sizeof(double), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (n == 0) return cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) == cudaSuccess ? CA_OK : CA_ERR_LAUNCH;
  size_t qb = 0, wf = 0, wg = 0;
  ca_caqr_mixed_workspace(m, n, b, tree, slices, exact, &qb, &wf);
  const int nr = nrhs > 0 ? nrhs : 1;
  ca_geqrs_workspace(m, n, nr, b, tree, &wg);
  char *p = (char *)work;
  void *wfact = p;
  p += align256(wf);
  void *wgeq = p;
  p += align256(wg);
  double *W = (double *)p;  // m x nrhs: Q^T B
  p += align256((size_t)m * nr * 8);
  SolveWs sw;
  solve_ws_carve(p, n, sw);
  p += align256(solve_ws_bytes(n));
  LsWs lw;
  ls_ws_carve(p, m, n, nr, lw);
  int *status = dev_info + 1;
  const int sbit = CA_STATUS_SOLVE_TIMEOUT;
  // 1. QR <- A, CAQR with the tree update on the tensor cores (TSQR in FP64)
  if (cudaMemcpy2DAsync(QR, (size_t)ldqr * 8, A, (size_t)lda * 8, (size_t)m * 8, n, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  rc = caqr_factor_mixed(m, n, QR, ldqr, b, tree, slices, exact, qtree, qtree_bytes, wfact, wf, dev_info, stream);
  if (rc != CA_OK) return rc;
  if (nrhs == 0) return CA_OK;
  // 2. X = R^-1 (Q^T B)(0:n) with the reduced-precision factors
  if (cudaMemcpy2DAsync(W, (size_t)m * 8, B, (size_t)ldb * 8, (size_t)m * 8, nrhs, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  rc = caqr_geqrs(m, n, nrhs, QR, ldqr, b, tree, qtree, qtree_bytes, W, m, wgeq, wg, stream);
  if (rc != CA_OK) return rc;
  if (cudaMemcpy2DAsync(X, (size_t)ldx * 8, W, (size_t)m * 8, (size_t)n * 8, nrhs, cudaMemcpyDeviceToDevice,
                        stream) != cudaSuccess)
    return CA_ERR_LAUNCH;
  // 3. refinement on the corrected semi-normal equations, enqueued in full:
  //    R = B - A X and S = A^T R in FP64, the stop test on the device, then
  //    X += R^-1 R^-T S with the triangular factor
  if (ls_norms(m, n, A, lda, lw, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (ls_transpose_r(n, QR, ldqr, lw, nullptr, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (ls_begin(lw, nullptr, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  const int *stop = &lw.ctl->done;
  for (int it = 0;; ++it) {
    if (ls_residual(m, n, nrhs, A, lda, X, ldx, B, ldb, lw, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    if (ls_normal_residual(m, n, nrhs, A, lda, X, ldx, B, ldb, lw, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    if (ls_decide(it, max_iter, tol, nrhs, lw, dev_berr, dev_iters, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    if (it >= max_iter) break;
    if (trsm_left(true, false, n, nrhs, lw.Rt, n, lw.S, n, sw, status, sbit, stop, stream) != cudaSuccess ||
        trsm_left(false, false, n, nrhs, QR, ldqr, lw.S, n, sw, status, sbit, stop, stream) != cudaSuccess)
      return CA_ERR_LAUNCH;
    if (ls_update(n, nrhs, lw, X, ldx, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  }
  return CA_OK;
}

}  // extern "C"
