// api.cu -- the C-ABI: argument checks, the reduction-tree plan, workspace
// layout and the panel loops of CALU and CAQR (host side; every step runs in
// the kernels of panel_lu.cu, panel_qr.cu, gemm_fp64.cu and solve.cu).
#include <cstring>

#include "ca_internal.cuh"

namespace cagb {

// The plan of Sec. 3.1 / 3.2 reduction trees: per level, groups of fan_in
// consecutive nodes; binary style pairs neighbours until one node is left in
// each group, flat style merges a group at once; the last level takes every
// remaining node.
bool build_plan(int nleaves, const ca_tree_t &t, Plan &p) {
  p.nleaves = nleaves;
  p.nrounds = 0;
  p.nmerges = 0;
  if (nleaves < 1 || t.nlevels < 1 || t.nlevels > CA_MAX_LEVELS) return false;
  int cur = nleaves;
  for (int l = 0; l < t.nlevels; ++l) {
    int f = (l == t.nlevels - 1) ? cur : t.fan_in[l];
    if (f < 1) return false;
    int ngroups = (cur + f - 1) / f;
    int s = (ngroups == 1) ? cur : f;
    int s_last = cur - (ngroups - 1) * f;
    if (t.style[l] == CA_TREE_FLAT) {
      RoundDesc rd;
      rd.n_in = cur;
      rd.n_out = ngroups;
      rd.ngroups = ngroups;
      rd.s = s;
      rd.s_last = s_last;
      rd.w = s;
      rd.h = 1;
      rd.h_last = 1;
      rd.mfull = s >= 2 ? 1 : 0;
      rd.merge_base = p.nmerges;
      rd.max_cnt = s > s_last ? s : s_last;
      int merges = (ngroups - 1) * rd.mfull + (s_last >= 2 ? 1 : 0);
      if (merges > 0) {
        if (p.nrounds >= kMaxRounds) return false;
        p.r[p.nrounds++] = rd;
        p.nmerges += merges;
      }
    } else if (t.style[l] == CA_TREE_BINARY) {
      int in = cur;
      while (s > 1 || s_last > 1) {
        RoundDesc rd;
        rd.n_in = in;
        rd.ngroups = ngroups;
        rd.s = s;
        rd.s_last = s_last;
        rd.w = 2;
        rd.h = (s + 1) / 2;
        rd.h_last = (s_last + 1) / 2;
        rd.n_out = (ngroups - 1) * rd.h + rd.h_last;
        rd.mfull = s / 2;
        rd.merge_base = p.nmerges;
        rd.max_cnt = 2;
        int merges = (ngroups - 1) * rd.mfull + s_last / 2;
        if (merges > 0) {
          if (p.nrounds >= kMaxRounds) return false;
          p.r[p.nrounds++] = rd;
          p.nmerges += merges;
        }
        in = rd.n_out;
        s = rd.h;
        s_last = rd.h_last;
      }
    } else {
      return false;
    }
    cur = ngroups;
  }
  return cur == 1;
}

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
  int K = m < n ? m : n;
  *nl_max = 1;
  if (K == 0) return CA_OK;
  int bk = b < K ? b : K;
  if (bk > kMaxB) return CA_ERR_UNSUPPORTED;
  int nl = nleaves_of(m, tree->leaf_rows);
  Plan p;
  if (!build_plan(nl, *tree, p)) return CA_ERR_TREE;
  if (!lu_node_feasible(max_node_rows(p, m, tree->leaf_rows, bk), bk)) return CA_ERR_UNSUPPORTED;
  *nl_max = nl;
  return CA_OK;
}

int qr_shape(int m, int n, int b, const ca_tree_t *tree, int *nl_max, size_t *qbytes) {
  if (m < 0) return -1;
  if (n < 0 || n > m) return -2;
  if (b < 1) return -5;
  if (check_tree(tree, b)) return -6;
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

}  // namespace

extern "C" {

const char *ca_strerror(int code) {
  switch (code) {
    case CA_OK:
      return "success";
    case CA_ERR_WORKSPACE:
      return "workspace pointer is null or smaller than the workspace query";
    case CA_ERR_UNSUPPORTED:
      return "shape not supported by this build (panel width > 128 or a tree node too large)";
    case CA_ERR_LAUNCH:
      return "a CUDA kernel launch failed";
    case CA_ERR_TREE:
      return "malformed reduction tree";
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
  *work_bytes = lu_panel_ws_bytes(nl, b < kMaxB ? b : kMaxB);
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
  *work_bytes = qr_panel_ws_bytes(nl);
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
  *work_bytes = qr_panel_ws_bytes(nl);
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
  if (K > 0 && (!work || lwork < lu_panel_ws_bytes(nl, bw))) return CA_ERR_WORKSPACE;
  if (cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (K == 0) return CA_OK;
  LuPanelWs ws;
  lu_panel_ws_carve(work, nl, bw, ws);
  const int L = tree->leaf_rows;
  for (int kb = 0; kb < K; kb += b) {
    const int bk = (K - kb < b) ? K - kb : b;
    const int mk = m - kb;
    Plan plan;
    if (!build_plan(nleaves_of(mk, L), *tree, plan)) return CA_ERR_TREE;
    double *P = A + kb + (size_t)kb * lda;
    // 1. tournament pivoting over the tree (TSLU)
    if (tslu_panel(mk, bk, P, lda, L, plan, ws, ipiv + kb, kb, dev_info, stream) != cudaSuccess)
      return CA_ERR_LAUNCH;
    // 2. swap rows at left and right of the panel
    if (laswp_apply(n, A, lda, kb, ws, bk, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    // 3. L11 \ U11 into place, L21 = A21 U11^-1
    if (lu_panel_finish(mk, bk, P, lda, ws, stream) != cudaSuccess) return CA_ERR_LAUNCH;
    const int nt = n - kb - bk;
    if (nt > 0) {
      double *A12 = A + kb + (size_t)(kb + bk) * lda;
      // 4. U12 = L11^-1 A12
      if (trsm_u12(bk, nt, ws.lu11, bk, A12, lda, stream) != cudaSuccess) return CA_ERR_LAUNCH;
      // 5. A22 -= L21 U12
      if (mk - bk > 0 &&
          gemm_minus_f64(mk - bk, nt, bk, P + bk, lda, A12, lda, A12 + bk, lda, stream) != cudaSuccess)
        return CA_ERR_LAUNCH;
    }
  }
  return CA_OK;
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

int calu_getrs(int n, int nrhs, const double *LU, int lda, const int *ipiv, double *B, int ldb,
               cudaStream_t stream) {
  if (n < 0) return -1;
  if (nrhs < 0) return -2;
  if (n > 0 && !LU) return -3;
  if (lda < (n > 1 ? n : 1)) return -4;
  if (n > 0 && !ipiv) return -5;
  if (n > 0 && nrhs > 0 && !B) return -6;
  if (ldb < (n > 1 ? n : 1)) return -7;
  if (n == 0 || nrhs == 0) return CA_OK;
  if (getrs_swap(n, nrhs, ipiv, B, ldb, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (trsm_left(true, true, n, nrhs, LU, lda, B, ldb, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (trsm_left(false, false, n, nrhs, LU, lda, B, ldb, stream) != cudaSuccess) return CA_ERR_LAUNCH;
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
  if (n > 0 && (!work || lwork < qr_panel_ws_bytes(nl))) return CA_ERR_WORKSPACE;
  if (cudaMemsetAsync(dev_info, 0, 2 * sizeof(int), stream) != cudaSuccess) return CA_ERR_LAUNCH;
  if (n == 0) return CA_OK;
  QrPanelWs ws;
  qr_panel_ws_carve(work, nl, ws);
  const int L = tree->leaf_rows;
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    const int bk = (n - kb < b) ? n - kb : b;
    const int mk = m - kb;
    Plan plan;
    if (!build_plan(nleaves_of(mk, L), *tree, plan)) return CA_ERR_TREE;
    double *P = A + kb + (size_t)kb * lda;
    double *Tp = qtree + off;
    // 1. TSQR: leaves, then the R-elimination tree
    if (tsqr_panel(mk, bk, b, P, lda, L, plan, Tp, ws, dev_info, stream) != cudaSuccess)
      return CA_ERR_LAUNCH;
    // 2. trailing columns: leaves' Q^T (UPFACT), then merges' Q^T (UPELIM)
    const int nt = n - kb - bk;
    if (nt > 0 && tree_apply_qt(mk, bk, b, P, lda, L, plan, Tp, P + (size_t)bk * lda, lda, nt, ws,
                                stream) != cudaSuccess)
      return CA_ERR_LAUNCH;
    off += (size_t)(plan.nleaves + plan.nmerges) * b * b;
  }
  return CA_OK;
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
  if (!work || lwork < qr_panel_ws_bytes(nl)) return CA_ERR_WORKSPACE;
  QrPanelWs ws;
  qr_panel_ws_carve(work, nl, ws);
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
  if (trsm_left(false, false, n, nrhs, QR, lda, B, ldb, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  return CA_OK;
}

}  // extern "C"
