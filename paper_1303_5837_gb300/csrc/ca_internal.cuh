// ca_internal.cuh -- shared definitions of the GB300 CALU/CAQR library:
// the reduction-tree plan (host and device), workspace layout, launch
// helpers and small device utilities.
#pragma once

#include <cooperative_groups.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ca_gb300.h"

namespace cagb {

namespace cg = cooperative_groups;

constexpr int kMaxRounds = 64;
constexpr int kMaxPanel = 256;  // widest panel any kernel here accepts

// @region tree_plan
// ---------------------------------------------------------------------------
// Reduction tree plan (Sec. 3.1 / 3.2: leaves of the panel, then log Pr
// pairwise reduction steps per level).  A round merges groups of consecutive
// nodes of the previous round.  Its inputs form `ngroups` groups: all but the
// last hold `s` nodes, the last holds `s_last`.  Output o of a group merges
// `w` consecutive inputs (w = 2 for a binary step, w = s for a flat merge);
// a trailing output with a single input is a promotion.
// ---------------------------------------------------------------------------
struct RoundDesc {
  int n_in, n_out;
  int ngroups, s, s_last;
  int w, h, h_last;  // merge width; outputs per full / last group
  int mfull;         // merges in a full group
  int merge_base;    // merges in all earlier rounds
  int max_cnt;       // largest number of inputs of one output
};

struct Plan {
  int nleaves;
  int nrounds;
  int nmerges;
  RoundDesc r[kMaxRounds];
};

__host__ __device__ inline void round_node(const RoundDesc &rd, int o, int &start, int &cnt,
                                           int &midx) {
  int g = (o < (rd.ngroups - 1) * rd.h) ? o / rd.h : rd.ngroups - 1;
  int t = o - g * rd.h;
  int sg = (g == rd.ngroups - 1) ? rd.s_last : rd.s;
  start = g * rd.s + t * rd.w;
  int rem = sg - t * rd.w;
  cnt = rem < rd.w ? rem : rd.w;
  midx = rd.merge_base + g * rd.mfull + t;
}

// Builds the plan for `nleaves` leaves; returns false for a malformed tree.
// Per level, groups of fan_in consecutive nodes; binary style pairs
// neighbours until one node is left in each group, flat style merges a group
// at once; the last level takes every remaining node.
__host__ __device__ inline bool build_plan(int nleaves, const ca_tree_t &t, Plan &p) {
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
// @endregion tree_plan

// ---------------------------------------------------------------------------
// Argmax helpers: |x| compared through the bit pattern (an integer compare,
// so the FP64 pipe is left to the arithmetic); ties go to the lower position.
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long absbits(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}

struct ArgMax {
  unsigned long long key;  // |x| bits
  int pos;                 // position (smaller wins on equal key)
};

__device__ __forceinline__ ArgMax argmax_better(ArgMax a, ArgMax b) {
  if (b.key > a.key || (b.key == a.key && b.pos < a.pos)) return b;
  return a;
}

__device__ __forceinline__ ArgMax warp_argmax(ArgMax v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    ArgMax o;
    o.key = __shfl_xor_sync(0xffffffffu, v.key, off);
    o.pos = __shfl_xor_sync(0xffffffffu, v.pos, off);
    v = argmax_better(v, o);
  }
  return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

__device__ __forceinline__ bool not_finite(double x) {
  return ((unsigned long long)__double_as_longlong(x) & 0x7ff0000000000000ull) ==
         0x7ff0000000000000ull;
}

// ---------------------------------------------------------------------------
// Launch accounting (prof.cu): construct a ProfScope right before a launch.
// ---------------------------------------------------------------------------
enum KernelClass {
  kClsTsluNode = 0,
  kClsLaswp,
  kClsLuFinish,
  kClsTrsmU12,
  kClsGemm,
  kClsTsqrNode,
  kClsTreeApply,
  kClsSolve,
  kClsSplit,
  kClsGemmTc,
  kClsRefine,
  kClsBatched,
  kClsTreeNarrow,
  kNumClasses
};

class ProfScope {
 public:
  ProfScope(int cls, cudaStream_t st, double flops);
  ~ProfScope();
  ProfScope(const ProfScope &) = delete;
  ProfScope &operator=(const ProfScope &) = delete;

 private:
  int cls_;
  cudaStream_t st_;
  double flops_;
  cudaEvent_t a_ = nullptr, b_ = nullptr;
};

// round up to a multiple of 256 bytes
inline size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

// ---------------------------------------------------------------------------
// Kernel launch entry points implemented in the .cu files (host side).
// Every function enqueues on `st` and returns a cudaError_t.
// ---------------------------------------------------------------------------

// LU panel (panel_lu.cu)
struct LuPanelWs {
  int *cand[2];      // candidate row labels, [node][b]
  int *ncand[2];     // candidate count per node
  double *lu11;      // b x b root factors (column-major, ld b)
  int *perm_src;     // net row permutation of the panel swap: rows
  int *perm_dst;     //   perm_src[i] move to perm_dst[i], i < *perm_cnt
  int *perm_cnt;
};
size_t lu_panel_ws_bytes(int nleaves_max, int b);
void lu_panel_ws_carve(void *work, int nleaves_max, int b, LuPanelWs &ws);

// skip (all launchers below that take it): when not null, the kernels do
// nothing if *skip != 0 at the time they run -- a stage enqueued ahead whose
// need is decided on the device (the refactorization fallback of the mixed
// solve).
cudaError_t tslu_panel(int mk, int bk, double *P, int lda, int leaf_rows, const Plan &plan,
                       const LuPanelWs &ws, int *ipiv_k, int ipiv_base, int *dev_info,
                       cudaStream_t st, const int *skip = nullptr);
cudaError_t laswp_apply(int ncols, double *A, int lda, int row0, const LuPanelWs &ws, int bk,
                        cudaStream_t st, const int *skip = nullptr);
// the tournament with the 2D multilevel operator (batched.cu): one CTA per
// node, the node factored in shared memory by CALU of the levels below
bool op_params_ok(const ca_tree_t &t);
bool op_node_feasible(int rows, int bk, const ca_tree_t &t);
size_t op_ws_bytes(int nodes, const ca_tree_t &t);
cudaError_t tslu_panel_op(int mk, int bk, double *P, int lda, const ca_tree_t &tree, const Plan &plan,
                          const LuPanelWs &ws, int *opws, int *ipiv_k, int ipiv_base, int *dev_info,
                          cudaStream_t st, const int *skip = nullptr);
cudaError_t lu_panel_finish(int mk, int bk, double *P, int lda, const LuPanelWs &ws,
                            cudaStream_t st, const int *skip = nullptr);
cudaError_t trsm_u12(int bk, int nt, const double *L11, int ldl, double *A12, int lda,
                     cudaStream_t st, const int *skip = nullptr);

// FP64 GEMM C -= A B (gemm_fp64.cu); A m x k, B k x n, column-major.  With
// skip != null the kernel does nothing when *skip != 0 (a refinement loop
// enqueued ahead whose stop test has fired).
cudaError_t gemm_minus_f64(int m, int n, int k, const double *A, int lda, const double *B,
                           int ldb, double *C, int ldc, cudaStream_t st, const int *skip = nullptr);

// QR panel and tree update (panel_qr.cu)
struct QrPanelWs {
  int *top[2];  // first panel row of each node's R rows
  int *c[2];    // number of R rows of each node
};
size_t qr_panel_ws_bytes(int nleaves_max);
void qr_panel_ws_carve(void *work, int nleaves_max, QrPanelWs &ws);

// One round of TSQR nodes (leaves, or the merges of one tree round).
struct TsqrNodeArgs {
  double *P;  // panel, ld lda
  int lda, mk, bk, b;
  int leaf_rows;
  int is_leaf;
  RoundDesc rd;
  const int *top_in, *c_in;
  int *top_out, *c_out;
  double *Tp;     // the panel's T blocks (b x b each)
  int nleaves;
  int rloc, ld;   // tile rows per CTA, tile leading dimension (odd)
  int *dev_info;
};
// Register-resident TSQR nodes (panel_qr_reg.cu) for nodes of at most 256
// rows and 64 columns held by one CTA; *done = false when the shape is not
// covered (the shared-memory node kernel then runs).
bool tsqr_reg_fits(int rows, int bk);
// Cluster form of the register-resident node (64 < bk <= 128, 129 .. 1024
// rows): its cluster size, 0 when the shape is not covered.
int tsqr_creg_cluster(int rows, int bk);
cudaError_t launch_tsqr_creg(const TsqrNodeArgs &a, int nodes, int rows, cudaStream_t st);
cudaError_t launch_tsqr_reg(const TsqrNodeArgs &a, int nodes, int rows, cudaStream_t st, bool *done);
cudaError_t tsqr_panel(int mk, int bk, int b, double *P, int lda, int leaf_rows,
                       const Plan &plan, double *Tp, const QrPanelWs &ws, int *dev_info,
                       cudaStream_t st);
cudaError_t tree_apply_qt(int mk, int bk, int b, const double *P, int lda, int leaf_rows,
                          const Plan &plan, const double *Tp, double *C, int ldc, int ncols,
                          const QrPanelWs &ws, cudaStream_t st);

// tensor-core update C -= sign A B with FP64 operands split into S bf16 digit
// slices (gemm_tc.cu); ws holds the slices and exponents.
// An operand is a batch of matrices given as vectors of length K (the rows of
// A, the columns of B): element (v, k) of item b is
// X[b * sb + off[b] + v * sv + k * sk] under a structure rule (shape 0 dense,
// 1 unit lower, 2 upper on (r, q) = (v + roff, k), or (k + roff, v) if trans).
struct TcOperand {
  const double *X;
  long long sv, sk, sb;
  const int *off;       // per-item element offset (device), or null
  int nv, nv_last;      // vectors per item / in the last item
  const int *nv_item;   // per-item vector count (device), or null
  int K, K_last;        // contraction length per item / in the last item
  const int *K_item;    // per-item length (device), or null
  int shape, trans, roff;
};
struct TcGemm {
  TcOperand A, B;
  int nbatch;
  double *C;            // item b: C + b * sbc + coff[b], ld ldc
  int ldc;
  long long sbc;
  const int *coff;
  double sign;
  int S, exact;
  const int *skip;      // as for the LU launchers (null: always run)
};
cudaError_t gemm_tc(const TcGemm &g, void *ws, int *status, cudaStream_t st);
size_t tc_gemm_ws_bytes_batched(int m, int n, int k, int S, int nbatch);
size_t tc_gemm_ws_bytes(int m, int n, int k, int S);
bool tc_gemm_supported(int k, int S, int exact);
cudaError_t gemm_minus_tc(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                          int ldc, int S, int exact, void *ws, int *status, cudaStream_t st,
                          const int *skip = nullptr);

// CAQR tree update on the tensor cores (update_tc.cu)
size_t tree_tc_ws_bytes(int mk, int bk, int ncols, int leaf_rows, int nleaves, int S);
cudaError_t tree_apply_qt_tc(int mk, int bk, int b, const double *P, int lda, int leaf_rows, const Plan &plan,
                             const double *Tp, double *C, int ldc, int ncols, const QrPanelWs &ws, void *tcws,
                             int S, int exact, int *status, cudaStream_t st);

// triangular solves (solve.cu).  The dependency-ordered solve keeps its
// ready flags in caller memory (SolveWs, solve_ws_bytes(n) bytes): word 0
// records a wait that gave up, the flags follow.  status / status_bit: where
// a given-up wait is recorded (the workspace's word 0, or a dev_info word);
// skip: as for gemm_minus_f64.
struct SolveWs {
  int *status;
  int *flags;
};
size_t solve_ws_bytes(int n);
void solve_ws_carve(void *w, int n, SolveWs &s);
void solve_test_hook(long long wait_cycles, int withhold_blk);
cudaError_t getrs_swap(int n, int nrhs, const int *ipiv, double *B, int ldb, cudaStream_t st,
                       const int *skip = nullptr);
cudaError_t trsm_left(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B, int ldb,
                      const SolveWs &ws, int *status, int status_bit, const int *skip, cudaStream_t st);

// iterative refinement pieces (ir.cu).  Every kernel of a refinement step
// takes the loop's stop word (IrWs::ctl) and does nothing once it is set, so
// the whole loop is enqueued without waiting on the host.
struct IrCtl {
  int done;       // the phase has stopped (or never started): its kernels do nothing
  int ok;         // it stopped at berr <= tol
  int ran;        // it started
  int stall;      // consecutive steps whose backward error did not halve
  int iters;      // corrections applied in this phase
  int iter_base;  // corrections of the phases before it
  double slow;    // a step reducing the error by less than 1/slow ends the phase
  double prev;    // backward error (least squares: correction size) of the previous step
  double berr;    // latest backward error (largest over the right-hand sides)
  double dx;      // least squares: relative size of the last correction
};
constexpr int kIrPhases = 3;  // AUTO: classic, GMRES, refactorization with 7 exact digits
struct IrWs {
  double *partial, *R, *rowsum, *anorm, *berr;
  IrCtl *ctl;                // the control block of the phase these calls drive
  IrCtl *phase[kIrPhases];   // all phases' control blocks
  int *info2;                // dev_info of the refactorization
};
size_t ir_ws_bytes(int n, int nrhs);
void ir_ws_carve(void *ws, int n, int nrhs, IrWs &w);
cudaError_t ir_anorm(int n, const double *A, int lda, const IrWs &w, cudaStream_t st);
cudaError_t ir_begin(const IrWs &w, double slow, cudaStream_t st);
// a phase after `prev`: it runs only if prev did not reach tol
cudaError_t ir_begin_next(const IrCtl *prev, const IrWs &w, double slow, cudaStream_t st);
// dst = src (m x n) unless *skip
cudaError_t copy_matrix(int m, int n, const double *src, int lds, double *dst, int ldd, const int *skip,
                        cudaStream_t st);
// after the refactorization phase (w.ctl): if it ran, its dev_info replaces
// the first factorization's, plus the CA_STATUS_REFACTORED bit
cudaError_t ir_merge_info(const IrWs &w, const int *info2, int *dev_info, cudaStream_t st);
cudaError_t ir_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, const IrWs &w, cudaStream_t st);
cudaError_t ir_berr(int n, int nrhs, const double *X, int ldx, const double *B, int ldb, const IrWs &w,
                    cudaStream_t st);
// the stop test of step `it` of the phase (device): berr <= tol, it ==
// max_iter, a slow step, or two steps in a row that failed to halve the
// backward error; writes the latest backward error and the corrections so far
// to *berr_out / *iters_out when not null.
cudaError_t ir_decide(int it, int max_iter, double tol, int nrhs, const IrWs &w, double *berr_out,
                      int *iters_out, cudaStream_t st);
cudaError_t ir_update(int n, int nrhs, const IrWs &w, double *X, int ldx, cudaStream_t st);

// least-squares refinement (ir.cu): corrected semi-normal equations with the
// triangular factor R; r = b - A x (m x nrhs), s = A^T r, x += R^-1 R^-T s
struct LsWs {
  double *partial, *R, *S, *Rt, *sums, *anorm, *a1, *berr;
  IrCtl *ctl;
  IrCtl *phase[kIrPhases];
  int *info2;
};
size_t ls_ws_bytes(int m, int n, int nrhs);
void ls_ws_carve(void *ws, int m, int n, int nrhs, LsWs &w);
cudaError_t ls_norms(int m, int n, const double *A, int lda, const LsWs &w, cudaStream_t st);
cudaError_t ls_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, const LsWs &w, cudaStream_t st);
// s = A^T r and the backward error ||s|| / (||A||_1 (||A||inf ||x|| + ||b||)) per right-hand side
cudaError_t ls_normal_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                               const double *B, int ldb, const LsWs &w, cudaStream_t st);
cudaError_t ls_transpose_r(int n, const double *QR, int ldq, const LsWs &w, const int *skip, cudaStream_t st);
cudaError_t ls_update(int n, int nrhs, const LsWs &w, double *X, int ldx, cudaStream_t st);
cudaError_t ls_decide(int it, int max_iter, double tol, int nrhs, const LsWs &w, double *berr_out, int *iters_out,
                      cudaStream_t st);
cudaError_t ls_begin(const LsWs &w, const IrCtl *prev, cudaStream_t st);
cudaError_t ls_merge_info(const LsWs &w, int *dev_info, cudaStream_t st);

// GMRES corrections (ir.cu): at most kGmMax Arnoldi steps per correction,
// stopped when the preconditioned residual has dropped by kGmTol.
constexpr int kGmMax = 20;
constexpr double kGmTol = 1e-6;
struct GmCtl {
  int stop;    // Arnoldi finished (converged, breakdown, kGmMax) or not running
  int active;  // this correction runs at all
  int k;       // Arnoldi steps taken
  int pad;
  double beta, scale;
  double h[kGmMax + 1];
  double H[(kGmMax + 1) * kGmMax];
  double cs[kGmMax], sn[kGmMax], g[kGmMax + 1], y[kGmMax];
};
struct GmWs {
  double *V;        // n x (kGmMax + 1) Arnoldi vectors
  double *w;        // n
  double *partial;  // dot-product partial sums
  double *mv;       // matrix-vector partial sums
  GmCtl *ctl;
};
size_t gm_ws_bytes(int n);
void gm_ws_carve(void *ws, int n, GmWs &g);
cudaError_t ir_gmres_correction(int n, const double *A, int lda, const double *LU, int ldlu, const int *ipiv,
                                const IrWs &w, const GmWs &g, int j, double *X, int ldx, const SolveWs &sw,
                                int *status, int status_bit, cudaStream_t st);

}  // namespace cagb
