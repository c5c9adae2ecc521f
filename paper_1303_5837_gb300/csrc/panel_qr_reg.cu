// panel_qr_reg.cu -- TSQR tree nodes held in the registers of one CTA.
//
// A node of R <= 16 TS rows and bk <= 16 TC columns (a leaf of the panel, or
// the stacked R factors of a merge: Sec. 3.1) is factored by Householder QR
// with its tile in the registers of 256 threads: thread (rg, cg), rg = lane
// mod 16 and cg = 2 warp + lane / 16, holds rows rg + 16 s (s < TS) and
// columns cg + 16 t (t < TC).  A half-warp therefore holds every row of its
// TC columns, so the column sums of the method need no shared memory and no
// barrier: a few shuffles inside the half-warp.  Per column j, one barrier:
//   * the owner of column j (the half-warp with cg = j mod 16) has published
//     x = A(j+1:, j) (zeros at rows <= j), tau_j and s_j = 1 / (alpha - beta)
//     in shared memory (v_j = s_j x below the diagonal, 1 on it);
//   * every thread multiplies x with its columns over its rows and the
//     half-warp sums the products: d_q = A(j, q) + s_j x^T A(j+1:, q) for
//     every column q, so the work of a step is the same in every warp;
//   * q > j: A(j, q) -= tau_j d_q and A(i, q) -= x_i s_j tau_j d_q;
//   * q < j: d_q = x_q(j) + s_j x_q^T x, and Z(q, j) = v_q^T v_j = s_q d_q,
//     the dot products larft needs for T, from the same pass;
//   * the owner of column j + 1 updates that column first and derives its
//     reflector before its other columns (look-ahead), so the reflector's
//     square root and divisions overlap with the other warps' updates.
// The stored x of every column is scaled by s_q once, after the last column.
// On this part the FP64 pipe (2 multiply-adds per clock per SM) is the scarce
// resource; this layout keeps every warp's FP64 instructions full and
// balanced, where a shared-memory tile with column-per-thread dot products
// leaves half the warps idle once fewer than half the columns remain.
#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {

namespace {

constexpr int kRegThreads = 256;

template <int TC, int TS>
struct RegSmem {
  double xs[2][16 * TS];                 // x of the published column, by column parity
  double tau[16 * TC], scal[16 * TC];    // tau_q, s_q (1 when tau_q = 0)
  double Z[16 * TC * (16 * TC - 1) / 2];  // v_i^T v_j, i < j, at j (j - 1) / 2 + i
  double T[16 * TC * (16 * TC - 1) / 2];  // strict upper part of T, same packing
};

// Sum of e[t] over the 16 lanes of the half-warp, for every t, on every lane
// (the same value on all of them): reduce-scatter over the first log2(TC)
// offsets, butterfly over the rest, then each sum is read from one lane.
template <int TC>
__device__ __forceinline__ void half_allsum(double (&e)[TC], int rg) {
  constexpr int L = TC == 1 ? 0 : TC == 2 ? 1 : TC == 4 ? 2 : 3;
  double v[TC];
#pragma unroll
  for (int t = 0; t < TC; ++t) v[t] = e[t];
#pragma unroll
  for (int k = 0; k < L; ++k) {
    const int o = 8 >> k;
    const int h = TC >> (k + 1);
    const bool up = (rg & o) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const double keep = up ? v[i + h] : v[i];
      const double send = up ? v[i] : v[i + h];
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, o, 16);
    }
  }
#pragma unroll
  for (int k = L; k < 4; ++k) v[0] += __shfl_xor_sync(0xffffffffu, v[0], 8 >> k, 16);
  // lane rg now holds the sum of value rg >> (4 - L)
#pragma unroll
  for (int t = 0; t < TC; ++t) e[t] = __shfl_sync(0xffffffffu, v[0], t << (4 - L), 16);
}

// Rows of a node that can be nonzero below the diagonal of column j (and so
// take part in its reflector): a leaf's rows below the diagonal; in a merge
// whose first child holds every diagonal row (c0 >= kmax) and whose other
// children have one height h, the other children's rows are kept in the
// order of their index t within the child (row t of every child, then row
// t + 1 ...), so the rows with t <= j -- the only ones of those children not
// structurally zero in column j -- come first, and the first child's rows
// below the diagonal are zero.  Row blocks [beg, end(j)) hold them all;
// skipping the others drops only exact zeros.  Other merges run dense.
template <bool MERGE>
struct NodeRows {
  int reord;  // 1: merge rows in the order above
  int beg;    // first block that can hold such rows
  int c0, nk, h, R;
  // leaves run every block (the zero rows of a short leaf cost nothing wrong)
  __device__ __forceinline__ int first() const { return MERGE ? beg : 0; }
  __device__ __forceinline__ int end(int j) const {
    if (!MERGE) return 1 << 20;
    const int p = reord ? c0 + nk * min(j + 1, h) : R;
    return (p + 15) >> 4;
  }
};

// Reflector of column jc = 16 U + jr, by the half-warp that holds it (cg =
// jr): beta = -sign(alpha) ||(alpha, x)||, tau = (beta - alpha) / beta,
// s = 1 / (alpha - beta); R(jc, jc) = beta; x published to xs.
template <int TC, int TS, int U, bool MERGE>
__device__ __forceinline__ void reflect(double (&A)[TS][TC], const NodeRows<MERGE> &nr, int rg, int jr, int jc,
                                        double *xs, double *tau, double *scal) {
  const unsigned hm = 0xffffu << (threadIdx.x & 16);
  const int se = nr.end(jc);
  double ss = 0.0;
#pragma unroll
  for (int s = U; s < TS; ++s) {
    if (s >= se) break;
    if (s < nr.first()) continue;
    if (s > U || rg > jr) ss = fma(A[s][U], A[s][U], ss);
  }
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(hm, ss, o, 16);
  const double alpha = __shfl_sync(hm, A[U][U], jr, 16);
  double t = 0.0, sc = 1.0;
  if (ss != 0.0) {
    const double nrm = sqrt(fma(alpha, alpha, ss));
    const double beta = (alpha >= 0.0) ? -nrm : nrm;
    t = (beta - alpha) / beta;
    sc = 1.0 / (alpha - beta);
    if (rg == jr) A[U][U] = beta;
  }
#pragma unroll
  for (int s = U; s < TS; ++s) {
    if (s >= se) break;
    if (s < nr.first()) continue;
    xs[16 * s + rg] = (s > U || rg > jr) ? A[s][U] : 0.0;
  }
  if (rg == 0) {
    tau[jc] = t;
    scal[jc] = sc;
  }
}

// A(:, q) -= v_j w_q for the thread's column t (q = cg + 16 t > j): row j
// takes w_q itself, rows below it x_i s_j w_q (x is zero at rows <= j).
template <int TC, int TS, int U>
__device__ __forceinline__ void update_col(double (&A)[TS][TC], const double (&x)[TS], int sb, int se, int t,
                                           double wt, double sw, bool row_j) {
#pragma unroll
  for (int s = U; s < TS; ++s) {
    if (s >= se) break;
    if (s < sb) continue;
    A[s][t] = fma(-x[s], sw, A[s][t]);
  }
  if (row_j) A[U][t] -= wt;
}

// Columns j = 16 U .. 16 U + 15 (those below kmax); row blocks [sb, se).
template <int TC, int TS, int U, bool MERGE>
__device__ __forceinline__ void qr_block(double (&A)[TS][TC], const NodeRows<MERGE> &nr, RegSmem<TC, TS> &sm,
                                         int rg, int cg, int kmax) {
  for (int jr = 0; jr < 16; ++jr) {
    const int j = 16 * U + jr;
    if (j >= kmax) return;
    __syncthreads();  // column j's x, tau_j and s_j are published
    const double tj = sm.tau[j], sj = sm.scal[j];
    const double *xb = sm.xs[j & 1];
    const int sb = nr.first(), se = nr.end(j);
    double x[TS];
#pragma unroll
    for (int s = 0; s < TS; ++s) x[s] = 0.0;
#pragma unroll
    for (int s = U; s < TS; ++s) {
      if (s >= se) break;
      if (s < sb) continue;
      x[s] = xb[16 * s + rg];
    }
    double w[TC];
#pragma unroll
    for (int t = 0; t < TC; ++t) w[t] = 0.0;
    if (tj != 0.0) {
      double e[TC];
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        double acc = 0.0;
#pragma unroll
        for (int s = U; s < TS; ++s) {
          if (s >= se) break;
          if (s < sb) continue;
          acc = fma(x[s], A[s][t], acc);
        }
        e[t] = acc;
      }
      half_allsum<TC>(e, rg);
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        const int q = cg + 16 * t;
        const double d = fma(sj, e[t], __shfl_sync(0xffffffffu, A[U][t], jr, 16));
        if (q > j) w[t] = tj * d;
        if (q < j && rg == 0) sm.Z[j * (j - 1) / 2 + q] = sm.scal[q] * d;
      }
    } else if (rg == 0) {
#pragma unroll
      for (int t = 0; t < TC; ++t) {
        const int q = cg + 16 * t;
        if (q < j) sm.Z[j * (j - 1) / 2 + q] = 0.0;
      }
    }
    const bool row_j = rg == jr;
    // the column after j first, then its reflector, then the other columns
    if (tj != 0.0 && cg > jr) update_col<TC, TS, U>(A, x, sb, se, U, w[U], sj * w[U], row_j);
    if (jr == 15) {
      if constexpr (U + 1 < TC) {
        if (tj != 0.0) update_col<TC, TS, U>(A, x, sb, se, U + 1, w[U + 1], sj * w[U + 1], row_j);
        if (j + 1 < kmax && cg == 0) reflect<TC, TS, U + 1, MERGE>(A, nr, rg, 0, j + 1, sm.xs[(j + 1) & 1], sm.tau, sm.scal);
#pragma unroll
        for (int t = U + 2; t < TC; ++t)
          if (tj != 0.0) update_col<TC, TS, U>(A, x, sb, se, t, w[t], sj * w[t], row_j);
      }
    } else {
      if (j + 1 < kmax && cg == jr + 1) reflect<TC, TS, U, MERGE>(A, nr, rg, jr + 1, j + 1, sm.xs[(j + 1) & 1], sm.tau, sm.scal);
#pragma unroll
      for (int t = U + 1; t < TC; ++t)
        if (tj != 0.0) update_col<TC, TS, U>(A, x, sb, se, t, w[t], sj * w[t], row_j);
    }
  }
}

template <int TC, int TS, int U, bool MERGE>
__device__ __forceinline__ void qr_blocks(double (&A)[TS][TC], const NodeRows<MERGE> &nr, RegSmem<TC, TS> &sm,
                                          int rg, int cg, int kmax) {
  if constexpr (U < TC) {
    qr_block<TC, TS, U, MERGE>(A, nr, sm, rg, cg, kmax);
    qr_blocks<TC, TS, U + 1, MERGE>(A, nr, sm, rg, cg, kmax);
  }
}

// Nodes of at most 128 rows, or 32 columns, leave room for two CTAs per SM,
// which hide each other's per-column barrier and reflector.
template <int TC, int TS>
constexpr int reg_min_blocks() {
  return TC * TS <= 32 ? 2 : 1;
}

template <int TC, int TS, bool MERGE>
__global__ void __launch_bounds__(kRegThreads, reg_min_blocks<TC, TS>()) tsqr_reg_kernel(TsqrNodeArgs a) {
  __shared__ RegSmem<TC, TS> sm;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = lane & 15, cg = 2 * warp + (lane >> 4);
  const int node = blockIdx.x;
  const int bk = a.bk;

  // ---- node rows: a leaf's consecutive panel rows, or the children's R rows
  int R, r0 = 0, start = 0, cnt = 1, midx = 0;
  if (a.is_leaf) {
    r0 = node * a.leaf_rows;
    R = min(a.leaf_rows, a.mk - r0);
  } else {
    round_node(a.rd, node, start, cnt, midx);
    if (cnt == 1) {  // promotion: nothing to factor
      if (tid == 0) {
        a.top_out[node] = a.top_in[start];
        a.c_out[node] = a.c_in[start];
      }
      return;
    }
    R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.c_in[start + ch];
  }
  const int kmax = min(R, bk);
  NodeRows<MERGE> nr;
  nr.R = R;
  nr.reord = 0;
  nr.beg = 0;
  nr.c0 = nr.nk = nr.h = 0;
  if (!a.is_leaf) {
    const int c0 = a.c_in[start], h = a.c_in[start + 1];
    bool same = true;
    for (int ch = 2; ch < cnt; ++ch) same &= a.c_in[start + ch] == h;
    if (same && c0 >= kmax) {
      nr.reord = 1;
      nr.c0 = c0;
      nr.nk = cnt - 1;
      nr.h = h;
      nr.beg = c0 >> 4;
    }
  }
  // panel row of local row r and its first structurally nonzero column (a
  // merge row that is row t of its child's R is zero left of column t)
  auto row_info = [&](int r, int &prow, int &fz) {
    prow = -1;
    fz = 1 << 30;
    if (r >= R) return;
    if (a.is_leaf) {
      prow = r0 + r;
      fz = 0;
      return;
    }
    if (nr.reord && r >= nr.c0) {
      const int t = (r - nr.c0) / nr.nk, k = 1 + (r - nr.c0) % nr.nk;
      prow = a.top_in[start + k] + t;
      fz = t;
      return;
    }
    int off = 0;
    for (int ch = 0; ch < cnt; ++ch) {
      const int c = a.c_in[start + ch];
      if (r < off + c) {
        prow = a.top_in[start + ch] + (r - off);
        fz = r - off;
        return;
      }
      off += c;
    }
  };

  // ---- load: lanes of a half-warp read 16 consecutive rows of a column ----
  double A[TS][TC];
  bool bad = false;
#pragma unroll
  for (int s = 0; s < TS; ++s) {
    int prow, fz;
    row_info(rg + 16 * s, prow, fz);
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int q = cg + 16 * t;
      double v = 0.0;
      if (prow >= 0 && q < bk && q >= fz) v = a.P[prow + (size_t)q * a.lda];
      bad |= not_finite(v);
      A[s][t] = v;
    }
  }
  if (bad && a.dev_info) atomicOr(a.dev_info + 1, CA_STATUS_NONFINITE);

  // ---- Householder QR, one barrier per column ----------------------------
  if (kmax > 0 && cg == 0) reflect<TC, TS, 0, MERGE>(A, nr, rg, 0, 0, sm.xs[0], sm.tau, sm.scal);
  qr_blocks<TC, TS, 0, MERGE>(A, nr, sm, rg, cg, kmax);
  __syncthreads();  // every tau, s and Z entry is written

  // v = s x below the diagonal of every reflector column
#pragma unroll
  for (int t = 0; t < TC; ++t) {
    const int q = cg + 16 * t;
    if (q < kmax) {
      const double sq = sm.scal[q];
#pragma unroll
      for (int s = 0; s < TS; ++s)
        if (rg + 16 * s > q) A[s][t] *= sq;
    }
  }

  // ---- T (larft, forward columnwise): T(i, j) = -tau_j sum_{q=i}^{j-1} T(i, q) Z(q, j),
  //      T(j, j) = tau_j; four threads per row i, each over every fourth q
  {
    const int i = tid >> 2, part = tid & 3;
    for (int j = 1; j < kmax; ++j) {
      const double tj = sm.tau[j];
      double acc = 0.0;
      if (i < j && tj != 0.0)
        for (int q = i + part; q < j; q += 4) {
          const double tiq = (q == i) ? sm.tau[i] : sm.T[q * (q - 1) / 2 + i];
          acc = fma(tiq, sm.Z[j * (j - 1) / 2 + q], acc);
        }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      acc += __shfl_xor_sync(0xffffffffu, acc, 2);
      if (i < j && part == 0) sm.T[j * (j - 1) / 2 + i] = (tj != 0.0) ? -tj * acc : 0.0;
      __syncthreads();  // column j of T is complete before column j + 1 reads it
    }
  }
  {
    const int b = a.b;
    double *Tg = a.Tp + (size_t)(a.is_leaf ? node : a.nleaves + midx) * b * b;
    for (int idx = tid; idx < b * b; idx += kRegThreads) {
      const int i = idx % b, jj = idx / b;
      double v = 0.0;
      if (jj < kmax && i <= jj) v = (i == jj) ? sm.tau[jj] : sm.T[jj * (jj - 1) / 2 + i];
      Tg[idx] = v;
    }
  }

  // ---- write back: leaf in place; merge: R into the first child's rows, Y
  //      into the other children's rows (on and above their diagonal)
#pragma unroll
  for (int s = 0; s < TS; ++s) {
    int prow, fz;
    row_info(rg + 16 * s, prow, fz);
#pragma unroll
    for (int t = 0; t < TC; ++t) {
      const int q = cg + 16 * t;
      if (prow >= 0 && q < bk && q >= fz) a.P[prow + (size_t)q * a.lda] = A[s][t];
    }
  }
  if (tid == 0) {
    a.top_out[node] = a.is_leaf ? r0 : a.top_in[start];
    a.c_out[node] = kmax;
  }
}

template <int TC, int TS>
cudaError_t launch_reg(const TsqrNodeArgs &a, int nodes, cudaStream_t st) {
  if (a.is_leaf)
    tsqr_reg_kernel<TC, TS, false><<<nodes, kRegThreads, 0, st>>>(a);
  else
    tsqr_reg_kernel<TC, TS, true><<<nodes, kRegThreads, 0, st>>>(a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Cluster form: a node of R <= 16 TS G rows (G <= 8 CTAs of one cluster) and
// 64 < bk <= 128 columns; CTA `rank` holds node rows 16 TS rank + rg + 16 s
// in registers with the same thread layout (TC = 8).  The column sums of the
// method become cluster sums: each CTA publishes its partial, every CTA reads
// all G partials in rank order (the same value everywhere) -- two cluster
// barriers per column:
//   C1: the partial sums of squares of column j below its diagonal and
//       A(j, j) are published; one thread per CTA derives tau_j, s_j, beta_j;
//       the owner half-warp stages its part of x;
//   C2: the partial dot products x^T A(:, q) of every column and row j are
//       published; every thread forms d_q and updates its rows, the owner of
//       column j + 1 first (and publishes that column's partial sum of
//       squares and, on the CTA that holds row j + 1, A(j + 1, j + 1)).
// Every CTA passes every barrier: control flow is uniform over the cluster.
// ---------------------------------------------------------------------------
constexpr int kCTC = 8;  // columns per thread: bk <= 128

template <int TS>
struct CRegSmem {
  double xs[16 * TS];              // this CTA's part of x_j (zeros at rows <= j)
  double epub[2][16 * kCTC];       // partial x_j^T A(:, q) over this CTA's rows, by step parity
  double rowpub[2][16 * kCTC];     // row j (on the CTA that holds it), by step parity
  double sspub[2];                 // partial sum of squares of a column below its diagonal
  double alphapub[2];              // its diagonal element (on the CTA that holds it)
  double tau[16 * kCTC], scal[16 * kCTC];
  double beta;
  double Z[16 * kCTC * (16 * kCTC - 1) / 2];  // v_i^T v_j, i < j (rank 0)
  double T[16 * kCTC * (16 * kCTC - 1) / 2];  // strict upper part of T (rank 0)
};

// Sum over the cluster's G partials of column q_t of this half-warp (every
// t), in rank order, on every lane: lane L of the half-warp reads ranks
// 4 (L & 1) .. + 3 of column t = L >> 1, the two halves are added, and each
// sum is broadcast from lane 2 t.
__device__ __forceinline__ void cluster_colsum(cg::cluster_group &cl, const double *pub, int cg, int rg, int G,
                                               double (&e)[kCTC]) {
  const int t = rg >> 1, h = rg & 1;
  const double *col = pub + cg + 16 * t;
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int r = 4 * h + k;
    if (r < G) s += *cl.map_shared_rank(col, r);
  }
  const double other = __shfl_xor_sync(0xffffffffu, s, 1, 16);
  s = h ? other + s : s + other;  // (ranks 0-3) + (ranks 4-7) on both lanes
#pragma unroll
  for (int u = 0; u < kCTC; ++u) e[u] = __shfl_sync(0xffffffffu, s, 2 * u, 16);
}

// Columns j = 16 U .. 16 U + 15 below kmax, cluster form.
template <int TS, int U>
__device__ __forceinline__ void cqr_block(cg::cluster_group &cl, double (&A)[TS][kCTC], CRegSmem<TS> &sm, int rg,
                                          int cg, int rank, int G, int p0, int kmax) {
  constexpr int RL = 16 * TS;  // rows per CTA
  constexpr int SJ = U % TS;   // block of row j within its CTA
  for (int jr = 0; jr < 16; ++jr) {
    const int j = 16 * U + jr;
    if (j >= kmax) return;
    const int q = j & 1;
    const int oj = j / RL;  // the CTA that holds row j
    cl.sync();              // C1: partial sums of squares and A(j, j) of column j are published
    if (threadIdx.x == 0) {
      double xn2 = 0.0;
      for (int r = 0; r < G; ++r) xn2 += *cl.map_shared_rank(&sm.sspub[q], r);
      const double alpha = *cl.map_shared_rank(&sm.alphapub[q], oj);
      double t = 0.0, sc = 1.0, be = alpha;
      if (xn2 != 0.0) {
        const double nrm = sqrt(fma(alpha, alpha, xn2));
        be = (alpha >= 0.0) ? -nrm : nrm;
        t = (be - alpha) / be;
        sc = 1.0 / (alpha - be);
      }
      sm.tau[j] = t;
      sm.scal[j] = sc;
      sm.beta = be;
    }
    __syncthreads();
    const double tj = sm.tau[j], sj = sm.scal[j];
    if (cg == jr) {  // the owner half-warp stages its part of x; row j takes beta
#pragma unroll
      for (int s = 0; s < TS; ++s) sm.xs[rg + 16 * s] = (p0 + rg + 16 * s > j) ? A[s][U] : 0.0;
      if (rank == oj && rg == jr) A[SJ][U] = sm.beta;
    }
    // row j as it stands (before this step's update), for d_q on every CTA
    if (rank == oj && rg == jr) {
#pragma unroll
      for (int t = 0; t < kCTC; ++t) sm.rowpub[q][cg + 16 * t] = A[SJ][t];
    }
    __syncthreads();
    double x[TS];
#pragma unroll
    for (int s = 0; s < TS; ++s) x[s] = sm.xs[rg + 16 * s];
    double e[kCTC];
#pragma unroll
    for (int t = 0; t < kCTC; ++t) {
      double acc = 0.0;
#pragma unroll
      for (int s = 0; s < TS; ++s) acc = fma(x[s], A[s][t], acc);
      e[t] = acc;
    }
    half_allsum<kCTC>(e, rg);
    if (rg == 0) {
#pragma unroll
      for (int t = 0; t < kCTC; ++t) sm.epub[q][cg + 16 * t] = e[t];
    }
    cl.sync();  // C2: every CTA's partial dot products and row j are published
    cluster_colsum(cl, sm.epub[q], cg, rg, G, e);
    double rowj[kCTC];
    {
      const double *rp = cl.map_shared_rank(sm.rowpub[q], oj);
      const double v = (rg < kCTC) ? rp[cg + 16 * rg] : 0.0;
#pragma unroll
      for (int t = 0; t < kCTC; ++t) rowj[t] = __shfl_sync(0xffffffffu, v, t, 16);
    }
    double w[kCTC];
#pragma unroll
    for (int t = 0; t < kCTC; ++t) {
      const int qc = cg + 16 * t;
      const double d = fma(sj, e[t], rowj[t]);
      w[t] = (qc > j && tj != 0.0) ? tj * d : 0.0;
      if (rank == 0 && rg == 0 && qc < j) sm.Z[j * (j - 1) / 2 + qc] = sm.scal[qc] * d;
    }
    const bool row_j = (rank == oj && rg == jr);
    // the column after j first, its partial sum of squares and diagonal, then the rest
    auto upd = [&](int t) {
#pragma unroll
      for (int s = 0; s < TS; ++s) A[s][t] = fma(-x[s], sj * w[t], A[s][t]);
      if (row_j) A[SJ][t] -= w[t];
    };
    auto publish_next = [&](int t, int sjn) {  // column j + 1 = cg + 16 t, held by this half-warp
      double ss = 0.0;
#pragma unroll
      for (int s = 0; s < TS; ++s)
        if (p0 + rg + 16 * s > j + 1) ss = fma(A[s][t], A[s][t], ss);
      const unsigned hm = 0xffffu << (threadIdx.x & 16);
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(hm, ss, o, 16);
      if (rg == 0) sm.sspub[q ^ 1] = ss;
      if (rank == (j + 1) / RL && rg == ((j + 1) & 15)) {
#pragma unroll
        for (int s = 0; s < TS; ++s)
          if (s == sjn) sm.alphapub[q ^ 1] = A[s][t];
      }
    };
    const bool more = j + 1 < kmax;
    if (cg > jr) upd(U);
    if (jr == 15) {
      if constexpr (U + 1 < kCTC) {
        upd(U + 1);
        if (more && cg == 0) publish_next(U + 1, (U + 1) % TS);
#pragma unroll
        for (int t = U + 2; t < kCTC; ++t) upd(t);
      }
    } else {
      if (more && cg == jr + 1) publish_next(U, SJ);
#pragma unroll
      for (int t = U + 1; t < kCTC; ++t) upd(t);
    }
  }
}

template <int TS, int U>
__device__ __forceinline__ void cqr_blocks(cg::cluster_group &cl, double (&A)[TS][kCTC], CRegSmem<TS> &sm, int rg,
                                           int cg, int rank, int G, int p0, int kmax) {
  if constexpr (U < kCTC) {
    cqr_block<TS, U>(cl, A, sm, rg, cg, rank, G, p0, kmax);
    cqr_blocks<TS, U + 1>(cl, A, sm, rg, cg, rank, G, p0, kmax);
  }
}

template <int TS>
__global__ void __launch_bounds__(kRegThreads, 1) tsqr_creg_kernel(TsqrNodeArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int G = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int node = blockIdx.x / G;
  extern __shared__ __align__(16) char craw[];
  CRegSmem<TS> &sm = *reinterpret_cast<CRegSmem<TS> *>(craw);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int rg = lane & 15, cg = 2 * warp + (lane >> 4);
  const int bk = a.bk;
  constexpr int RL = 16 * TS;
  const int p0 = rank * RL;

  int R, r0 = 0, start = 0, cnt = 1, midx = 0;
  if (a.is_leaf) {
    r0 = node * a.leaf_rows;
    R = min(a.leaf_rows, a.mk - r0);
  } else {
    round_node(a.rd, node, start, cnt, midx);
    if (cnt == 1) {  // promotion: the whole cluster returns before any barrier
      if (rank == 0 && tid == 0) {
        a.top_out[node] = a.top_in[start];
        a.c_out[node] = a.c_in[start];
      }
      return;
    }
    R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.c_in[start + ch];
  }
  auto row_info = [&](int r, int &prow, int &fz) {  // node row r
    prow = -1;
    fz = 1 << 30;
    if (r >= R) return;
    if (a.is_leaf) {
      prow = r0 + r;
      fz = 0;
      return;
    }
    int off = 0;
    for (int ch = 0; ch < cnt; ++ch) {
      const int c = a.c_in[start + ch];
      if (r < off + c) {
        prow = a.top_in[start + ch] + (r - off);
        fz = r - off;
        return;
      }
      off += c;
    }
  };

  double A[TS][kCTC];
  bool bad = false;
#pragma unroll
  for (int s = 0; s < TS; ++s) {
    int prow, fz;
    row_info(p0 + rg + 16 * s, prow, fz);
#pragma unroll
    for (int t = 0; t < kCTC; ++t) {
      const int qc = cg + 16 * t;
      double v = 0.0;
      if (prow >= 0 && qc < bk && qc >= fz) v = a.P[prow + (size_t)qc * a.lda];
      bad |= not_finite(v);
      A[s][t] = v;
    }
  }
  if (bad && a.dev_info) atomicOr(a.dev_info + 1, CA_STATUS_NONFINITE);

  const int kmax = min(R, bk);
  // column 0's partial sum of squares and diagonal
  if (cg == 0) {
    double ss = 0.0;
#pragma unroll
    for (int s = 0; s < TS; ++s)
      if (p0 + rg + 16 * s > 0) ss = fma(A[s][0], A[s][0], ss);
    const unsigned hm = 0xffffu << (tid & 16);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) ss += __shfl_xor_sync(hm, ss, o, 16);
    if (rg == 0) sm.sspub[0] = ss;
    if (rank == 0 && rg == 0) sm.alphapub[0] = A[0][0];
  }
  cqr_blocks<TS, 0>(cl, A, sm, rg, cg, rank, G, p0, kmax);
  cl.sync();  // every peer has read this CTA's published sums; tau and scal are final

  // v = s x below the diagonal of every reflector column
#pragma unroll
  for (int t = 0; t < kCTC; ++t) {
    const int qc = cg + 16 * t;
    if (qc < kmax) {
      const double sq = sm.scal[qc];
#pragma unroll
      for (int s = 0; s < TS; ++s)
        if (p0 + rg + 16 * s > qc) A[s][t] *= sq;
    }
  }
  if (rank == 0) {
    // T (larft, forward columnwise), two threads per row i (rows up to 127)
    const int i = tid >> 1, part = tid & 1;
    for (int j = 1; j < kmax; ++j) {
      const double tj = sm.tau[j];
      double acc = 0.0;
      if (i < j && tj != 0.0)
        for (int qq = i + part; qq < j; qq += 2) {
          const double tiq = (qq == i) ? sm.tau[i] : sm.T[qq * (qq - 1) / 2 + i];
          acc = fma(tiq, sm.Z[j * (j - 1) / 2 + qq], acc);
        }
      acc += __shfl_xor_sync(0xffffffffu, acc, 1);
      if (i < j && part == 0) sm.T[j * (j - 1) / 2 + i] = (tj != 0.0) ? -tj * acc : 0.0;
      __syncthreads();
    }
    const int b = a.b;
    double *Tg = a.Tp + (size_t)(a.is_leaf ? node : a.nleaves + midx) * b * b;
    for (int idx = tid; idx < b * b; idx += kRegThreads) {
      const int ii = idx % b, jj = idx / b;
      double v = 0.0;
      if (jj < kmax && ii <= jj) v = (ii == jj) ? sm.tau[jj] : sm.T[jj * (jj - 1) / 2 + ii];
      Tg[idx] = v;
    }
  }
#pragma unroll
  for (int s = 0; s < TS; ++s) {
    int prow, fz;
    row_info(p0 + rg + 16 * s, prow, fz);
#pragma unroll
    for (int t = 0; t < kCTC; ++t) {
      const int qc = cg + 16 * t;
      if (prow >= 0 && qc < bk && qc >= fz) a.P[prow + (size_t)qc * a.lda] = A[s][t];
    }
  }
  if (rank == 0 && tid == 0) {
    a.top_out[node] = a.is_leaf ? r0 : a.top_in[start];
    a.c_out[node] = kmax;
  }
}

template <int TS>
cudaError_t launch_creg(const TsqrNodeArgs &a, int nodes, int G, cudaStream_t st) {
  const size_t smem = sizeof(CRegSmem<TS>);
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(tsqr_creg_kernel<TS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)sizeof(CRegSmem<TS>));
  });
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nodes * G);
  cfg.blockDim = dim3(kRegThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tsqr_creg_kernel<TS>, a);
}

}  // namespace

bool tsqr_reg_fits(int rows, int bk) { return bk >= 1 && bk <= 64 && rows >= 1 && rows <= 256; }

// Cluster form: 64 < bk <= 128 and more rows than one CTA holds, at most 8
// CTAs of 64 (TS = 4) or 128 (TS = 8) rows.
int tsqr_creg_cluster(int rows, int bk) {
  if (bk <= 64 || bk > 128 || rows <= 128 || rows > 1024) return 0;
  if (rows <= 512) return (rows + 63) / 64;
  return (rows + 127) / 128;
}

cudaError_t launch_tsqr_creg(const TsqrNodeArgs &a, int nodes, int rows, cudaStream_t st) {
  const int G = tsqr_creg_cluster(rows, a.bk);
  if (G < 2) return cudaErrorInvalidValue;
  return rows <= 512 ? launch_creg<4>(a, nodes, G, st) : launch_creg<8>(a, nodes, G, st);
}

cudaError_t launch_tsqr_reg(const TsqrNodeArgs &a, int nodes, int rows, cudaStream_t st, bool *done) {
  *done = false;
  if (!tsqr_reg_fits(rows, a.bk)) return cudaSuccess;
  *done = true;
  if (a.bk <= 32) {
    if (rows <= 128) return launch_reg<2, 8>(a, nodes, st);
    return launch_reg<2, 16>(a, nodes, st);
  }
  if (rows <= 128) return launch_reg<4, 8>(a, nodes, st);
  return launch_reg<4, 16>(a, nodes, st);
}

}  // namespace cagb
