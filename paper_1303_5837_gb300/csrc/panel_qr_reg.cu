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

}  // namespace

bool tsqr_reg_fits(int rows, int bk) { return bk >= 1 && bk <= 64 && rows >= 1 && rows <= 256; }

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
