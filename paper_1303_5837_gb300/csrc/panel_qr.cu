// panel_qr.cu -- TSQR (Householder QR over the reduction tree) and the tree
// update that applies the panel's Q^T to the trailing columns (CAQR).
//
// Tree node = one thread-block cluster of G CTAs; the node's rows (a leaf of
// the panel, or the stacked upper-triangular R factors of its children) are
// split over the CTAs' shared memory.  Per column: the partial sums of
// squares and the partial dot products with the trailing columns are reduced
// inside each CTA (warp shuffles, shared memory) and across the cluster
// through distributed shared memory, in a fixed order, so every CTA derives
// the same reflector (Sec. 3.1: leaves factored, then the R factors
// eliminated two by two; Q kept as Y T Y^T).
#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {

constexpr int kQrThreads = 256;
constexpr int kQrWarps = kQrThreads / 32;
constexpr size_t kQrSmemBudget = 220 * 1024;
constexpr int kQrGroups = 4;  // row groups of the dot-product mapping

__host__ __device__ inline size_t tsqr_smem_bytes(int rloc, int ld, int bk) {
  size_t s = (size_t)ld * bk * 8;          // tile
  s += (size_t)kQrGroups * bk * 8;         // dot partials per row group
  s += (size_t)bk * 8;                     // CTA partial of w (read by peers)
  s += (size_t)bk * 8;                     // w
  s += (size_t)bk * 8;                     // tau
  s += 128;                                // scalars and reduce scratch
  s += (size_t)rloc * 4;                   // first structurally nonzero column per row
  s += (size_t)rloc * 4;                   // panel row of each local row
  size_t zs = (size_t)bk * (bk - 1) / 2 * 8 + 8;  // packed strict upper Gram matrix
  return s + zs + 64;
}

__device__ __forceinline__ void qr_sync(cg::cluster_group &cl, int G) {
  if (G > 1)
    cl.sync();
  else
    __syncthreads();
}

__device__ __forceinline__ double block_sum(double v, double *red, int tid) {
  v = warp_sum(v);
  __syncthreads();
  if ((tid & 31) == 0) red[tid >> 5] = v;
  __syncthreads();
  double s = 0.0;
#pragma unroll
  for (int w = 0; w < kQrWarps; ++w) s += red[w];
  return s;
}

__global__ void __launch_bounds__(kQrThreads, 1) tsqr_node_kernel(TsqrNodeArgs a) {
  cg::cluster_group cl = cg::this_cluster();
  const int G = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int node = blockIdx.x / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bk = a.bk, rloc = a.rloc, ld = a.ld;
  extern __shared__ __align__(16) char smem_raw[];
  double *tile = (double *)smem_raw;
  double *part = tile + (size_t)ld * bk;        // [kQrGroups][bk]
  double *wcta = part + (size_t)kQrGroups * bk; // bk
  double *w = wcta + bk;                        // bk
  double *tau = w + bk;                         // bk
  double *sc = tau + bk;                        // 8 scalars + 8 reduce slots
  int *fz = (int *)(sc + 16);                   // rloc
  int *prw = fz + rloc;                         // rloc: panel row of each local row
  // Z(i, j), i < j, packed column by column at j (j - 1) / 2 + i
  double *Z = (double *)(((uintptr_t)(prw + rloc) + 15) & ~(uintptr_t)15);
  // sc: [0] ss partial of this CTA, [1] beta, [2] tau, [3] scal, [4] skip;
  //     sc[8..15]: block-reduction scratch

  // ---- node inputs ------------------------------------------------------
  int R, start = 0, cnt = 1, midx = 0;
  int r0 = 0;
  const int p0 = rank * rloc;
  if (a.is_leaf) {
    r0 = node * a.leaf_rows;
    R = min(a.leaf_rows, a.mk - r0);
    for (int i = tid; i < rloc; i += kQrThreads) fz[i] = 0;
  } else {
    round_node(a.rd, node, start, cnt, midx);
    if (cnt == 1) {
      if (rank == 0 && tid == 0) {
        a.top_out[node] = a.top_in[start];
        a.c_out[node] = a.c_in[start];
      }
      return;
    }
    R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.c_in[start + ch];
    for (int i = tid; i < rloc; i += kQrThreads) {
      int p = p0 + i, off = 0, t = 0;
      for (int ch = 0; ch < cnt; ++ch) {
        int c = a.c_in[start + ch];
        if (p < off + c) {
          t = p - off;
          break;
        }
        off += c;
      }
      fz[i] = t;  // child-local row t: zeros left of column t
    }
  }
  __syncthreads();
  const int myrows = max(0, min(rloc, R - p0));

  // row index in the panel of local row i
  auto prow_of = [&](int i) -> int {
    if (a.is_leaf) return r0 + p0 + i;
    int p = p0 + i, off = 0;
    for (int ch = 0; ch < cnt; ++ch) {
      int c = a.c_in[start + ch];
      if (p < off + c) return a.top_in[start + ch] + (p - off);
      off += c;
    }
    return -1;
  };

  // ---- load (lanes over rows: consecutive rows of a column are adjacent) --
  for (int i = tid; i < myrows; i += kQrThreads) prw[i] = prow_of(i);
  __syncthreads();
  bool bad = false;
  for (int k = warp; k < bk; k += kQrWarps) {
    const double *col = a.P + (size_t)k * a.lda;
    for (int i = lane; i < myrows; i += 32) {
      double v = 0.0;
      if (k >= fz[i]) v = col[prw[i]];
      bad |= not_finite(v);
      tile[i + (size_t)k * ld] = v;
    }
  }
  if (bad && a.dev_info) atomicOr(a.dev_info + 1, CA_STATUS_NONFINITE);
  __syncthreads();
  // merge rows are structurally zero left of their child-local index (fz);
  // leaves have none, and their loops skip the test
  const bool leaf = a.is_leaf != 0;

  // ---- Householder QR on the distributed tile --------------------------
  const int kmax = min(R, bk);
  if (G == 1) {
    // One CTA holds the node: five barriers per column.  Column j's sub-
    // diagonal part x is scaled to v = x / (alpha - beta) only at the start
    // of the next column's pass (sc[6] holds the factor), so the dot
    // products w_q = tau v^T A(:, q) = tau (A(j, q) + s x^T A(j+1:, q)) and
    // the update A(:, q) -= v w_q = x (s w_q) read the unscaled column.
    const int g = tid / (kQrThreads / kQrGroups);
    const int qq0 = tid - g * (kQrThreads / kQrGroups);
    if (tid == 0) sc[6] = 1.0;
    for (int j = 0; j < kmax; ++j) {
      // pass 1: scale the previous column's v, sum of squares of this one
      const double sprev = sc[6];
      double ss = 0.0;
      for (int i = j + tid; i < myrows; i += kQrThreads) {
        if (j > 0 && (leaf || fz[i] <= j - 1)) tile[i + (size_t)(j - 1) * ld] *= sprev;
        if (i > j && (leaf || fz[i] <= j)) {
          const double v = tile[i + (size_t)j * ld];
          ss = fma(v, v, ss);
        }
      }
      ss = warp_sum(ss);
      if (lane == 0) sc[8 + warp] = ss;
      __syncthreads();
      if (tid == 0) {
        double xn2 = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < kQrWarps; ++w2) xn2 += sc[8 + w2];
        const double alpha = tile[j + (size_t)j * ld];
        if (xn2 == 0.0) {
          sc[4] = 1.0;
          sc[6] = 1.0;
          tau[j] = 0.0;
        } else {
          const double nrm = sqrt(fma(alpha, alpha, xn2));
          const double beta = (alpha >= 0.0) ? -nrm : nrm;
          tau[j] = (beta - alpha) / beta;
          sc[6] = 1.0 / (alpha - beta);
          sc[4] = 0.0;
          tile[j + (size_t)j * ld] = beta;
        }
      }
      __syncthreads();
      if (sc[4] != 0.0) continue;
      const double scal = sc[6], tj = tau[j];
      // pass 2: partial dot products over rows i = g mod 4, i > j
      const int nq = bk - j - 1;
      for (int qq = qq0; qq < nq; qq += kQrThreads / kQrGroups) {
        const int q = j + 1 + qq;
        const double *cq = tile + (size_t)q * ld;
        const double *cj = tile + (size_t)j * ld;
        double acc = 0.0;
        for (int i = j + 1 + g; i < myrows; i += kQrGroups)
          if (leaf || fz[i] <= j) acc = fma(cj[i], cq[i], acc);
        part[g * bk + q] = (g == 0 ? cq[j] : 0.0) + scal * acc;
      }
      __syncthreads();
      for (int q = j + 1 + tid; q < bk; q += kQrThreads) {
        double s2 = part[q];
#pragma unroll
        for (int g2 = 1; g2 < kQrGroups; ++g2) s2 += part[g2 * bk + q];
        w[q] = tj * s2;
      }
      __syncthreads();
      // pass 3: A(j, q) -= w_q; A(i, q) -= x_i (s w_q) for i > j
      for (int qq = qq0; qq < nq; qq += kQrThreads / kQrGroups) {
        const int q = j + 1 + qq;
        double *cq = tile + (size_t)q * ld;
        const double *cj = tile + (size_t)j * ld;
        const double wq = w[q], swq = scal * wq;
        if (g == 0) cq[j] -= wq;
        for (int i = j + 1 + g; i < myrows; i += kQrGroups)
          if (leaf || fz[i] <= j) cq[i] = fma(-cj[i], swq, cq[i]);
      }
      __syncthreads();
    }
    // the last column's deferred scaling
    if (kmax > 0) {
      const double sprev = sc[6];
      const int jl = kmax - 1;
      for (int i = jl + 1 + tid; i < myrows; i += kQrThreads)
        if (leaf || fz[i] <= jl) tile[i + (size_t)jl * ld] *= sprev;
    }
    __syncthreads();
  }
  for (int j = 0; j < (G == 1 ? 0 : kmax); ++j) {
    const int oj = j / rloc, lj = j - oj * rloc;
    // (a) partial ||x2||^2 over positions > j (structurally nonzero rows)
    double ss = 0.0;
    for (int i = max(j + 1 - p0, 0) + tid; i < myrows; i += kQrThreads)
      if (leaf || fz[i] <= j) {
        double v = tile[i + (size_t)j * ld];
        ss = fma(v, v, ss);
      }
    ss = block_sum(ss, sc + 8, tid);
    if (tid == 0) sc[0] = ss;
    qr_sync(cl, G);
    // (b) reflector from the cluster's partials (fixed order: same value in
    //     every CTA)
    // the G partial sums and alpha, read in parallel through DSMEM
    if (tid < G) part[tid] = (tid == rank) ? sc[0] : *cl.map_shared_rank(sc, tid);
    if (tid == 32)
      sc[5] = (oj == rank) ? tile[lj + (size_t)j * ld] : *cl.map_shared_rank(tile + lj + (size_t)j * ld, oj);
    __syncthreads();
    if (tid == 0) {
      double xn2 = 0.0;
      for (int q = 0; q < G; ++q) xn2 += part[q];  // fixed order: the same value in every CTA
      const double alpha = sc[5];
      if (xn2 == 0.0) {
        sc[4] = 1.0;
        sc[2] = 0.0;
      } else {
        double nrm = sqrt(fma(alpha, alpha, xn2));
        double beta = (alpha >= 0.0) ? -nrm : nrm;
        sc[1] = beta;
        sc[2] = (beta - alpha) / beta;
        sc[3] = 1.0 / (alpha - beta);
        sc[4] = 0.0;
      }
      tau[j] = sc[2];
    }
    qr_sync(cl, G);  // peers have read sc[0] and alpha
    if (sc[4] != 0.0) continue;
    const double scal = sc[3], tj = sc[2];
    // (c) v = x2 / (alpha - beta); R_jj = beta
    for (int i = max(j + 1 - p0, 0) + tid; i < myrows; i += kQrThreads)
      if (leaf || fz[i] <= j) tile[i + (size_t)j * ld] *= scal;
    if (oj == rank && tid == 0) tile[lj + (size_t)j * ld] = sc[1];
    __syncthreads();
    // (d) partial w_q = v^T A(:, q) for q > j: thread (g, qq), rows = g mod 4
    const int nq = bk - j - 1;
    {
      const int g = tid / (kQrThreads / kQrGroups);
      const int qq0 = tid - g * (kQrThreads / kQrGroups);
      for (int qq = qq0; qq < nq; qq += kQrThreads / kQrGroups) {
        const int q = j + 1 + qq;
        double acc = 0.0;
        for (int i = max(j - p0, 0) + g; i < myrows; i += kQrGroups) {
          if (!leaf && fz[i] > j) continue;
          double v = (p0 + i == j) ? 1.0 : tile[i + (size_t)j * ld];
          acc = fma(v, tile[i + (size_t)q * ld], acc);
        }
        part[g * bk + q] = acc;
      }
    }
    __syncthreads();
    for (int q = j + 1 + tid; q < bk; q += kQrThreads) {
      double s = part[q];
#pragma unroll
      for (int g = 1; g < kQrGroups; ++g) s += part[g * bk + q];
      wcta[q] = s;
    }
    qr_sync(cl, G);
    for (int q = j + 1 + tid; q < bk; q += kQrThreads) {
      double v[8];
#pragma unroll
      for (int r = 0; r < 8; ++r)  // all remote loads in flight, then the ordered sum
        v[r] = (r < G) ? ((r == rank) ? wcta[q] : *cl.map_shared_rank(wcta + q, r)) : 0.0;
      double s = 0.0;
#pragma unroll
      for (int r = 0; r < 8; ++r)
        if (r < G) s += v[r];
      w[q] = tj * s;
    }
    __syncthreads();
    // (e) A(:, q) -= v w_q for active rows >= j
    {
      const int g = tid / (kQrThreads / kQrGroups);
      const int qq0 = tid - g * (kQrThreads / kQrGroups);
      for (int qq = qq0; qq < nq; qq += kQrThreads / kQrGroups) {
        const int q = j + 1 + qq;
        const double wq = w[q];
        for (int i = max(j - p0, 0) + g; i < myrows; i += kQrGroups) {
          if (!leaf && fz[i] > j) continue;
          double v = (p0 + i == j) ? 1.0 : tile[i + (size_t)j * ld];
          tile[i + (size_t)q * ld] = fma(-v, wq, tile[i + (size_t)q * ld]);
        }
      }
    }
    qr_sync(cl, G);  // wcta may be overwritten by the next column
  }

  // ---- T (LAPACK larft, forward columnwise) ----------------------------
  // Z(i, j) = v_i^T v_j for i < j: partial over this CTA's rows; each thread
  // owns whole dot products (no cross-lane FP64 reductions: on this part the
  // FP64 pipe is the scarce resource)
  const int kk = kmax;
  const int nz = kk * (kk - 1) / 2;
  for (int idx = tid; idx < kk * kk; idx += kQrThreads) {
    const int i = idx % kk, jj = idx / kk;
    if (i >= jj) continue;
    double acc = 0.0;
    for (int r = max(jj - p0, 0); r < myrows; ++r) {
      const int pos = p0 + r;
      const double vi = tile[r + (size_t)i * ld];  // pos >= jj > i: stored entry of v_i
      const double vj = (pos == jj) ? 1.0 : tile[r + (size_t)jj * ld];
      acc = fma(vi, vj, acc);
    }
    Z[jj * (jj - 1) / 2 + i] = acc;
  }
  qr_sync(cl, G);
  if (rank == 0) {
    for (int idx = tid; idx < nz; idx += kQrThreads)
      for (int r = 1; r < G; ++r) Z[idx] += *cl.map_shared_rank(Z + idx, r);
  }
  qr_sync(cl, G);  // peers may exit after this
  if (rank == 0) {
    double *T = a.Tp + (size_t)(a.is_leaf ? node : a.nleaves + midx) * a.b * a.b;
    const int b = a.b;
    for (int idx = tid; idx < b * b; idx += kQrThreads) T[idx] = 0.0;
    __syncthreads();
    for (int jj = 0; jj < kk; ++jj) {
      const double tj = tau[jj];
      // T(i, jj) = -tau_jj * sum_{q=i}^{jj-1} T(i, q) Z(q, jj)
      for (int i = tid; i < jj; i += kQrThreads) {
        double s = 0.0;
        if (tj != 0.0)
          for (int q = i; q < jj; ++q) s = fma(T[i + (size_t)q * b], Z[jj * (jj - 1) / 2 + q], s);
        T[i + (size_t)jj * b] = -tj * s;
      }
      if (tid == 0) T[jj + (size_t)jj * b] = tj;
      __syncthreads();
    }
  }

  // ---- write back: leaf in place; merge: R into the first child's rows,
  //      Y blocks into the other children's rows (on and above the diagonal)
  for (int k = warp; k < bk; k += kQrWarps) {
    double *col = a.P + (size_t)k * a.lda;
    for (int i = lane; i < myrows; i += 32)
      if (k >= fz[i]) col[prw[i]] = tile[i + (size_t)k * ld];
  }
  if (rank == 0 && tid == 0) {
    a.top_out[node] = a.is_leaf ? r0 : a.top_in[start];
    a.c_out[node] = kmax;
  }
}

// @region tree_apply_kernel
// ---------------------------------------------------------------------------
// Tree update: C <- Q_node^T C for every node (leaves, then merge rounds).
// One CTA per (node, tile of kCt columns).  W = Y^T C accumulated in
// registers over row chunks, W <- T^T W, then C -= Y W over the same chunks.
// Y of a leaf: unit lower trapezoid stored in the panel rows; Y of a merge:
// the identity on the first child's rows and the stored upper trapezoids on
// the others (Sec. 3.1: UPFACT on the leaves, UPELIM on the merges).
// ---------------------------------------------------------------------------
constexpr int kCt = 32;       // columns per CTA
constexpr int kCs = kCt + 1;  // odd row stride of the C chunk in shared memory
constexpr int kChunk = 32;    // rows per chunk
constexpr int kApThreads = 256;

struct ApplyArgs {
  const double *P;
  int lda, mk, bk, b;
  int leaf_rows;
  int is_leaf;
  RoundDesc rd;
  const int *top_in, *c_in;
  int *top_out, *c_out;
  const double *Tp;
  int nleaves;
  double *C;
  int ldc, ncols;
};

// W[u][v] += sum over the chunk's rows of Y(i, kb + 32 u) C(i, cb + 8 v) for
// U0 <= u < U1 (the k-slices that hold nonzeros of Y in this chunk).
template <int U0, int U1>
__device__ __forceinline__ void accum_w(const double *Ys, const double *Cs, int nr, int ldy, int kb, int cb,
                                        int bk, double (&W)[4][4]) {
  for (int i = 0; i < nr; ++i) {
    double yv[4], cv[4];
#pragma unroll
    for (int u = U0; u < U1; ++u) yv[u] = (kb + 32 * u < bk) ? Ys[i * ldy + kb + 32 * u] : 0.0;
#pragma unroll
    for (int v = 0; v < 4; ++v) cv[v] = Cs[i * kCs + cb + 8 * v];
#pragma unroll
    for (int u = U0; u < U1; ++u)
#pragma unroll
      for (int v = 0; v < 4; ++v) W[u][v] = fma(yv[u], cv[v], W[u][v]);
  }
}

__global__ void __launch_bounds__(kApThreads, 1) tree_apply_kernel(ApplyArgs a) {
  extern __shared__ __align__(16) double asm_[];
  const int bk = a.bk;
  const int ldy = bk + 1;            // odd leading dimension (row-major Y chunk)
  double *Ys = asm_;                 // kChunk x ldy
  double *Cs = Ys + kChunk * ldy;    // kChunk x kCt (row-major, stride kCs)
  double *Ws = Cs + kChunk * kCs;    // bk x kCt
  double *Ts = Ws + (size_t)bk * kCt;  // bk x ldy (T, ld ldy)
  const int tid = threadIdx.x;
  const int node = blockIdx.x;
  const int c0 = blockIdx.y * kCt;
  const int ncl = min(kCt, a.ncols - c0);

  // segments of the node: {panel row of its first row, rows, type}
  // type 0 = leaf (unit lower trapezoid), 1 = identity, 2 = upper trapezoid
  int start = 0, cnt = 1, midx = 0, kk;
  int lrow0 = 0, lrows = 0;
  if (a.is_leaf) {
    lrow0 = node * a.leaf_rows;
    lrows = min(a.leaf_rows, a.mk - lrow0);
    kk = min(lrows, bk);
    if (blockIdx.y == 0 && tid == 0) {
      a.top_out[node] = lrow0;
      a.c_out[node] = kk;
    }
  } else {
    round_node(a.rd, node, start, cnt, midx);
    int R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.c_in[start + ch];
    kk = min(R, bk);
    if (blockIdx.y == 0 && tid == 0) {
      a.top_out[node] = a.top_in[start];
      a.c_out[node] = (cnt == 1) ? a.c_in[start] : kk;
    }
    if (cnt == 1) return;
  }
  const double *T = a.Tp + (size_t)(a.is_leaf ? node : a.nleaves + midx) * a.b * a.b;

  // W mapping: thread -> k = kb + 32 u (u < 4 for bk <= 128), c = cb + 8 v (v < 4)
  const int kb = tid & 31, cb = tid >> 5;
  double W[4][4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v) W[u][v] = 0.0;

  const int nseg = a.is_leaf ? 1 : cnt;
  // Software pipeline over row chunks: the next chunk's Y (and C) are loaded
  // into registers while the current chunk is multiplied from shared memory.
  constexpr int kYPer = kChunk * 128 / kApThreads;  // Y chunk elements per thread (bk <= 128)
  constexpr int kCPer = kChunk * kCt / kApThreads;  // C chunk elements per thread
  double py[kYPer], pc[kCPer];
  auto load_y = [&](int srow, int type, int r0, int nr) {
#pragma unroll
    for (int t = 0; t < kYPer; ++t) {
      const int idx = tid + t * kApThreads;
      const int i = idx % kChunk, k = idx / kChunk;  // rows fastest: coalesced column reads
      const int gi = r0 + i;
      double y = 0.0;
      if (i < nr && k < bk) {
        if (type == 0)
          y = (gi > k) ? a.P[srow + gi + (size_t)k * a.lda] : (gi == k ? 1.0 : 0.0);
        else
          y = (gi <= k) ? a.P[srow + gi + (size_t)k * a.lda] : 0.0;
      }
      py[t] = y;
    }
  };
  auto store_y = [&]() {
#pragma unroll
    for (int t = 0; t < kYPer; ++t) {
      const int idx = tid + t * kApThreads;
      const int i = idx % kChunk, k = idx / kChunk;
      if (k < bk) Ys[i * ldy + k] = py[t];
    }
  };
  auto load_c = [&](int srow, int r0, int nr) {
#pragma unroll
    for (int t = 0; t < kCPer; ++t) {
      const int idx = tid + t * kApThreads;
      const int i = idx % kChunk, c = idx / kChunk;
      pc[t] = (i < nr && c < ncl) ? a.C[srow + r0 + i + (size_t)(c0 + c) * a.ldc] : 0.0;
    }
  };
  auto store_c = [&]() {
#pragma unroll
    for (int t = 0; t < kCPer; ++t) {
      const int idx = tid + t * kApThreads;
      Cs[(idx % kChunk) * kCs + idx / kChunk] = pc[t];
    }
  };
  // ---- phase 1: W = Y^T C ---------------------------------------------
  for (int sg = 0; sg < nseg; ++sg) {
    int srow, srows, type;
    if (a.is_leaf) {
      srow = lrow0;
      srows = lrows;
      type = 0;
    } else {
      srow = a.top_in[start + sg];
      srows = a.c_in[start + sg];
      type = (sg == 0) ? 1 : 2;
    }
    if (type == 1) {  // identity block: W(k, :) += C(k, :)
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int k = kb + 32 * u;
        if (k >= srows) continue;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int c = cb + 8 * v;
          if (c < ncl) W[u][v] += a.C[srow + k + (size_t)(c0 + c) * a.ldc];
        }
      }
      continue;
    }
    load_y(srow, type, 0, min(kChunk, srows));
    load_c(srow, 0, min(kChunk, srows));
    for (int r0 = 0; r0 < srows; r0 += kChunk) {
      const int nr = min(kChunk, srows - r0);
      __syncthreads();
      store_y();
      store_c();
      __syncthreads();
      if (r0 + kChunk < srows) {
        load_y(srow, type, r0 + kChunk, min(kChunk, srows - r0 - kChunk));
        load_c(srow, r0 + kChunk, min(kChunk, srows - r0 - kChunk));
      }
      // Y of a leaf is unit lower trapezoidal (row gi has nonzeros at k <= gi),
      // a merge block upper trapezoidal (k >= gi): only k-slices u with
      // 32 u <= r0 + 31 (leaf) or 32 u + 31 >= r0 (merge) hold nonzeros
      const int uq = r0 >> 5;
      if (type == 0) {
        switch (uq) {
          case 0: accum_w<0, 1>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          case 1: accum_w<0, 2>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          case 2: accum_w<0, 3>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          default: accum_w<0, 4>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
        }
      } else {
        switch (uq) {
          case 0: accum_w<0, 4>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          case 1: accum_w<1, 4>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          case 2: accum_w<2, 4>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
          default: accum_w<3, 4>(Ys, Cs, nr, ldy, kb, cb, bk, W); break;
        }
      }
    }
  }
  // ---- phase 2: W <- T^T W ----------------------------------------------
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (kb + 32 * u < bk) Ws[(kb + 32 * u) * kCt + cb + 8 * v] = W[u][v];
  for (int idx = tid; idx < bk * bk; idx += kApThreads) {
    int l = idx % bk, k = idx / bk;
    Ts[l + (size_t)k * ldy] = (l <= k && l < kk && k < kk) ? T[l + (size_t)k * a.b] : 0.0;
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u) {
    const int k = kb + 32 * u;
    if (k >= bk) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      double s = 0.0;
      for (int l = 0; l <= k; ++l) s = fma(Ts[l + (size_t)k * ldy], Ws[l * kCt + cb + 8 * v], s);
      W[u][v] = s;
    }
  }
  __syncthreads();
#pragma unroll
  for (int u = 0; u < 4; ++u)
#pragma unroll
    for (int v = 0; v < 4; ++v)
      if (kb + 32 * u < bk) Ws[(kb + 32 * u) * kCt + cb + 8 * v] = W[u][v];
  __syncthreads();
  // ---- phase 3: C -= Y W --------------------------------------------------
  for (int sg = 0; sg < nseg; ++sg) {
    int srow, srows, type;
    if (a.is_leaf) {
      srow = lrow0;
      srows = lrows;
      type = 0;
    } else {
      srow = a.top_in[start + sg];
      srows = a.c_in[start + sg];
      type = (sg == 0) ? 1 : 2;
    }
    if (type == 1) {
      for (int idx = tid; idx < srows * ncl; idx += kApThreads) {
        int i = idx % srows, c = idx / srows;
        a.C[srow + i + (size_t)(c0 + c) * a.ldc] -= Ws[i * kCt + c];
      }
      continue;
    }
    load_y(srow, type, 0, min(kChunk, srows));
    for (int r0 = 0; r0 < srows; r0 += kChunk) {
      const int nr = min(kChunk, srows - r0);
      __syncthreads();
      store_y();
      __syncthreads();
      if (r0 + kChunk < srows) load_y(srow, type, r0 + kChunk, min(kChunk, srows - r0 - kChunk));
      // thread -> (row i = tid % 32, columns c = tid / 32 + 8 v)
      const int i = tid & 31;
      if (i < nr) {
        double acc[4] = {0.0, 0.0, 0.0, 0.0};
        // the chunk's nonzero columns of Y: k <= r0 + 31 (leaf), k >= r0 (merge)
        const int k_lo = (type == 2) ? r0 : 0;
        const int k_hi = (type == 0) ? min(bk, r0 + kChunk) : bk;
        for (int k = k_lo; k < k_hi; ++k) {
          const double y = Ys[i * ldy + k];
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[v] = fma(y, Ws[k * kCt + cb + 8 * v], acc[v]);
        }
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          int c = cb + 8 * v;
          if (c < ncl) a.C[srow + r0 + i + (size_t)(c0 + c) * a.ldc] -= acc[v];
        }
      }
    }
  }
}

// @endregion tree_apply_kernel
// @region tree_apply_narrow_kernel
// ---------------------------------------------------------------------------
// Narrow tree update: the operation of tree_apply_kernel on NC <= 8 columns
// per CTA, with the threads spread over the reflectors and the rows instead
// of over 32 columns, so that no multiply-add works on padding columns.  It
// serves Q^T B with few right-hand sides and updates whose 32-column tiles
// would not give every SM a CTA (the look-ahead update of the next panel's
// columns, the last panels).  Every FP64 multiply-add costs 16 cycles of an
// SM's FP64 pipe per warp, so only the multiply-adds executed matter.
//   phase 1: thread (k = tid % 128, row half h = tid / 128) sums
//            Y(i, k) C(i, :) over its 16 rows of each 32-row chunk;
//   phase 2: W <- T^T W, thread (k, column parity);
//   phase 3: thread (row i = tid % 32, k-slice q = tid / 32 of 16 reflectors)
//            sums Y(i, k) W(k, :) over its slice; the 8 slices are added in
//            shared memory and subtracted from C.
// ---------------------------------------------------------------------------
constexpr int kNcChunk = 32;

template <int NC>
__global__ void __launch_bounds__(kApThreads, 2) tree_apply_narrow_kernel(ApplyArgs a) {
  extern __shared__ __align__(16) double nsm_[];
  const int bk = a.bk;
  const int ldy = bk + 1;
  double *Ys = nsm_;                       // kNcChunk x ldy (row-major chunk of Y)
  double *Cs = Ys + kNcChunk * ldy;        // kNcChunk x NC
  double *Ws = Cs + kNcChunk * NC;         // 128 x NC
  double *red = Ws + 128 * NC;             // 8 x kNcChunk x NC (phase 3), 128 x NC (phase 1)
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int node = blockIdx.x;
  const int c0 = blockIdx.y * NC;
  const int ncl = min(NC, a.ncols - c0);

  int start = 0, cnt = 1, midx = 0, kk;
  int lrow0 = 0, lrows = 0;
  if (a.is_leaf) {
    lrow0 = node * a.leaf_rows;
    lrows = min(a.leaf_rows, a.mk - lrow0);
    kk = min(lrows, bk);
    if (blockIdx.y == 0 && tid == 0) {
      a.top_out[node] = lrow0;
      a.c_out[node] = kk;
    }
  } else {
    round_node(a.rd, node, start, cnt, midx);
    int R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.c_in[start + ch];
    kk = min(R, bk);
    if (blockIdx.y == 0 && tid == 0) {
      a.top_out[node] = a.top_in[start];
      a.c_out[node] = (cnt == 1) ? a.c_in[start] : kk;
    }
    if (cnt == 1) return;
  }
  const double *T = a.Tp + (size_t)(a.is_leaf ? node : a.nleaves + midx) * a.b * a.b;
  const int nseg = a.is_leaf ? 1 : cnt;
  auto segment = [&](int sg, int &srow, int &srows, int &type) {
    if (a.is_leaf) {
      srow = lrow0;
      srows = lrows;
      type = 0;
    } else {
      srow = a.top_in[start + sg];
      srows = a.c_in[start + sg];
      type = (sg == 0) ? 1 : 2;
    }
  };
  // Y chunk (rows r0 .. r0 + nr - 1 of the segment) into Ys, rows fastest
  // (coalesced column reads); zero outside the stored structure
  auto stage_y = [&](int srow, int type, int r0, int nr) {
    for (int idx = tid; idx < kNcChunk * bk; idx += kApThreads) {
      const int i = idx % kNcChunk, k = idx / kNcChunk;
      const int gi = r0 + i;
      double y = 0.0;
      if (i < nr) {
        if (type == 0)
          y = (gi > k) ? a.P[srow + gi + (size_t)k * a.lda] : (gi == k ? 1.0 : 0.0);
        else
          y = (gi <= k) ? a.P[srow + gi + (size_t)k * a.lda] : 0.0;
      }
      Ys[i * ldy + k] = y;
    }
  };

  // ---- phase 1: W = Y^T C ---------------------------------------------
  const int k1 = tid & 127, h1 = tid >> 7;
  const int ks1 = 32 * ((tid >> 5) & 3);  // first reflector of this warp's slice
  double acc[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) acc[c] = 0.0;
  for (int sg = 0; sg < nseg; ++sg) {
    int srow, srows, type;
    segment(sg, srow, srows, type);
    if (type == 1) {  // identity block: W(k, :) += C(k, :)
      if (h1 == 0 && k1 < srows) {
#pragma unroll
        for (int c = 0; c < NC; ++c)
          if (c < ncl) acc[c] += a.C[srow + k1 + (size_t)(c0 + c) * a.ldc];
      }
      continue;
    }
    for (int r0 = 0; r0 < srows; r0 += kNcChunk) {
      const int nr = min(kNcChunk, srows - r0);
      __syncthreads();
      stage_y(srow, type, r0, nr);
      for (int idx = tid; idx < kNcChunk * NC; idx += kApThreads) {
        const int i = idx % kNcChunk, c = idx / kNcChunk;
        Cs[i * NC + c] = (i < nr && c < ncl) ? a.C[srow + r0 + i + (size_t)(c0 + c) * a.ldc] : 0.0;
      }
      __syncthreads();
      // rows of this thread: r0 + 16 h1 .. r0 + 16 h1 + 15; the warp's slice
      // holds nonzeros only if some k >= ks1 is <= the last row (leaf,
      // unit lower) or some k <= ks1 + 31 is >= the first row (merge, upper)
      const int i0 = 16 * h1, i1 = min(16 * h1 + 16, nr);
      const bool live = k1 < bk && i0 < i1 &&
                        (type == 0 ? ks1 <= r0 + i1 - 1 : ks1 + 31 >= r0 + i0);
      if (live) {
        for (int i = i0; i < i1; ++i) {
          const double y = Ys[i * ldy + k1];
#pragma unroll
          for (int c = 0; c < NC; ++c) acc[c] = fma(y, Cs[i * NC + c], acc[c]);
        }
      }
    }
  }
  __syncthreads();
  if (h1 == 1) {
#pragma unroll
    for (int c = 0; c < NC; ++c) red[k1 * NC + c] = acc[c];
  }
  __syncthreads();
  if (h1 == 0) {
#pragma unroll
    for (int c = 0; c < NC; ++c) Ws[k1 * NC + c] = acc[c] + red[k1 * NC + c];
  }
  __syncthreads();

  // ---- phase 2: W <- T^T W (T upper triangular, kk x kk) ------------------
  double s[NC];
#pragma unroll
  for (int c = 0; c < NC; ++c) s[c] = 0.0;
  if (k1 < kk) {
    const double *Tk = T + (size_t)k1 * a.b;
    for (int l = 0; l <= k1; ++l) {
      const double t = __ldg(Tk + l);
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if ((c & 1) == h1) s[c] = fma(t, Ws[l * NC + c], s[c]);
    }
  }
  __syncthreads();
#pragma unroll
  for (int c = 0; c < NC; ++c)
    if ((c & 1) == h1) Ws[k1 * NC + c] = s[c];  // zero for k >= kk
  __syncthreads();

  // ---- phase 3: C -= Y W ----------------------------------------------------
  const int kq = 16 * warp;  // this warp's 16 reflectors
  for (int sg = 0; sg < nseg; ++sg) {
    int srow, srows, type;
    segment(sg, srow, srows, type);
    if (type == 1) {
      for (int idx = tid; idx < srows * ncl; idx += kApThreads) {
        const int i = idx % srows, c = idx / srows;
        a.C[srow + i + (size_t)(c0 + c) * a.ldc] -= Ws[i * NC + c];
      }
      continue;
    }
    for (int r0 = 0; r0 < srows; r0 += kNcChunk) {
      const int nr = min(kNcChunk, srows - r0);
      __syncthreads();
      stage_y(srow, type, r0, nr);
      __syncthreads();
      // nonzero reflectors of the chunk: k <= r0 + 31 (leaf), k >= r0 (merge)
      const int k_lo = max(kq, type == 2 ? r0 : 0);
      const int k_hi = min(min(kq + 16, bk), type == 0 ? r0 + kNcChunk : bk);
      double p[NC];
#pragma unroll
      for (int c = 0; c < NC; ++c) p[c] = 0.0;
      if (lane < nr) {
        for (int k = k_lo; k < k_hi; ++k) {
          const double y = Ys[lane * ldy + k];
#pragma unroll
          for (int c = 0; c < NC; ++c) p[c] = fma(y, Ws[k * NC + c], p[c]);
        }
      }
#pragma unroll
      for (int c = 0; c < NC; ++c) red[(warp * kNcChunk + lane) * NC + c] = p[c];
      __syncthreads();
      for (int o = tid; o < kNcChunk * NC; o += kApThreads) {
        const int i = o % kNcChunk, c = o / kNcChunk;
        if (i < nr && c < ncl) {
          double v = 0.0;
#pragma unroll
          for (int q = 0; q < kApThreads / 32; ++q) v += red[(q * kNcChunk + i) * NC + c];
          a.C[srow + r0 + i + (size_t)(c0 + c) * a.ldc] -= v;
        }
      }
    }
  }
}

size_t narrow_smem_bytes(int bk, int nc) {
  return ((size_t)kNcChunk * (bk + 1) + kNcChunk * nc + 128 * nc + (size_t)(kApThreads / 32) * kNcChunk * nc) * 8;
}

// @endregion tree_apply_narrow_kernel
// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t qr_panel_ws_bytes(int nleaves_max) { return 4 * align256((size_t)nleaves_max * 4); }

void qr_panel_ws_carve(void *work, int nleaves_max, QrPanelWs &ws) {
  char *p = (char *)work;
  for (int i = 0; i < 2; ++i) {
    ws.top[i] = (int *)p;
    p += align256((size_t)nleaves_max * 4);
    ws.c[i] = (int *)p;
    p += align256((size_t)nleaves_max * 4);
  }
}

static int pick_qr_cluster(int R, int bk, int nodes, int *rloc, int *ld) {
  int G = 1;
  auto fits = [&](int g) {
    int rl = (R + g - 1) / g;
    return tsqr_smem_bytes(rl, rl | 1, bk) <= kQrSmemBudget;
  };
  while (G < 8 && !fits(G)) G *= 2;
  while (G < 8 && nodes * G * 2 <= 152 && (R + 2 * G - 1) / (2 * G) >= 32) G *= 2;
  if (!fits(G)) return -1;
  *rloc = (R + G - 1) / G;
  *ld = *rloc | 1;
  return G;
}

static cudaError_t launch_tsqr_node(const TsqrNodeArgs &args, int nodes, int G, cudaStream_t st) {
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(tsqr_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kQrSmemBudget + 4096);
  });
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  const double r = args.is_leaf ? (args.leaf_rows < args.mk ? args.leaf_rows : args.mk)
                                : (double)args.rd.max_cnt * args.bk;
  const double c = args.bk;
  // Householder QR (2 r c^2 - 2 c^3 / 3) plus T (r c^2 / ... about r c^2)
  ProfScope ps(kClsTsqrNode, st, nodes * (2.0 * r * c * c - 2.0 * c * c * c / 3.0 + r * c * c));
  if (G == 0) {  // the node fits the registers of one CTA
    bool done = false;
    e = launch_tsqr_reg(args, nodes, (int)r, st, &done);
    return (e == cudaSuccess && !done) ? cudaErrorInvalidValue : e;
  }
  if (G < 0) return launch_tsqr_creg(args, nodes, (int)r, st);  // registers of a cluster
  cfg.gridDim = dim3(nodes * G);
  cfg.blockDim = dim3(kQrThreads);
  cfg.dynamicSmemBytes = tsqr_smem_bytes(args.rloc, args.ld, args.bk);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tsqr_node_kernel, args);
}

cudaError_t tsqr_panel(int mk, int bk, int b, double *P, int lda, int leaf_rows, const Plan &plan,
                       double *Tp, const QrPanelWs &ws, int *dev_info, cudaStream_t st) {
  TsqrNodeArgs a = {};
  a.P = P;
  a.lda = lda;
  a.mk = mk;
  a.bk = bk;
  a.b = b;
  a.leaf_rows = leaf_rows;
  a.Tp = Tp;
  a.nleaves = plan.nleaves;
  a.dev_info = dev_info;
  int R = leaf_rows < mk ? leaf_rows : mk;
  int rloc = 0, ld = 0;
  // G = 0: the register-resident node kernel; -1: its cluster form; else
  // the shared-memory node kernel on a cluster of G CTAs
  auto pick = [&](int rows, int nodes) {
    if (tsqr_reg_fits(rows, bk)) return 0;
    if (tsqr_creg_cluster(rows, bk) >= 2) return -1;
    const int g = pick_qr_cluster(rows, bk, nodes, &rloc, &ld);
    return g > 0 ? g : -2;
  };
  int G = pick(R, plan.nleaves);
  if (G == -2) return cudaErrorInvalidValue;
  a.is_leaf = 1;
  a.rloc = rloc;
  a.ld = ld;
  a.top_out = ws.top[0];
  a.c_out = ws.c[0];
  cudaError_t e = launch_tsqr_node(a, plan.nleaves, G, st);
  if (e != cudaSuccess) return e;
  int buf = 0;
  for (int r = 0; r < plan.nrounds; ++r) {
    const RoundDesc &rd = plan.r[r];
    G = pick(rd.max_cnt * bk, rd.n_out);
    if (G == -2) return cudaErrorInvalidValue;
    a.is_leaf = 0;
    a.rd = rd;
    a.rloc = rloc;
    a.ld = ld;
    a.top_in = ws.top[buf];
    a.c_in = ws.c[buf];
    a.top_out = ws.top[buf ^ 1];
    a.c_out = ws.c[buf ^ 1];
    e = launch_tsqr_node(a, rd.n_out, G, st);
    if (e != cudaSuccess) return e;
    buf ^= 1;
  }
  return cudaSuccess;
}

cudaError_t tree_apply_qt(int mk, int bk, int b, const double *P, int lda, int leaf_rows,
                          const Plan &plan, const double *Tp, double *C, int ldc, int ncols,
                          const QrPanelWs &ws, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  if (bk > 128) return cudaErrorInvalidValue;
  const int ldy = bk + 1;
  size_t smem = ((size_t)kChunk * ldy + kChunk * kCs + (size_t)bk * kCt + (size_t)bk * ldy) * 8;
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    const size_t most = ((size_t)kChunk * 129 + kChunk * kCs + 128 * kCt + 128 * 129) * 8;
    const int nmost = (int)narrow_smem_bytes(128, 8);
    const cudaFuncAttribute a = cudaFuncAttributeMaxDynamicSharedMemorySize;
    cudaError_t r;
    if ((r = cudaFuncSetAttribute(tree_apply_kernel, a, (int)most)) != cudaSuccess ||
        (r = cudaFuncSetAttribute(tree_apply_narrow_kernel<1>, a, nmost)) != cudaSuccess ||
        (r = cudaFuncSetAttribute(tree_apply_narrow_kernel<2>, a, nmost)) != cudaSuccess ||
        (r = cudaFuncSetAttribute(tree_apply_narrow_kernel<4>, a, nmost)) != cudaSuccess)
      return r;
    return cudaFuncSetAttribute(tree_apply_narrow_kernel<8>, a, nmost);
  });
  if (e != cudaSuccess) return e;
  int sms = 0;
  if ((e = device_sm_count(&sms)) != cudaSuccess) return e;
  ApplyArgs a = {};
  a.P = P;
  a.lda = lda;
  a.mk = mk;
  a.bk = bk;
  a.b = b;
  a.leaf_rows = leaf_rows;
  a.Tp = Tp;
  a.nleaves = plan.nleaves;
  a.C = C;
  a.ldc = ldc;
  a.ncols = ncols;
  const int ntiles = (ncols + kCt - 1) / kCt;
  // narrow kernel for a few columns, or when the 32-column tiles of the leaf
  // update would leave SMs without a CTA
  const int nc = ncols <= 1 ? 1 : ncols <= 2 ? 2 : ncols <= 4 ? 4 : 8;
  const bool narrow = ncols <= 8 || (long long)plan.nleaves * ntiles < sms;
  const int gy = narrow ? (ncols + nc - 1) / nc : ntiles;
  const size_t nsmem = narrow_smem_bytes(bk, nc);
  auto launch = [&](int gx) {
    const dim3 grid(gx, gy);
    if (!narrow)
      tree_apply_kernel<<<grid, kApThreads, smem, st>>>(a);
    else if (nc == 1)
      tree_apply_narrow_kernel<1><<<grid, kApThreads, nsmem, st>>>(a);
    else if (nc == 2)
      tree_apply_narrow_kernel<2><<<grid, kApThreads, nsmem, st>>>(a);
    else if (nc == 4)
      tree_apply_narrow_kernel<4><<<grid, kApThreads, nsmem, st>>>(a);
    else
      tree_apply_narrow_kernel<8><<<grid, kApThreads, nsmem, st>>>(a);
  };
  a.is_leaf = 1;
  a.top_out = ws.top[0];
  a.c_out = ws.c[0];
  {
    // W = Y^T C and C -= Y W over the nonzeros of every leaf's unit lower
    // trapezoid Y (rows x k, k = min(rows, bk)), and W = T^T W (triangular)
    double f = 0.0;
    for (int j = 0; j < plan.nleaves; ++j) {
      const double r = (double)(leaf_rows < mk - j * leaf_rows ? leaf_rows : mk - j * leaf_rows);
      const double k = r < bk ? r : bk;
      f += (4.0 * (r * k - k * (k - 1) / 2.0) + k * (k + 1)) * ncols;
    }
    ProfScope ps(narrow ? kClsTreeNarrow : kClsTreeApply, st, f);
    launch(plan.nleaves);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  int buf = 0;
  for (int r = 0; r < plan.nrounds; ++r) {
    a.is_leaf = 0;
    a.rd = plan.r[r];
    a.top_in = ws.top[buf];
    a.c_in = ws.c[buf];
    a.top_out = ws.top[buf ^ 1];
    a.c_out = ws.c[buf ^ 1];
    {
      // each merge: the non-first children's upper triangular Y blocks
      // (bk x bk, bk (bk + 1) / 2 nonzeros each), W = T^T W (triangular),
      // and the first child's identity block (one add and one subtract)
      const RoundDesc &rd = plan.r[r];
      double f = 0.0;
      const double kb2 = (double)bk;
      for (int o = 0; o < rd.n_out; ++o) {
        int s0, cnt, mi;
        round_node(rd, o, s0, cnt, mi);
        if (cnt >= 2) f += (4.0 * (cnt - 1) * kb2 * (kb2 + 1) / 2.0 + kb2 * (kb2 + 1) + 2.0 * kb2) * ncols;
      }
      ProfScope ps(narrow ? kClsTreeNarrow : kClsTreeApply, st, f);
      launch(plan.r[r].n_out);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    buf ^= 1;
  }
  return cudaSuccess;
}

}  // namespace cagb

namespace cagb {
bool qr_node_feasible(int rows, int bk) {
  int rloc, ld;
  return bk <= 128 && pick_qr_cluster(rows, bk, 1 << 20, &rloc, &ld) > 0;
}
}  // namespace cagb
