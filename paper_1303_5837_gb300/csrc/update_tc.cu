// update_tc.cu -- the CAQR tree update (UPFACT on the leaves, UPELIM on the
// merges, Sec. 3.1 / Algorithm ML-CAQR) with its three contractions on the
// tensor cores:
//     W = Y^T C,   W' = T^T W,   C -= Y W'
// for every leaf (Y unit lower trapezoidal in the leaf's rows) and every merge
// node (Y = [I; Y_1; ...], Y_i upper trapezoidal in child i's R rows; the
// identity block is an FP64 copy and subtraction).  Each contraction is one
// batched launch of gemm_tc over a chunk of tree nodes; the FP64 digit split
// of the operands is done per node, so accuracy is that of gemm_tc's mode
// (7 exact digits: the FP64 level).
#include "ca_internal.cuh"

namespace cagb {

constexpr int kChunkLeaves = 16;   // tree nodes per batched launch
constexpr int kHalfK = 128;        // contraction length per exact launch

// For merge round rd: item arrays in merge order (item = midx - merge_base)
// and the next round's (top, c) for every output.
__global__ void merge_items_kernel(RoundDesc rd, const int *top_in, const int *c_in, int *top_out, int *c_out,
                                   int *it_top0, int *it_top, int *it_c, int maxc, int bk) {
  const int o = blockIdx.x * blockDim.x + threadIdx.x;
  if (o >= rd.n_out) return;
  int start, cnt, midx;
  round_node(rd, o, start, cnt, midx);
  if (cnt >= 2) {
    const int b = midx - rd.merge_base;
    const int nitems = rd.n_out;  // stride of the per-child arrays (>= merges)
    it_top0[b] = top_in[start];
    for (int ci = 1; ci < maxc; ++ci) {
      it_top[(ci - 1) * nitems + b] = (ci < cnt) ? top_in[start + ci] : 0;
      it_c[(ci - 1) * nitems + b] = (ci < cnt) ? c_in[start + ci] : 0;
    }
    int R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += c_in[start + ch];
    top_out[o] = top_in[start];
    c_out[o] = R < bk ? R : bk;
  } else {
    top_out[o] = top_in[start];
    c_out[o] = c_in[start];
  }
}

// W_b(r, c) = C(top0[b] + r, c), r < bk  (the identity block of a merge's Y);
// grid (column blocks of 8, items), one warp per column
__global__ void gather_rows_kernel(int bk, int ncols, const double *C, int ldc, const int *top0, double *W) {
  const int b = blockIdx.y;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= ncols) return;
  const double *src = C + top0[b] + (size_t)c * ldc;
  double *dst = W + ((size_t)b * ncols + c) * bk;
  for (int r = threadIdx.x & 31; r < bk; r += 32) dst[r] = src[r];
}

// C(top0[b] + r, c) -= W'_b(r, c)
__global__ void sub_rows_kernel(int bk, int ncols, double *C, int ldc, const int *top0, const double *Wp) {
  const int b = blockIdx.y;
  const int c = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (c >= ncols) return;
  double *dst = C + top0[b] + (size_t)c * ldc;
  const double *src = Wp + ((size_t)b * ncols + c) * bk;
  for (int r = threadIdx.x & 31; r < bk; r += 32) dst[r] -= src[r];
}

__global__ void leaf_items_kernel(int nleaves, int L, int mk, int bk, int *top, int *c) {
  const int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= nleaves) return;
  const int rows = min(L, mk - j * L);
  top[j] = j * L;
  c[j] = rows < bk ? rows : bk;
}

size_t tree_tc_ws_bytes(int mk, int bk, int ncols, int leaf_rows, int nleaves, int S) {
  const int ch = kChunkLeaves;
  const size_t w = (size_t)ch * bk * ncols * 8;
  size_t g = tc_gemm_ws_bytes_batched(bk, ncols, kHalfK, S, ch);           // W = Y^T C (per half)
  g = g > tc_gemm_ws_bytes_batched(leaf_rows, ncols, bk, S, ch) ? g
                                                                   : tc_gemm_ws_bytes_batched(leaf_rows, ncols, bk, S, ch);
  const size_t items = 3 * align256((size_t)(nleaves + 1) * 4 * 8);
  (void)mk;
  return 2 * align256(w) + align256(g) + items + 256;
}

cudaError_t tree_apply_qt_tc(int mk, int bk, int b, const double *P, int lda, int leaf_rows, const Plan &plan,
                             const double *Tp, double *C, int ldc, int ncols, const QrPanelWs &ws, void *tcws,
                             int S, int exact, int *status, cudaStream_t st) {
  if (ncols <= 0) return cudaSuccess;
  const int L = leaf_rows, nl = plan.nleaves;
  const int ch = kChunkLeaves;
  char *p = (char *)(((uintptr_t)tcws + 255) & ~(uintptr_t)255);
  double *W = (double *)p;
  p += align256((size_t)ch * bk * ncols * 8);
  double *Wp = (double *)p;
  p += align256((size_t)ch * bk * ncols * 8);
  size_t g = tc_gemm_ws_bytes_batched(bk, ncols, kHalfK, S, ch);
  const size_t g3 = tc_gemm_ws_bytes_batched(L, ncols, bk, S, ch);
  if (g3 > g) g = g3;
  void *gws = p;
  p += align256(g);
  int *it_top0 = (int *)p;
  p += align256((size_t)(nl + 1) * 4 * 8);
  int *it_top = (int *)p;
  p += align256((size_t)(nl + 1) * 4 * 8);
  int *it_c = (int *)p;
  const size_t wbytes = (size_t)ch * bk * ncols * 8;
  cudaError_t e;

  // ---- leaves (UPFACT) ----------------------------------------------------
  {
    ProfScope ps(kClsTreeApply, st, 0.0);
    leaf_items_kernel<<<(nl + 255) / 256, 256, 0, st>>>(nl, L, mk, bk, ws.top[0], ws.c[0]);
  }
  for (int j0 = 0; j0 < nl; j0 += ch) {
    const int nb = (nl - j0 < ch) ? nl - j0 : ch;
    const bool has_last = (j0 + nb == nl);
    const int L_last = has_last ? mk - (nl - 1) * L : L;
    const int kk = L < bk ? L : bk;
    const int kk_last = L_last < bk ? L_last : bk;
    if ((e = cudaMemsetAsync(W, 0, wbytes, st)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(Wp, 0, wbytes, st)) != cudaSuccess) return e;
    // W = Y^T C, in contraction halves of 128 leaf rows
    for (int h = 0; h * kHalfK < L; ++h) {
      TcGemm g1 = {};
      g1.A.X = P + (size_t)j0 * L + h * kHalfK;
      g1.A.sv = lda;
      g1.A.sk = 1;
      g1.A.sb = L;
      g1.A.nv = kk;
      g1.A.nv_last = kk_last;
      g1.A.K = (L - h * kHalfK < kHalfK) ? L - h * kHalfK : kHalfK;
      int kl = L_last - h * kHalfK;
      g1.A.K_last = kl < 0 ? 0 : (kl < kHalfK ? kl : kHalfK);
      g1.A.shape = 1;  // unit lower: Y(r, q), r = leaf row
      g1.A.trans = 1;
      g1.A.roff = h * kHalfK;
      g1.B = g1.A;
      g1.B.X = C + (size_t)j0 * L + h * kHalfK;
      g1.B.sv = ldc;
      g1.B.nv = g1.B.nv_last = ncols;
      g1.B.shape = 0;
      g1.B.trans = 0;
      g1.B.roff = 0;
      g1.nbatch = nb;
      g1.C = W;
      g1.ldc = bk;
      g1.sbc = (long long)bk * ncols;
      g1.sign = -1.0;
      g1.S = S;
      g1.exact = exact;
      if ((e = gemm_tc(g1, gws, status, st)) != cudaSuccess) return e;
    }
    // W' = T^T W
    TcGemm g2 = {};
    g2.A.X = Tp + (size_t)j0 * b * b;
    g2.A.sv = b;
    g2.A.sk = 1;
    g2.A.sb = (long long)b * b;
    g2.A.nv = kk;
    g2.A.nv_last = kk_last;
    g2.A.K = kk;
    g2.A.K_last = kk_last;
    g2.B.X = W;
    g2.B.sv = bk;
    g2.B.sk = 1;
    g2.B.sb = (long long)bk * ncols;
    g2.B.nv = g2.B.nv_last = ncols;
    g2.B.K = kk;
    g2.B.K_last = kk_last;
    g2.nbatch = nb;
    g2.C = Wp;
    g2.ldc = bk;
    g2.sbc = (long long)bk * ncols;
    g2.sign = -1.0;
    g2.S = S;
    g2.exact = exact;
    if ((e = gemm_tc(g2, gws, status, st)) != cudaSuccess) return e;
    // C -= Y W'
    TcGemm g3 = {};
    g3.A.X = P + (size_t)j0 * L;
    g3.A.sv = 1;
    g3.A.sk = lda;
    g3.A.sb = L;
    g3.A.nv = L;
    g3.A.nv_last = L_last;
    g3.A.K = kk;
    g3.A.K_last = kk_last;
    g3.A.shape = 1;
    g3.B = g2.B;
    g3.B.X = Wp;
    g3.nbatch = nb;
    g3.C = C + (size_t)j0 * L;
    g3.ldc = ldc;
    g3.sbc = L;
    g3.sign = 1.0;
    g3.S = S;
    g3.exact = exact;
    if ((e = gemm_tc(g3, gws, status, st)) != cudaSuccess) return e;
  }

  // ---- merges (UPELIM), bottom-up -----------------------------------------
  int buf = 0;
  for (int r = 0; r < plan.nrounds; ++r) {
    const RoundDesc &rd = plan.r[r];
    const int maxc = rd.max_cnt;
    int nmerge = 0;
    for (int o = 0; o < rd.n_out; ++o) {
      int s0, cnt, mi;
      round_node(rd, o, s0, cnt, mi);
      if (cnt >= 2) ++nmerge;
    }
    {
      ProfScope ps(kClsTreeApply, st, 0.0);
      merge_items_kernel<<<(rd.n_out + 127) / 128, 128, 0, st>>>(rd, ws.top[buf], ws.c[buf], ws.top[buf ^ 1],
                                                                 ws.c[buf ^ 1], it_top0, it_top, it_c, maxc, bk);
    }
    for (int i0 = 0; i0 < nmerge; i0 += ch) {
      const int nb = (nmerge - i0 < ch) ? nmerge - i0 : ch;
      if ((e = cudaMemsetAsync(Wp, 0, wbytes, st)) != cudaSuccess) return e;
      {
        ProfScope ps(kClsTreeApply, st, 0.0);
        gather_rows_kernel<<<dim3((ncols + 7) / 8, nb), 256, 0, st>>>(bk, ncols, C, ldc, it_top0 + i0, W);
      }
      for (int ci = 1; ci < maxc; ++ci) {
        const int *top_ci = it_top + (size_t)(ci - 1) * rd.n_out + i0;
        const int *c_ci = it_c + (size_t)(ci - 1) * rd.n_out + i0;
        TcGemm g1 = {};
        g1.A.X = P;  // Y_ci^T: element (q, t) = Y_ci(t, q), t <= q, in child ci's R rows
        g1.A.sv = lda;
        g1.A.sk = 1;
        g1.A.off = top_ci;
        g1.A.nv = g1.A.nv_last = bk;
        g1.A.K = g1.A.K_last = bk;
        g1.A.K_item = c_ci;
        g1.A.shape = 2;
        g1.A.trans = 1;
        g1.B.X = C;
        g1.B.sv = ldc;
        g1.B.sk = 1;
        g1.B.off = top_ci;
        g1.B.nv = g1.B.nv_last = ncols;
        g1.B.K = g1.B.K_last = bk;
        g1.B.K_item = c_ci;
        g1.nbatch = nb;
        g1.C = W;
        g1.ldc = bk;
        g1.sbc = (long long)bk * ncols;
        g1.sign = -1.0;
        g1.S = S;
        g1.exact = exact;
        if ((e = gemm_tc(g1, gws, status, st)) != cudaSuccess) return e;
      }
      TcGemm g2 = {};
      g2.A.X = Tp + (size_t)(nl + rd.merge_base + i0) * b * b;
      g2.A.sv = b;
      g2.A.sk = 1;
      g2.A.sb = (long long)b * b;
      g2.A.nv = g2.A.nv_last = bk;
      g2.A.K = g2.A.K_last = bk;
      g2.B.X = W;
      g2.B.sv = bk;
      g2.B.sk = 1;
      g2.B.sb = (long long)bk * ncols;
      g2.B.nv = g2.B.nv_last = ncols;
      g2.B.K = g2.B.K_last = bk;
      g2.nbatch = nb;
      g2.C = Wp;
      g2.ldc = bk;
      g2.sbc = (long long)bk * ncols;
      g2.sign = -1.0;
      g2.S = S;
      g2.exact = exact;
      if ((e = gemm_tc(g2, gws, status, st)) != cudaSuccess) return e;
      {
        ProfScope ps(kClsTreeApply, st, 0.0);
        sub_rows_kernel<<<dim3((ncols + 7) / 8, nb), 256, 0, st>>>(bk, ncols, C, ldc, it_top0 + i0, Wp);
      }
      for (int ci = 1; ci < maxc; ++ci) {
        const int *top_ci = it_top + (size_t)(ci - 1) * rd.n_out + i0;
        const int *c_ci = it_c + (size_t)(ci - 1) * rd.n_out + i0;
        TcGemm g3 = {};
        g3.A.X = P;  // Y_ci: element (t, q), t <= q
        g3.A.sv = 1;
        g3.A.sk = lda;
        g3.A.off = top_ci;
        g3.A.nv = g3.A.nv_last = bk;
        g3.A.nv_item = c_ci;
        g3.A.K = g3.A.K_last = bk;
        g3.A.shape = 2;
        g3.B = g2.B;
        g3.B.X = Wp;
        g3.nbatch = nb;
        g3.C = C;
        g3.ldc = ldc;
        g3.coff = top_ci;
        g3.sign = 1.0;
        g3.S = S;
        g3.exact = exact;
        if ((e = gemm_tc(g3, gws, status, st)) != cudaSuccess) return e;
      }
    }
    // the item arrays are rewritten by the next round only after this
    // round's launches (stream order)
    buf ^= 1;
  }
  return cudaSuccess;
}

}  // namespace cagb
