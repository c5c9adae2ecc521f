// batched.cu -- many small, uneven CALU / CAQR factorizations in one
// persistent launch.
//
// One CTA factors one whole matrix at a time: it takes the next item of an
// LPT-ordered list (largest flop count first) from a device counter, runs the
// item's CALU or CAQR panel loop with the item's own panel width and tree,
// and moves on.  Every tree node lives in the CTA's shared memory; the
// trailing updates run from global memory (L2-resident for these sizes)
// through shared-memory tiles.  The numerics are those of calu_factor /
// caqr_factor: the same tree (Sec. 3.1 / 3.2), GEPP with the first-maximum
// rule at every node, LAPACK larfg / larft Householder conventions and the
// same tree storage of Y and T, in FP64 or FP32.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {
namespace {

constexpr int kBT = 256;  // threads per CTA
constexpr int kBW = kBT / 32;
constexpr int kBMaxRows = 1024;  // rows of a node tile
constexpr int kBMaxB = 128;      // widest panel
constexpr int kBMultiB = 64;     // widest panel when a trailing update follows
constexpr int kTl = 64;          // tile of the trailing updates (rows and columns)
constexpr int kTs = kTl + 1;     // odd stride of those tiles
constexpr int kGk = 32;          // k chunk of the Schur-complement tile
constexpr unsigned kPlanMagic = 0x43414231u;

struct BatchHeader {
  unsigned magic;
  int count, dtype, ctas;
  int smem_region;  // bytes of the phase region (after the fixed part)
  int pad;
  size_t slot_bytes;
  size_t work_bytes;
  double flops;
};
constexpr size_t kHeaderBytes = 256;

template <class T>
struct Num;
template <>
struct Num<double> {
  static __device__ __forceinline__ unsigned long long key(double x) {
    return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
  }
  static __device__ __forceinline__ bool bad(double x) { return not_finite(x); }
  static __device__ __forceinline__ double root(double x) { return sqrt(x); }
};
template <>
struct Num<float> {
  static __device__ __forceinline__ unsigned long long key(float x) {
    return (unsigned long long)(__float_as_uint(x) & 0x7fffffffu);
  }
  static __device__ __forceinline__ bool bad(float x) {
    return (__float_as_uint(x) & 0x7f800000u) == 0x7f800000u;
  }
  static __device__ __forceinline__ float root(float x) { return sqrtf(x); }
};

template <class T>
__device__ __forceinline__ T wsum(T v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// Fixed part of shared memory (the phase region follows it).
template <class T>
struct Fixed {
  Plan plan;
  int prow[kBMaxRows];  // panel row of each node row
  int fz[kBMaxRows];    // merge rows: child-local index t (zeros left of column t);
                        // LU with the 2D operator: labels of the level-1 scratch rows
  int lab2[kBMaxRows];  // labels of the level-2 scratch rows (2D operator)
  int sel[kBMaxB], rev_top[kBMaxB], top_c[kBMaxB], far_c[kBMaxB];
  int perm_src[2 * kBMaxB], perm_dst[2 * kBMaxB];
  int iscal[16];
  ArgMax wbest[kBW];
  T tau[kBMaxB], w[kBMaxB], z[kBMaxB];
  T red[kBW];
  T scal[8];
  int item, nperm, info0, status;
};

__host__ __device__ inline size_t fixed_bytes(int dtype) {
  return ((dtype == CA_DTYPE_F32 ? sizeof(Fixed<float>) : sizeof(Fixed<double>)) + 15) & ~size_t(15);
}

__host__ __device__ inline int odd_ld(int rows) { return rows | 1; }

// Element-wise copy of `total` elements, ld(e) -> st(e, v): each thread
// issues the loads of kU elements before any of their stores, so that the
// latencies of the global loads overlap.
constexpr int kU = 8;
template <class T, class Ld, class St>
__device__ __forceinline__ void stage(int total, Ld ld, St st) {
  for (int base = threadIdx.x; base < total; base += kBT * kU) {
    T v[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = base + u * kBT;
      v[u] = (e < total) ? ld(e) : T(0);
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      const int e = base + u * kBT;
      if (e < total) st(e, v[u]);
    }
  }
}

// ---------------------------------------------------------------------------
// GEPP on the node tile (rows x bk, ld), rows permuted physically with their
// labels lab[]; first maximum of |a| in the current order.  Returns the
// number of steps, min(rows, bk).
// ---------------------------------------------------------------------------
template <class T>
__device__ int node_gepp(T *tile, int ld, int rows, int bk, int *lab, Fixed<T> &F, bool root, int kb) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kmax = min(rows, bk);
  for (int j = 0; j < kmax; ++j) {
    ArgMax best{0ull, INT_MAX};
    const T *cj = tile + (size_t)j * ld;
    for (int p = j + tid; p < rows; p += kBT) best = argmax_better(best, ArgMax{Num<T>::key(cj[p]), p});
    best = warp_argmax(best);
    if (lane == 0) F.wbest[warp] = best;
    __syncthreads();
    if (tid == 0) {
      ArgMax bb = F.wbest[0];
      for (int q = 1; q < kBW; ++q) bb = argmax_better(bb, F.wbest[q]);
      F.iscal[0] = bb.pos;
      F.iscal[1] = (bb.key == 0ull);
      if (bb.key == 0ull && root && F.info0 == 0) F.info0 = kb + j + 1;
      if (bb.key != 0ull) F.scal[0] = T(1) / cj[bb.pos];
    }
    __syncthreads();
    if (F.iscal[1]) continue;  // zero column: no swap, no update
    const int p = F.iscal[0];
    if (p != j) {
      for (int k = tid; k < bk; k += kBT) {
        T t = tile[p + (size_t)k * ld];
        tile[p + (size_t)k * ld] = tile[j + (size_t)k * ld];
        tile[j + (size_t)k * ld] = t;
      }
      if (tid == 0) {
        int t = lab[p];
        lab[p] = lab[j];
        lab[j] = t;
      }
      __syncthreads();
    }
    const T rinv = F.scal[0];
    T *cjw = tile + (size_t)j * ld;
    for (int q = j + 1 + tid; q < rows; q += kBT) cjw[q] *= rinv;
    __syncthreads();
    for (int k = j + 1 + warp; k < bk; k += kBW) {
      const T u = tile[j + (size_t)k * ld];
      T *ck = tile + (size_t)k * ld;
      for (int q = j + 1 + lane; q < rows; q += 32) ck[q] = fma(-cjw[q], u, ck[q]);
    }
    __syncthreads();
  }
  return kmax;
}

// ---------------------------------------------------------------------------
// The 2D multilevel CALU reduction operator (Algorithm 2D-ML-CALU): a node
// tile (rows x c, labels lab[]) is factored by CALU of the level below --
// panels of op_b[level] columns; each panel's pivots chosen by a tournament
// over leaves of op_leaf_rows[level] tile rows and a binary tree, whose
// nodes (copies of the current rows in the scratch tile scr) are factored by
// the operator one level further down (GEPP at the bottom); the chosen rows
// swapped to the top (all c columns, labels with them), then eliminated
// without further pivoting.  The first min(rows, c) labels are the node's
// pivot rows in pivot order and the top of the tile holds L \ U of them.
// wsi: the global candidate buffers of this level (and, after them, of the
// levels below).
// ---------------------------------------------------------------------------
// one level's buffers: two candidate lists (nodes x panel width <= 2 x
// kBMaxRows) and two count lists
constexpr int kOpCandList = 2 * kBMaxRows;
constexpr int kOpCand = 2 * kOpCandList + 2 * kBMaxRows;

// Elimination steps j0 <= j < j1 of the tile without pivot search (zero
// pivot: no scaling, no update; reported at the root).
template <class T>
__device__ void elim_nopiv(T *tile, int ld, int rows, int c, int j0, int j1, Fixed<T> &F, bool root, int kb) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  for (int j = j0; j < j1; ++j) {
    if (tid == 0) {
      const T piv = tile[j + (size_t)j * ld];
      F.iscal[1] = (piv == T(0));
      if (piv == T(0) && root && F.info0 == 0) F.info0 = kb + j + 1;
      if (piv != T(0)) F.scal[0] = T(1) / piv;
    }
    __syncthreads();
    if (F.iscal[1]) continue;
    const T rinv = F.scal[0];
    T *cj = tile + (size_t)j * ld;
    for (int q = j + 1 + tid; q < rows; q += kBT) cj[q] *= rinv;
    __syncthreads();
    for (int k = j + 1 + warp; k < c; k += kBW) {
      const T u = tile[j + (size_t)k * ld];
      T *ck = tile + (size_t)k * ld;
      for (int q = j + 1 + lane; q < rows; q += 32) ck[q] = fma(-cj[q], u, ck[q]);
    }
    __syncthreads();
  }
}

template <class T, int D>
__device__ int node_factor(T *tile, int ld, int rows, int c, int *lab, Fixed<T> &F, bool root, int kb,
                           const ca_tree_t &tr, int level, T *scr, int *wsi) {
  if constexpr (D == 0) {
    return node_gepp(tile, ld, rows, c, lab, F, root, kb);
  } else {
    const int tid = threadIdx.x;
    const int b1 = tr.op_b[level], L1 = tr.op_leaf_rows[level];
    int *slab = (level == 0) ? F.fz : F.lab2;  // labels of the scratch rows: tile positions
    int *cand[2] = {wsi, wsi + kOpCandList};
    int *ncand[2] = {wsi + 2 * kOpCandList, wsi + 2 * kOpCandList + kBMaxRows};
    const int K = min(rows, c);
    for (int k0 = 0; k0 < K; k0 += b1) {
      const int c1 = min(b1, K - k0);
      const int r1 = rows - k0;
      const int nl1 = (r1 + L1 - 1) / L1;
      // copies rows slab[0..rr) of tile columns k0..k0+c1 into the scratch tile
      auto gather = [&](int rr, int ldS) {
        for (int e = tid; e < rr * c1; e += kBT) {
          const int q = e / rr, p = e - q * rr;
          scr[p + (size_t)q * ldS] = tile[slab[p] + (size_t)(k0 + q) * ld];
        }
        __syncthreads();
      };
      // ---- tournament: leaves ----
      for (int j = 0; j < nl1; ++j) {
        const int rr = min(L1, r1 - j * L1), ldS = odd_ld(rr);
        for (int p = tid; p < rr; p += kBT) slab[p] = k0 + j * L1 + p;
        __syncthreads();
        gather(rr, ldS);
        const int km = node_factor<T, D - 1>(scr, ldS, rr, c1, slab, F, false, kb, tr, level + 1,
                                             scr + (size_t)ldS * c1, wsi + kOpCand);
        for (int p = tid; p < km; p += kBT) cand[0][j * c1 + p] = slab[p];
        if (tid == 0) ncand[0][j] = km;
        __syncthreads();
      }
      // ---- tournament: binary rounds ----
      int cur = nl1, buf = 0;
      while (cur > 1) {
        const int nout = (cur + 1) / 2;
        for (int o = 0; o < nout; ++o) {
          if (2 * o + 1 >= cur) {
            const int cc = ncand[buf][2 * o];
            for (int p = tid; p < cc; p += kBT) cand[buf ^ 1][o * c1 + p] = cand[buf][2 * o * c1 + p];
            if (tid == 0) ncand[buf ^ 1][o] = cc;
            __syncthreads();
            continue;
          }
          const int na = ncand[buf][2 * o], rr = na + ncand[buf][2 * o + 1], ldS = odd_ld(rr);
          for (int p = tid; p < rr; p += kBT)
            slab[p] = p < na ? cand[buf][2 * o * c1 + p] : cand[buf][(2 * o + 1) * c1 + p - na];
          __syncthreads();
          gather(rr, ldS);
          const int km = node_factor<T, D - 1>(scr, ldS, rr, c1, slab, F, false, kb, tr, level + 1,
                                               scr + (size_t)ldS * c1, wsi + kOpCand);
          for (int p = tid; p < km; p += kBT) cand[buf ^ 1][o * c1 + p] = slab[p];
          if (tid == 0) ncand[buf ^ 1][o] = km;
          __syncthreads();
        }
        buf ^= 1;
        cur = nout;
      }
      // ---- LAPACK swap sequence moving the chosen rows to k0.. (tid 0) ----
      if (tid == 0) {
        for (int t = 0; t < c1; ++t) {
          F.sel[t] = cand[buf][t] - k0;
          F.rev_top[t] = t;
          F.top_c[t] = t;
          F.far_c[t] = F.sel[t];
        }
        for (int i = 0; i < c1; ++i) {
          const int lb = F.sel[i];
          int pp, fslot = -1;
          if (lb < c1) {
            const int rv = F.rev_top[lb];
            if (rv >= 0) {
              pp = rv;
            } else {
              fslot = -rv - 1;
              pp = F.sel[fslot];
            }
          } else {
            pp = lb;
            fslot = i;
          }
          F.perm_dst[i] = pp;
          if (pp == i) continue;
          const int ci = F.top_c[i];
          F.top_c[i] = lb;
          if (pp < c1) {
            F.top_c[pp] = ci;
            F.rev_top[ci] = pp;
          } else {
            F.far_c[fslot] = ci;
            F.rev_top[ci] = -(fslot + 1);
          }
          if (lb < c1) F.rev_top[lb] = i;
        }
      }
      __syncthreads();
      // ---- apply the swaps to every column (in order), labels with them ----
      for (int q = tid; q < c; q += kBT) {
        T *col = tile + (size_t)q * ld + k0;
        for (int i = 0; i < c1; ++i) {
          const int pp = F.perm_dst[i];
          if (pp != i) {
            const T t = col[i];
            col[i] = col[pp];
            col[pp] = t;
          }
        }
      }
      if (tid == 0)
        for (int i = 0; i < c1; ++i) {
          const int pp = F.perm_dst[i];
          if (pp != i) {
            const int t = lab[k0 + i];
            lab[k0 + i] = lab[k0 + pp];
            lab[k0 + pp] = t;
          }
        }
      __syncthreads();
      // ---- eliminate the panel's columns without further pivoting ----
      elim_nopiv(tile, ld, rows, c, k0, k0 + c1, F, root, kb);
    }
    return K;
  }
}

// Node factorization with the tree's operator (GEPP, or the 2D operator of
// depth 1 or 2); scr: shared scratch after the node tile, wsi: the slot's
// candidate buffers of the operator.
template <class T>
__device__ int node_op(T *tile, int ld, int rows, int bk, Fixed<T> &F, bool root, int kb, const ca_tree_t &tr,
                       int *wsi) {
  T *scr = tile + (size_t)ld * bk;
  if (tr.op_depth == 1) return node_factor<T, 1>(tile, ld, rows, bk, F.prow, F, root, kb, tr, 0, scr, wsi);
  if (tr.op_depth == 2) return node_factor<T, 2>(tile, ld, rows, bk, F.prow, F, root, kb, tr, 0, scr, wsi);
  return node_gepp(tile, ld, rows, bk, F.prow, F, root, kb);
}

// Loads the node rows F.prow[0..rows) of panel columns 0..bk-1 into the tile;
// merge rows skip (zero) the entries left of F.fz (use_fz).
template <class T>
__device__ void load_rows(const T *P, int lda, int rows, int bk, T *tile, int ld, Fixed<T> &F, bool use_fz) {
  bool bad = false;
  stage<T>(
      rows * bk,
      [&](int e) -> T {
        const int k = e / rows, p = e - k * rows;
        return (!use_fz || k >= F.fz[p]) ? P[F.prow[p] + (size_t)k * lda] : T(0);
      },
      [&](int e, T v) {
        const int k = e / rows, p = e - k * rows;
        bad |= Num<T>::bad(v);
        tile[p + (size_t)k * ld] = v;
      });
  if (bad) atomicOr(&F.status, CA_STATUS_NONFINITE);
  __syncthreads();
}

// ---------------------------------------------------------------------------
// CALU of one matrix
// ---------------------------------------------------------------------------
template <class T>
__device__ void cta_calu(const ca_batch_item_t &it, Fixed<T> &F, T *R, int region_elems, char *slot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *A = (T *)it.A;
  const int lda = it.lda, m = it.m, n = it.n, b = it.b, L = it.tree.leaf_rows;
  const int K = min(m, n);
  const int nlmax = (m + L - 1) / L;
  int *cand[2] = {(int *)slot, (int *)slot + (size_t)nlmax * b};
  int *ncand[2] = {cand[1] + (size_t)nlmax * b, cand[1] + (size_t)nlmax * b + nlmax};
  T *lu11 = (T *)(((uintptr_t)(ncand[1] + nlmax) + 15) & ~(uintptr_t)15);
  int *wsi = (int *)(((uintptr_t)(lu11 + (size_t)b * b) + 15) & ~(uintptr_t)15);  // operator buffers
  for (int kb = 0; kb < K; kb += b) {
    const int bk = min(b, K - kb), mk = m - kb;
    T *P = A + kb + (size_t)kb * lda;
    const int nl = (mk + L - 1) / L;
    if (tid == 0) build_plan(nl, it.tree, F.plan);
    __syncthreads();
    const int nrounds = F.plan.nrounds;
    // ---- tournament: leaves ----
    for (int j = 0; j < nl; ++j) {
      const int r0 = j * L, rows = min(L, mk - r0), ld = odd_ld(rows);
      for (int p = tid; p < rows; p += kBT) F.prow[p] = r0 + p;
      __syncthreads();
      load_rows(P, lda, rows, bk, R, ld, F, false);
      const int km = node_op(R, ld, rows, bk, F, nrounds == 0, kb, it.tree, wsi);
      for (int p = tid; p < km; p += kBT) cand[0][(size_t)j * b + p] = F.prow[p];
      if (tid == 0) ncand[0][j] = km;
      if (nrounds == 0)
        for (int k = warp; k < bk; k += kBW)
          for (int p = lane; p < bk; p += 32) lu11[p + (size_t)k * b] = R[p + (size_t)k * ld];
      __syncthreads();
    }
    // ---- tournament: merge rounds ----
    int buf = 0;
    for (int r = 0; r < nrounds; ++r) {
      const RoundDesc rd = F.plan.r[r];
      const bool last = (r == nrounds - 1);
      const int *cin = cand[buf], *nin = ncand[buf];
      int *cout = cand[buf ^ 1], *nout = ncand[buf ^ 1];
      for (int o = 0; o < rd.n_out; ++o) {
        int start, cnt, midx;
        round_node(rd, o, start, cnt, midx);
        if (cnt == 1) {
          const int c = nin[start];
          for (int p = tid; p < c; p += kBT) cout[(size_t)o * b + p] = cin[(size_t)start * b + p];
          if (tid == 0) nout[o] = c;
          __syncthreads();
          continue;
        }
        int rows = 0;
        for (int ch = 0; ch < cnt; ++ch) rows += nin[start + ch];
        for (int p = tid; p < rows; p += kBT) {
          int off = 0, ch = 0;
          while (p >= off + nin[start + ch]) off += nin[start + ch++];
          F.prow[p] = cin[(size_t)(start + ch) * b + (p - off)];
        }
        __syncthreads();
        const int ld = odd_ld(rows);
        load_rows(P, lda, rows, bk, R, ld, F, false);
        const int km = node_op(R, ld, rows, bk, F, last, kb, it.tree, wsi);
        for (int p = tid; p < km; p += kBT) cout[(size_t)o * b + p] = F.prow[p];
        if (tid == 0) nout[o] = km;
        if (last)
          for (int k = warp; k < bk; k += kBW)
            for (int p = lane; p < bk; p += 32) lu11[p + (size_t)k * b] = R[p + (size_t)k * ld];
        __syncthreads();
      }
      buf ^= 1;
    }
    // ---- LAPACK swap sequence from the root's selection ----
    // (the root's labels are in F.prow[0..bk) after the last node)
    if (tid == 0) {
      for (int t = 0; t < bk; ++t) {
        F.sel[t] = F.prow[t];
        F.rev_top[t] = t;
        F.top_c[t] = t;
        F.far_c[t] = F.sel[t];
      }
      for (int i = 0; i < bk; ++i) {
        const int lab = F.sel[i];
        int pp, fslot = -1;
        if (lab < bk) {
          const int rr = F.rev_top[lab];
          if (rr >= 0) {
            pp = rr;
          } else {
            fslot = -rr - 1;
            pp = F.sel[fslot];
          }
        } else {
          pp = lab;
          fslot = i;
        }
        it.ipiv[kb + i] = kb + pp + 1;
        if (pp == i) continue;
        const int ci = F.top_c[i];
        F.top_c[i] = lab;
        if (pp < bk) {
          F.top_c[pp] = ci;
          F.rev_top[ci] = pp;
        } else {
          F.far_c[fslot] = ci;
          F.rev_top[ci] = -(fslot + 1);
        }
        if (lab < bk) F.rev_top[lab] = i;
      }
      int np = 0;
      for (int t = 0; t < bk; ++t)
        if (F.top_c[t] != t) {
          F.perm_dst[np] = t;
          F.perm_src[np] = F.top_c[t];
          ++np;
        }
      for (int t = 0; t < bk; ++t)
        if (F.sel[t] >= bk) {
          F.perm_dst[np] = F.sel[t];
          F.perm_src[np] = F.far_c[t];
          ++np;
        }
      F.nperm = np;
    }
    __syncthreads();
    // ---- swap rows at left and right (all n columns) ----
    {
      const int np = F.nperm;
      for (int c = warp; c < n; c += kBW) {
        T *col = A + kb + (size_t)c * lda;
        T v[2 * kBMaxB / 32];
#pragma unroll
        for (int t = 0; t < 2 * kBMaxB / 32; ++t) {
          const int i = lane + 32 * t;
          if (i < np) v[t] = col[F.perm_src[i]];
        }
        __syncwarp();
#pragma unroll
        for (int t = 0; t < 2 * kBMaxB / 32; ++t) {
          const int i = lane + 32 * t;
          if (i < np) col[F.perm_dst[i]] = v[t];
        }
      }
    }
    __syncthreads();
    // ---- L11 \ U11 in place; L21 = A21 U11^-1 ----
    {
      T *U = R;                        // bk x bk, ld bk
      T *rdg = U + (size_t)bk * bk;    // reciprocals of U's diagonal
      T *Tt = rdg + bk;                // rt x bk, ld rt|1
      int rt = (region_elems - bk * bk - bk) / bk - 1;  // the tile's ld is rt + 1
      rt = min(rt, kBT) & ~31;
      const int ldt = rt | 1;
      for (int k = warp; k < bk; k += kBW)
        for (int p = lane; p < bk; p += 32) {
          const T v = lu11[p + (size_t)k * b];
          P[p + (size_t)k * lda] = v;
          U[p + (size_t)k * bk] = v;
        }
      __syncthreads();
      for (int p = tid; p < bk; p += kBT) rdg[p] = T(1) / U[p + (size_t)p * bk];
      __syncthreads();
      for (int r0 = bk; r0 < mk; r0 += rt) {
        const int rows = min(rt, mk - r0);
        stage<T>(
            rows * bk,
            [&](int e) -> T {
              const int k = e / rows, p = e - k * rows;
              return P[r0 + p + (size_t)k * lda];
            },
            [&](int e, T v) {
              const int k = e / rows, p = e - k * rows;
              Tt[p + (size_t)k * ldt] = v;
            });
        __syncthreads();
        if (tid < rows) {
          T *x = Tt + tid;
          for (int j = 0; j < bk; ++j) {
            const T xj = x[(size_t)j * ldt] * rdg[j];
            x[(size_t)j * ldt] = xj;
            for (int k = j + 1; k < bk; ++k) x[(size_t)k * ldt] = fma(-xj, U[j + (size_t)k * bk], x[(size_t)k * ldt]);
          }
        }
        __syncthreads();
        for (int k = warp; k < bk; k += kBW)
          for (int p = lane; p < rows; p += 32) P[r0 + p + (size_t)k * lda] = Tt[p + (size_t)k * ldt];
        __syncthreads();
      }
    }
    const int nt = n - kb - bk;
    if (nt <= 0) continue;
    T *A12 = P + (size_t)bk * lda;
    // ---- U12 = L11^-1 A12 (unit lower) ----
    {
      T *Ls = R;                       // bk x bk, ld bk
      T *Ts = Ls + (size_t)bk * bk;    // bk x ct, row stride ct
      int ct = (region_elems - bk * bk) / bk;
      ct = min(ct, kBT) & ~31;
      for (int k = warp; k < bk; k += kBW)
        for (int p = lane; p < bk; p += 32) Ls[p + (size_t)k * bk] = lu11[p + (size_t)k * b];
      __syncthreads();
      for (int c0 = 0; c0 < nt; c0 += ct) {
        const int cols = min(ct, nt - c0);
        stage<T>(
            cols * bk,
            [&](int e) -> T {
              const int c = e / bk, p = e - c * bk;
              return A12[p + (size_t)(c0 + c) * lda];
            },
            [&](int e, T v) {
              const int c = e / bk, p = e - c * bk;
              Ts[(size_t)p * ct + c] = v;
            });
        __syncthreads();
        if (tid < cols) {
          T *x = Ts + tid;
          for (int i = 1; i < bk; ++i) {
            T s = x[(size_t)i * ct];
            for (int j = 0; j < i; ++j) s = fma(-Ls[i + (size_t)j * bk], x[(size_t)j * ct], s);
            x[(size_t)i * ct] = s;
          }
        }
        __syncthreads();
        for (int c = warp; c < cols; c += kBW)
          for (int p = lane; p < bk; p += 32) A12[p + (size_t)(c0 + c) * lda] = Ts[(size_t)p * ct + c];
        __syncthreads();
      }
    }
    // ---- A22 -= L21 U12 (64 x 64 tiles, k in chunks of 32) ----
    {
      const int mr = mk - bk;
      const T *L21 = P + bk;
      T *A22 = A12 + bk;
      T *As = R;                     // kGk x kTl, As[k * kTl + r]
      T *Bs = As + kGk * kTl;        // kGk x kTl, Bs[k * kTl + c]
      const int tx = tid & 15, ty = tid >> 4;
      for (int c0 = 0; c0 < nt; c0 += kTl)
        for (int r0 = 0; r0 < mr; r0 += kTl) {
          T acc[4][4];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
          for (int k0 = 0; k0 < bk; k0 += kGk) {
            const int kc = min(kGk, bk - k0);
            stage<T>(
                2 * kGk * kTl,
                [&](int e) -> T {
                  if (e < kGk * kTl) {
                    const int r = e & (kTl - 1), k = e / kTl;
                    return (k < kc && r0 + r < mr) ? L21[r0 + r + (size_t)(k0 + k) * lda] : T(0);
                  }
                  e -= kGk * kTl;
                  const int k = e % kGk, c = e / kGk;
                  return (k < kc && c0 + c < nt) ? A12[k0 + k + (size_t)(c0 + c) * lda] : T(0);
                },
                [&](int e, T v) {
                  if (e < kGk * kTl) {
                    As[e] = v;
                  } else {
                    e -= kGk * kTl;
                    Bs[(e % kGk) * kTl + e / kGk] = v;
                  }
                });
            __syncthreads();
            for (int k = 0; k < kc; ++k) {
              T a[4], bb[4];
#pragma unroll
              for (int i = 0; i < 4; ++i) a[i] = As[k * kTl + tx + 16 * i];
#pragma unroll
              for (int j = 0; j < 4; ++j) bb[j] = Bs[k * kTl + ty + 16 * j];
#pragma unroll
              for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
            }
            __syncthreads();
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int c = c0 + ty + 16 * j;
            if (c >= nt) continue;
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              const int r = r0 + tx + 16 * i;
              if (r < mr) A22[r + (size_t)c * lda] -= acc[i][j];
            }
          }
        }
      __syncthreads();
    }
  }
}

// ---------------------------------------------------------------------------
// Householder QR of the node tile (rows x bk, ld); merge rows are zero left
// of F.fz (skipped).  tau to F.tau; T (larft, forward columnwise) to Tg
// (b x b, ld b, zero outside the top-left kmax x kmax).  Returns kmax.
// ---------------------------------------------------------------------------
template <class T>
__device__ int node_qr(T *tile, int ld, int rows, int bk, Fixed<T> &F, bool use_fz, T *Tg, int b,
                       int region_elems) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int kmax = min(rows, bk);
  for (int j = 0; j < kmax; ++j) {
    T *cj = tile + (size_t)j * ld;
    T ss = T(0);
    for (int p = j + 1 + tid; p < rows; p += kBT)
      if (!use_fz || F.fz[p] <= j) ss = fma(cj[p], cj[p], ss);
    ss = wsum(ss);
    if (lane == 0) F.red[warp] = ss;
    __syncthreads();
    if (tid == 0) {
      T xn2 = T(0);
      for (int q = 0; q < kBW; ++q) xn2 += F.red[q];
      const T alpha = cj[j];
      if (xn2 == T(0)) {
        F.scal[4] = T(1);
        F.tau[j] = T(0);
      } else {
        const T nrm = Num<T>::root(fma(alpha, alpha, xn2));
        const T beta = (alpha >= T(0)) ? -nrm : nrm;
        F.scal[1] = beta;
        F.tau[j] = (beta - alpha) / beta;
        F.scal[3] = T(1) / (alpha - beta);
        F.scal[4] = T(0);
      }
    }
    __syncthreads();
    if (F.scal[4] != T(0)) continue;
    const T scal = F.scal[3], tj = F.tau[j];
    for (int p = j + 1 + tid; p < rows; p += kBT)
      if (!use_fz || F.fz[p] <= j) cj[p] *= scal;
    __syncthreads();
    if (tid == 0) cj[j] = F.scal[1];
    // w_q = tau v^T A(:, q), then A(:, q) -= v w_q; a group of 8 lanes per
    // column (4 columns per warp), so that the cross-lane sum of each dot
    // product takes 3 steps: floating-point adds across lanes cost the same
    // pipe as the multiply-adds
    const int grp = lane >> 3, gl = lane & 7;
    for (int q0 = j + 1 + 4 * warp; q0 < bk; q0 += 4 * kBW) {
      const int q = q0 + grp;
      const bool act = q < bk;
      T *cq = tile + (size_t)(act ? q : j) * ld;
      T acc = T(0);
      if (act) {
        acc = (gl == 0) ? cq[j] : T(0);
        for (int p = j + 1 + gl; p < rows; p += 8)
          if (!use_fz || F.fz[p] <= j) acc = fma(cj[p], cq[p], acc);
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (act) {
        const T wq = tj * acc;
        if (gl == 0) cq[j] -= wq;
        for (int p = j + 1 + gl; p < rows; p += 8)
          if (!use_fz || F.fz[p] <= j) cq[p] = fma(-cj[p], wq, cq[p]);
      }
    }
    __syncthreads();
  }
  // T (larft, forward columnwise): column jj = -tau_jj T(0:jj, 0:jj) z with
  // z_q = v_q^T v_jj; built in shared memory after the tile when it fits
  // (odd leading dimension), else in place in Tg
  const int kk = kmax;
  const int ldw = kk | 1;
  const bool in_smem = (size_t)ld * bk + (size_t)ldw * kk <= (size_t)region_elems;
  T *Tw = in_smem ? tile + (size_t)ld * bk : Tg;
  const int ldt = in_smem ? ldw : b;
  if (!in_smem) {
    for (int e = tid; e < b * b; e += kBT) Tg[e] = T(0);
    __syncthreads();
  }
  const int grp = lane >> 3, gl = lane & 7;
  for (int jj = 0; jj < kk; ++jj) {
    // z_q = v_q^T v_jj (q < jj): a group of 8 lanes per q
    const T *cjj = tile + (size_t)jj * ld;
    for (int q0 = 4 * warp; q0 < jj; q0 += 4 * kBW) {
      const int q = q0 + grp;
      T acc = T(0);
      if (q < jj) {
        const T *cq = tile + (size_t)q * ld;
        acc = (gl == 0) ? cq[jj] : T(0);
        for (int p = jj + 1 + gl; p < rows; p += 8) acc = fma(cq[p], cjj[p], acc);
      }
#pragma unroll
      for (int off = 4; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (q < jj && gl == 0) F.z[q] = acc;
    }
    __syncthreads();
    // T(i, jj) = -tau_jj sum_{q=i}^{jj-1} T(i, q) z_q: one thread per row
    const T tj = F.tau[jj];
    for (int i = tid; i < jj; i += kBT) {
      T acc = T(0);
      for (int q = i; q < jj; ++q) acc = fma(Tw[i + (size_t)q * ldt], F.z[q], acc);
      Tw[i + (size_t)jj * ldt] = -tj * acc;
    }
    if (tid == 0) Tw[jj + (size_t)jj * ldt] = tj;
    __syncthreads();
  }
  if (in_smem) {
    for (int e = tid; e < b * b; e += kBT) {
      const int i = e % b, k = e / b;
      Tg[e] = (k < kk && i <= k) ? Tw[i + (size_t)k * ldw] : T(0);
    }
    __syncthreads();
  }
  return kmax;
}

// Node rows of merge `o` (children start..start+cnt-1 with R rows at
// top[], counts c[]): F.prow, F.fz; returns the row count, sets F.iscal[8] to
// the first child's count.
template <class T>
__device__ int merge_rows(const int *top, const int *c, int start, int cnt, Fixed<T> &F) {
  const int tid = threadIdx.x;
  int rows = 0;
  for (int ch = 0; ch < cnt; ++ch) rows += c[start + ch];
  for (int p = tid; p < rows; p += kBT) {
    int off = 0, ch = 0;
    while (p >= off + c[start + ch]) off += c[start + ch++];
    F.prow[p] = top[start + ch] + (p - off);
    F.fz[p] = p - off;
  }
  if (tid == 0) F.iscal[8] = c[start];
  __syncthreads();
  return rows;
}

// C <- Q_node^T C for the node rows F.prow[0..rows) (leaf: Y unit lower
// trapezoid stored in those rows; merge: identity on the first child's rows,
// stored upper trapezoids on the others), nref <= TK reflectors, T block Tg.
// Tile: TK reflectors x TC columns of C; thread (tx, ty) holds W(k, c) for
// k = tx + TX i, c = ty + TY j (i, j < 4).  W = Y^T C over row chunks of kRw,
// W' = T^T W, C -= Y W' over row chunks of TK.
constexpr int kRw = 64;

template <class T, int TK>
__device__ void node_apply_t(const T *P, int lda, T *C, int nt, int rows, int nref, bool leaf, const T *Tg, int b,
                             Fixed<T> &F, T *R) {
  constexpr int TX = TK / 4, TY = kBT / TX, TC = 4 * TY;
  constexpr int SK = TK + 1, SC = TC + 1;  // odd strides
  const int tid = threadIdx.x;
  const int tx = tid % TX, ty = tid / TX;
  T *Ys = R;                     // row chunk x TK, Ys[r * SK + k]
  T *CW = Ys + kRw * SK;         // C chunk Cs[r * SC + c], then W'[k * SC + c]
  T *Ts = CW + kRw * SC;         // T transposed: Ts[k * SK + i] = T(i, k)
  const int c0row = F.iscal[8];
  for (int e = tid; e < TK * TK; e += kBT) {
    const int i = e % TK, k = e / TK;
    Ts[k * SK + i] = (i < nref && k < nref) ? Tg[i + (size_t)k * b] : T(0);
  }
  // merges: the first child's block of Y is the identity, so its rows enter
  // W = C_0 + sum_i Y_i^T C_i and C_0 -= W' directly
  const int pstart = leaf ? 0 : c0row;
  // Y(p, k): leaf rows hold the unit lower trapezoid; merge rows past the
  // first child hold stored upper trapezoids (k >= child-local row)
  auto yval = [&](int p, int k) -> T {
    const bool stored = k < nref && (leaf ? p > k : k >= F.fz[p]);
    T v = stored ? P[F.prow[p] + (size_t)k * lda] : T(0);
    if (leaf && p == k) v = T(1);
    return v;
  };
  for (int c0 = 0; c0 < nt; c0 += TC) {
    const int cols = min(TC, nt - c0);
    T acc[4][4];
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int k = tx + TX * i, c = ty + TY * j;
        acc[i][j] = (!leaf && k < c0row && c < cols) ? C[F.prow[k] + (size_t)(c0 + c) * lda] : T(0);
      }
    // W = Y^T C
    for (int p0 = pstart; p0 < rows; p0 += kRw) {
      const int pr = min(kRw, rows - p0);
      __syncthreads();
      stage<T>(
          kRw * (TK + TC),
          [&](int e) -> T {
            const int r = e % kRw, q = e / kRw;
            if (r >= pr) return T(0);
            if (q < TK) return yval(p0 + r, q);
            return q - TK < cols ? C[F.prow[p0 + r] + (size_t)(c0 + q - TK) * lda] : T(0);
          },
          [&](int e, T v) {
            const int r = e % kRw, q = e / kRw;
            if (q < TK)
              Ys[r * SK + q] = v;
            else
              CW[r * SC + q - TK] = v;
          });
      __syncthreads();
      for (int r = 0; r < pr; ++r) {
        T y[4], cc[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = Ys[r * SK + tx + TX * i];
#pragma unroll
        for (int j = 0; j < 4; ++j) cc[j] = CW[r * SC + ty + TY * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) acc[i][j] = fma(y[i], cc[j], acc[i][j]);
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) CW[(tx + TX * i) * SC + ty + TY * j] = acc[i][j];
    __syncthreads();
    // W' = T^T W
#pragma unroll
    for (int i = 0; i < 4; ++i) {
      const int k = tx + TX * i;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        T sum = T(0);
        for (int q = 0; q <= k && q < nref; ++q) sum = fma(Ts[k * SK + q], CW[q * SC + ty + TY * j], sum);
        acc[i][j] = sum;
      }
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) CW[(tx + TX * i) * SC + ty + TY * j] = acc[i][j];
    if (!leaf) {
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = tx + TX * i, c = ty + TY * j;
          if (k < c0row && c < cols) C[F.prow[k] + (size_t)(c0 + c) * lda] -= acc[i][j];
        }
    }
    // C -= Y W' (thread: r = tx + TX i, c = ty + TY j; row chunks of TK)
    for (int p0 = pstart; p0 < rows; p0 += TK) {
      const int pr = min(TK, rows - p0);
      __syncthreads();
      stage<T>(
          TK * TK, [&](int e) -> T { return (e % TK) < pr ? yval(p0 + e % TK, e / TK) : T(0); },
          [&](int e, T v) { Ys[(e % TK) * SK + e / TK] = v; });
      __syncthreads();
      T o[4][4];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) o[i][j] = T(0);
      for (int k = 0; k < nref; ++k) {
        T y[4], ww[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) y[i] = Ys[(tx + TX * i) * SK + k];
#pragma unroll
        for (int j = 0; j < 4; ++j) ww[j] = CW[k * SC + ty + TY * j];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int j = 0; j < 4; ++j) o[i][j] = fma(y[i], ww[j], o[i][j]);
      }
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const int r = tx + TX * i;
        if (r >= pr) continue;
        T *crow = C + F.prow[p0 + r];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int c = ty + TY * j;
          if (c < cols) crow[(size_t)(c0 + c) * lda] -= o[i][j];
        }
      }
    }
    __syncthreads();
  }
}

template <class T>
__device__ void node_apply(const T *P, int lda, T *C, int nt, int rows, int nref, bool leaf, const T *Tg, int b,
                           Fixed<T> &F, T *R) {
  if (nref <= 32)
    node_apply_t<T, 32>(P, lda, C, nt, rows, nref, leaf, Tg, b, F, R);
  else
    node_apply_t<T, 64>(P, lda, C, nt, rows, nref, leaf, Tg, b, F, R);
}

// ---------------------------------------------------------------------------
// CAQR of one matrix
// ---------------------------------------------------------------------------
template <class T>
__device__ void cta_caqr(const ca_batch_item_t &it, Fixed<T> &F, T *R, int region_elems, char *slot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T *A = (T *)it.A;
  T *qtree = (T *)it.qtree;
  const int lda = it.lda, m = it.m, n = it.n, b = it.b, L = it.tree.leaf_rows;
  const int nlmax = (m + L - 1) / L;
  int *top[2] = {(int *)slot, (int *)slot + nlmax};
  int *cc[2] = {(int *)slot + 2 * nlmax, (int *)slot + 3 * nlmax};
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    const int bk = min(b, n - kb), mk = m - kb;
    T *P = A + kb + (size_t)kb * lda;
    T *Tp = qtree + off;
    const int nl = (mk + L - 1) / L;
    if (tid == 0) build_plan(nl, it.tree, F.plan);
    __syncthreads();
    const int nrounds = F.plan.nrounds, nmerges = F.plan.nmerges;
    // ---- TSQR: leaves ----
    for (int j = 0; j < nl; ++j) {
      const int r0 = j * L, rows = min(L, mk - r0), ld = odd_ld(rows);
      for (int p = tid; p < rows; p += kBT) F.prow[p] = r0 + p;
      __syncthreads();
      load_rows(P, lda, rows, bk, R, ld, F, false);
      const int km = node_qr(R, ld, rows, bk, F, false, Tp + (size_t)j * b * b, b, region_elems);
      for (int k = warp; k < bk; k += kBW)
        for (int p = lane; p < rows; p += 32) P[r0 + p + (size_t)k * lda] = R[p + (size_t)k * ld];
      if (tid == 0) {
        top[0][j] = r0;
        cc[0][j] = km;
      }
      __syncthreads();
    }
    // ---- TSQR: merge rounds ----
    int buf = 0;
    for (int r = 0; r < nrounds; ++r) {
      const RoundDesc rd = F.plan.r[r];
      for (int o = 0; o < rd.n_out; ++o) {
        int start, cnt, midx;
        round_node(rd, o, start, cnt, midx);
        if (cnt == 1) {
          if (tid == 0) {
            top[buf ^ 1][o] = top[buf][start];
            cc[buf ^ 1][o] = cc[buf][start];
          }
          __syncthreads();
          continue;
        }
        const int rows = merge_rows(top[buf], cc[buf], start, cnt, F);
        const int ld = odd_ld(rows);
        load_rows(P, lda, rows, bk, R, ld, F, true);
        const int km = node_qr(R, ld, rows, bk, F, true, Tp + (size_t)(nl + midx) * b * b, b, region_elems);
        for (int k = warp; k < bk; k += kBW)
          for (int p = lane; p < rows; p += 32)
            if (k >= F.fz[p]) P[F.prow[p] + (size_t)k * lda] = R[p + (size_t)k * ld];
        if (tid == 0) {
          top[buf ^ 1][o] = top[buf][start];
          cc[buf ^ 1][o] = km;
        }
        __syncthreads();
      }
      buf ^= 1;
    }
    // ---- tree update of the trailing columns ----
    const int nt = n - kb - bk;
    if (nt > 0) {
      T *C = P + (size_t)bk * lda;
      for (int j = 0; j < nl; ++j) {
        const int r0 = j * L, rows = min(L, mk - r0);
        for (int p = tid; p < rows; p += kBT) F.prow[p] = r0 + p;
        __syncthreads();
        node_apply(P, lda, C, nt, rows, min(rows, bk), true, Tp + (size_t)j * b * b, b, F, R);
        if (tid == 0) {
          top[0][j] = r0;
          cc[0][j] = min(rows, bk);
        }
        __syncthreads();
      }
      buf = 0;
      for (int r = 0; r < nrounds; ++r) {
        const RoundDesc rd = F.plan.r[r];
        for (int o = 0; o < rd.n_out; ++o) {
          int start, cnt, midx;
          round_node(rd, o, start, cnt, midx);
          if (cnt == 1) {
            if (tid == 0) {
              top[buf ^ 1][o] = top[buf][start];
              cc[buf ^ 1][o] = cc[buf][start];
            }
            __syncthreads();
            continue;
          }
          const int rows = merge_rows(top[buf], cc[buf], start, cnt, F);
          const int km = min(rows, bk);
          node_apply(P, lda, C, nt, rows, km, false, Tp + (size_t)(nl + midx) * b * b, b, F, R);
          if (tid == 0) {
            top[buf ^ 1][o] = top[buf][start];
            cc[buf ^ 1][o] = km;
          }
          __syncthreads();
        }
        buf ^= 1;
      }
    }
    off += (size_t)(nl + nmerges) * b * b;
  }
}

struct BatchArgs {
  const ca_batch_item_t *items;
  int count;
  int region_elems;
  char *slots;
  size_t slot_bytes;
  int *counter;
};

template <class T>
__global__ void __launch_bounds__(kBT, 1) batched_kernel(BatchArgs a) {
  extern __shared__ __align__(16) char smem_raw[];
  Fixed<T> &F = *reinterpret_cast<Fixed<T> *>(smem_raw);
  T *R = reinterpret_cast<T *>(smem_raw + ((sizeof(Fixed<T>) + 15) & ~size_t(15)));
  char *slot = a.slots + (size_t)blockIdx.x * a.slot_bytes;
  for (;;) {
    if (threadIdx.x == 0) {
      F.item = atomicAdd(a.counter, 1);
      F.info0 = 0;
      F.status = 0;
    }
    __syncthreads();
    const int idx = F.item;
    if (idx >= a.count) return;
    const ca_batch_item_t it = a.items[idx];
    if (it.op == CA_BATCH_CALU)
      cta_calu<T>(it, F, R, a.region_elems, slot);
    else
      cta_caqr<T>(it, F, R, a.region_elems, slot);
    __syncthreads();
    if (threadIdx.x == 0) {
      it.info[0] = F.info0;
      it.info[1] = F.status;
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
int tree_ok(const ca_tree_t &t, int b) {
  if (t.nlevels < 1 || t.nlevels > CA_MAX_LEVELS) return 0;
  if (t.leaf_rows < b || t.leaf_rows < 1) return 0;
  for (int l = 0; l < t.nlevels; ++l) {
    if (t.style[l] != CA_TREE_BINARY && t.style[l] != CA_TREE_FLAT) return 0;
    if (l < t.nlevels - 1 && t.fan_in[l] < 1) return 0;
  }
  return 1;
}

double item_flops(const ca_batch_item_t &it) {
  const double m = it.m, n = it.n;
  const double k = m < n ? m : n;
  if (it.op == CA_BATCH_CALU) {
    // LAPACK getrf count: m n k - (m + n) k^2 / 2 + k^3 / 3 multiply-adds
    // (m n^2 - n^3 / 3 flops for m >= n)
    return 2.0 * (m * n * k - (m + n) * k * k / 2.0 + k * k * k / 3.0);
  }
  return 2.0 * m * n * n - 2.0 * n * n * n / 3.0;
}

// Largest phase-region need (elements) of one item, and its slot bytes;
// returns 0 if the item cannot run here.
int item_needs(const ca_batch_item_t &it, size_t esz, size_t region_cap, size_t *elems, size_t *slot) {
  const int K = it.m < it.n ? it.m : it.n;
  const int b = it.b;
  const int bk = b < K ? b : K;
  const int L = it.tree.leaf_rows;
  const int nlmax = (it.m + L - 1) / L;
  size_t need = 0;
  // node tiles of the first panel (the largest); later panels have fewer rows
  Plan p;
  if (!build_plan(nlmax, it.tree, p)) return 0;
  int rows = L < it.m ? L : it.m;
  for (int r = 0; r < p.nrounds; ++r) rows = std::max(rows, p.r[r].max_cnt * bk);
  if (rows > kBMaxRows) return 0;
  need = std::max(need, (size_t)odd_ld(rows) * bk);
  const bool multi = it.n > bk;  // a trailing update follows the first panel
  if (multi && bk > kBMultiB) return 0;
  if (it.op == CA_BATCH_CALU) {
    // the 2D operator's scratch tiles after the node tile (level d: a leaf of
    // op_leaf_rows[d] rows or a binary merge of two op_b[d]-row sets)
    size_t scr = 0;
    int pr = rows, pw = bk;
    for (int d = 0; d < it.tree.op_depth; ++d) {
      const int w = std::min(it.tree.op_b[d], pw);
      const int r = std::min(std::max(it.tree.op_leaf_rows[d], 2 * w), pr);
      scr += (size_t)odd_ld(r) * w;
      pr = r;
      pw = w;
    }
    need = std::max(need, (size_t)odd_ld(rows) * bk + scr);
    need = std::max(need, (size_t)bk * bk + bk + 33 * (size_t)bk);  // L21 with 32-row tiles at least
    if (multi) {
      need = std::max(need, (size_t)bk * bk + 32 * (size_t)bk);
      need = std::max(need, (size_t)2 * kGk * kTl);
    }
    *slot = align256((size_t)4 * (2 * (size_t)nlmax * b + 2 * nlmax) + 16) + (size_t)b * b * esz + 16 +
            (size_t)4 * kOpCand * it.tree.op_depth;
  } else {
    if (multi) need = std::max(need, (size_t)3 * kTl * kTs);  // node_apply_t<T, 64>: 3 x 64 x 65 (the larger)
    *slot = (size_t)4 * 4 * nlmax;
  }
  if (need * esz > region_cap) return 0;
  *elems = need;
  return 1;
}

// ---------------------------------------------------------------------------
// The 2D multilevel reduction operator in the single-matrix CALU
// (calu_factor with op_depth 1 or 2): one CTA per tournament node of a
// round; the node's rows (a leaf, or the stacked candidate sets of its
// children) are loaded into the CTA's shared memory and factored by node_op
// -- the same code as the batched path -- and the node's first min(rows, bk)
// labels are its candidates.  The root also writes L11 \ U11 of its
// selected rows and the panel's swap sequence, as tslu_node_kernel does for
// GEPP nodes.
// ---------------------------------------------------------------------------
struct OpNodeArgs {
  const double *P;
  int lda, mk, bk, leaf_rows;
  int is_leaf, is_root;
  RoundDesc rd;
  const int *cand_in, *ncand_in;
  int *cand_out, *ncand_out;
  int cand_ld;
  double *lu11;
  int ldl;
  int *perm_src, *perm_dst, *perm_cnt, *ipiv_k;
  int ipiv_base;
  int *dev_info;
  const int *skip;
  ca_tree_t tree;
  int *opws;           // the operator's candidate buffers, opws_stride ints per node
  long long opws_stride;
};

__global__ void __launch_bounds__(kBT, 1) op_node_kernel(OpNodeArgs a) {
  extern __shared__ __align__(16) char smem_op[];
  if (a.skip && *a.skip) return;
  Fixed<double> &F = *reinterpret_cast<Fixed<double> *>(smem_op);
  double *R = reinterpret_cast<double *>(smem_op + fixed_bytes(CA_DTYPE_F64));
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int node = blockIdx.x, bk = a.bk;
  int rows;
  if (a.is_leaf) {
    const int r0 = node * a.leaf_rows;
    rows = min(a.leaf_rows, a.mk - r0);
    for (int p = tid; p < rows; p += kBT) F.prow[p] = r0 + p;
  } else {
    int start, cnt, midx;
    round_node(a.rd, node, start, cnt, midx);
    if (cnt == 1) {  // promotion
      const int c = a.ncand_in[start];
      for (int p = tid; p < c; p += kBT) a.cand_out[(size_t)node * a.cand_ld + p] = a.cand_in[(size_t)start * a.cand_ld + p];
      if (tid == 0) a.ncand_out[node] = c;
      return;
    }
    rows = 0;
    for (int ch = 0; ch < cnt; ++ch) rows += a.ncand_in[start + ch];
    for (int p = tid; p < rows; p += kBT) {
      int off = 0, ch = 0;
      while (p >= off + a.ncand_in[start + ch]) off += a.ncand_in[start + ch++];
      F.prow[p] = a.cand_in[(size_t)(start + ch) * a.cand_ld + (p - off)];
    }
  }
  if (tid == 0) {
    F.info0 = 0;
    F.status = 0;
  }
  __syncthreads();
  const int ld = odd_ld(rows);
  load_rows<double>(a.P, a.lda, rows, bk, R, ld, F, false);
  const int km = node_op<double>(R, ld, rows, bk, F, a.is_root != 0, a.ipiv_base, a.tree,
                                 a.opws + (size_t)node * a.opws_stride);
  int *co = a.cand_out + (size_t)node * a.cand_ld;
  for (int p = tid; p < km; p += kBT) co[p] = F.prow[p];
  if (tid == 0) {
    a.ncand_out[node] = km;
    if (F.status && a.dev_info) atomicOr(a.dev_info + 1, F.status);
  }
  if (!a.is_root) return;
  if (tid == 0 && F.info0 && a.dev_info) atomicCAS(a.dev_info, 0, F.info0);
  for (int k = warp; k < bk; k += kBW)
    for (int p = lane; p < bk; p += 32) a.lu11[p + (size_t)k * a.ldl] = R[p + (size_t)k * ld];
  __syncthreads();
  if (tid != 0) return;
  // LAPACK swap sequence moving the root's rows (in selection order) to the
  // top of the panel, and the panel's net row permutation
  for (int t = 0; t < bk; ++t) {
    F.sel[t] = F.prow[t];
    F.rev_top[t] = t;
    F.top_c[t] = t;
    F.far_c[t] = F.sel[t];
  }
  for (int i = 0; i < bk; ++i) {
    const int L = F.sel[i];
    int pp, fslot = -1;
    if (L < bk) {
      const int rr = F.rev_top[L];
      if (rr >= 0) {
        pp = rr;
      } else {
        fslot = -rr - 1;
        pp = F.sel[fslot];
      }
    } else {
      pp = L;
      fslot = i;
    }
    a.ipiv_k[i] = a.ipiv_base + pp + 1;
    if (pp == i) continue;
    const int ci = F.top_c[i];
    F.top_c[i] = L;
    if (pp < bk) {
      F.top_c[pp] = ci;
      F.rev_top[ci] = pp;
    } else {
      F.far_c[fslot] = ci;
      F.rev_top[ci] = -(fslot + 1);
    }
    if (L < bk) F.rev_top[L] = i;
  }
  int n = 0;
  for (int t = 0; t < bk; ++t)
    if (F.top_c[t] != t) {
      a.perm_dst[n] = t;
      a.perm_src[n] = F.top_c[t];
      ++n;
    }
  for (int t = 0; t < bk; ++t)
    if (F.sel[t] >= bk) {
      a.perm_dst[n] = F.sel[t];
      a.perm_src[n] = F.far_c[t];
      ++n;
    }
  *a.perm_cnt = n;
}

// shared-memory elements of a node tile of `rows` x bk with the operator's
// scratch tiles below it (as item_needs)
size_t op_node_elems(int rows, int bk, const ca_tree_t &t) {
  size_t scr = 0;
  int pr = rows, pw = bk;
  for (int d = 0; d < t.op_depth; ++d) {
    const int w = std::min(t.op_b[d], pw);
    const int r = std::min(std::max(t.op_leaf_rows[d], 2 * w), pr);
    scr += (size_t)odd_ld(r) * w;
    pr = r;
    pw = w;
  }
  return (size_t)odd_ld(rows) * bk + scr;
}

constexpr size_t kOpSmemCap = 227 * 1024 - 1024;

}  // namespace

bool op_params_ok(const ca_tree_t &t) {
  if (t.op_depth < 1 || t.op_depth > 2) return false;
  for (int d = 0; d < t.op_depth; ++d)
    if (t.op_b[d] < 1 || t.op_b[d] > kBMaxB || t.op_leaf_rows[d] < t.op_b[d] || t.op_leaf_rows[d] > kBMaxRows)
      return false;
  return true;
}

bool op_node_feasible(int rows, int bk, const ca_tree_t &t) {
  if (rows > kBMaxRows || bk > kBMaxB || !op_params_ok(t)) return false;
  return fixed_bytes(CA_DTYPE_F64) + op_node_elems(rows, bk, t) * 8 <= kOpSmemCap;
}

size_t op_ws_bytes(int nodes, const ca_tree_t &t) {
  if (t.op_depth < 1) return 0;
  return align256((size_t)nodes * kOpCand * t.op_depth * 4);
}

cudaError_t tslu_panel_op(int mk, int bk, double *P, int lda, const ca_tree_t &tree, const Plan &plan,
                          const LuPanelWs &ws, int *opws, int *ipiv_k, int ipiv_base, int *dev_info,
                          cudaStream_t st, const int *skip) {
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(op_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kOpSmemCap);
  });
  if (e != cudaSuccess) return e;
  OpNodeArgs a = {};
  a.P = P;
  a.lda = lda;
  a.mk = mk;
  a.bk = bk;
  a.leaf_rows = tree.leaf_rows;
  a.cand_ld = bk;
  a.lu11 = ws.lu11;
  a.ldl = bk;
  a.perm_src = ws.perm_src;
  a.perm_dst = ws.perm_dst;
  a.perm_cnt = ws.perm_cnt;
  a.ipiv_k = ipiv_k;
  a.ipiv_base = ipiv_base;
  a.dev_info = dev_info;
  a.skip = skip;
  a.tree = tree;
  a.opws = opws;
  a.opws_stride = (long long)kOpCand * tree.op_depth;
  auto launch = [&](int nodes, int rows) -> cudaError_t {
    const size_t smem = fixed_bytes(CA_DTYPE_F64) + op_node_elems(rows, bk, tree) * 8;
    if (smem > kOpSmemCap) return cudaErrorInvalidValue;
    ProfScope ps(kClsTsluNode, st, 0.0);
    op_node_kernel<<<nodes, kBT, smem, st>>>(a);
    return cudaGetLastError();
  };
  a.is_leaf = 1;
  a.is_root = plan.nrounds == 0;
  a.cand_in = nullptr;
  a.ncand_in = nullptr;
  a.cand_out = ws.cand[0];
  a.ncand_out = ws.ncand[0];
  if ((e = launch(plan.nleaves, std::min(tree.leaf_rows, mk))) != cudaSuccess) return e;
  int buf = 0;
  for (int r = 0; r < plan.nrounds; ++r) {
    a.is_leaf = 0;
    a.is_root = (r == plan.nrounds - 1);
    a.rd = plan.r[r];
    a.cand_in = ws.cand[buf];
    a.ncand_in = ws.ncand[buf];
    a.cand_out = ws.cand[buf ^ 1];
    a.ncand_out = ws.ncand[buf ^ 1];
    if ((e = launch(plan.r[r].n_out, plan.r[r].max_cnt * bk)) != cudaSuccess) return e;
    buf ^= 1;
  }
  return cudaSuccess;
}

}  // namespace cagb

using namespace cagb;

extern "C" {

int ca_batched_plan(int count, const ca_batch_item_t *items, int dtype, void *plan, size_t *plan_bytes,
                    size_t *work_bytes) {
  if (count < 0) return -1;
  if (count > 0 && !items) return -2;
  if (dtype != CA_DTYPE_F64 && dtype != CA_DTYPE_F32) return -3;
  if (!plan_bytes) return -5;
  if (!work_bytes) return -6;
  const size_t esz = dtype == CA_DTYPE_F64 ? 8 : 4;
  const size_t pb = kHeaderBytes + (size_t)count * sizeof(ca_batch_item_t);
  const size_t fixed = fixed_bytes(dtype);
  const size_t cap = 227 * 1024 - fixed - 1024;
  size_t region = 0, slot = 256;
  double flops = 0.0;
  for (int i = 0; i < count; ++i) {
    const ca_batch_item_t &it = items[i];
    if (it.op != CA_BATCH_CALU && it.op != CA_BATCH_CAQR) return CA_ERR_BATCH_ITEM;
    if (it.m < 0 || it.n < 0 || it.lda < (it.m > 1 ? it.m : 1) || it.b < 1 || it.b > kBMaxB)
      return CA_ERR_BATCH_ITEM;
    if (it.op == CA_BATCH_CAQR && it.n > it.m) return CA_ERR_BATCH_ITEM;
    if (!tree_ok(it.tree, it.b < (it.m < it.n ? it.m : it.n) ? it.b : (it.m < it.n ? it.m : it.n)))
      return CA_ERR_BATCH_ITEM;
    if (!it.info) return CA_ERR_BATCH_ITEM;
    const int K = it.m < it.n ? it.m : it.n;
    if (K == 0) continue;
    if (!it.A) return CA_ERR_BATCH_ITEM;
    if (it.op == CA_BATCH_CALU && !it.ipiv) return CA_ERR_BATCH_ITEM;
    if (it.op == CA_BATCH_CAQR && !it.qtree) return CA_ERR_BATCH_ITEM;
    if (it.op == CA_BATCH_CAQR && it.tree.op_depth != 0) return CA_ERR_BATCH_ITEM;  // no pivoting in QR
    if (it.tree.op_depth < 0 || it.tree.op_depth > 2) return CA_ERR_BATCH_ITEM;
    for (int d = 0; d < it.tree.op_depth; ++d)
      if (it.tree.op_b[d] < 1 || it.tree.op_b[d] > kBMaxB || it.tree.op_leaf_rows[d] < it.tree.op_b[d] ||
          it.tree.op_leaf_rows[d] > kBMaxRows)
        return CA_ERR_BATCH_ITEM;
    size_t e = 0, s = 0;
    if (!item_needs(it, esz, cap, &e, &s)) return CA_ERR_UNSUPPORTED;
    region = std::max(region, e * esz);
    slot = std::max(slot, align256(s));
    flops += item_flops(it);
  }
  // room for full 256-row / 256-column solve tiles when it fits
  region = std::max(region, std::min(cap, (size_t)(kBMultiB * kBMultiB + kBMultiB + (kBT + 1) * kBMultiB) * esz));
  region = (region + 15) & ~size_t(15);
  // one CTA per SM of the current device (sized for 152 SMs when no device
  // is visible: the plan is host data and may be made without a GPU)
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
    (void)cudaGetLastError();
    sms = 152;
  }
  const int ctas = count < sms ? (count > 0 ? count : 1) : sms;
  *plan_bytes = pb;
  *work_bytes = 256 + (size_t)ctas * slot;
  if (!plan) return CA_OK;
  BatchHeader h = {};
  h.magic = kPlanMagic;
  h.count = count;
  h.dtype = dtype;
  h.ctas = ctas;
  h.smem_region = (int)region;
  h.slot_bytes = slot;
  h.work_bytes = *work_bytes;
  h.flops = flops;
  std::memset(plan, 0, kHeaderBytes);
  std::memcpy(plan, &h, sizeof(h));
  // LPT order: largest flop count first (ties by input position)
  std::vector<int> order(count);
  for (int i = 0; i < count; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(),
                   [&](int x, int y) { return item_flops(items[x]) > item_flops(items[y]); });
  ca_batch_item_t *dst = (ca_batch_item_t *)((char *)plan + kHeaderBytes);
  for (int i = 0; i < count; ++i) dst[i] = items[order[i]];
  return CA_OK;
}

int ca_batched_factor(const void *plan_host, const void *plan_dev, void *work, size_t lwork, cudaStream_t stream) {
  if (!plan_host) return -1;
  BatchHeader h;
  std::memcpy(&h, plan_host, sizeof(h));
  if (h.magic != kPlanMagic) return -1;
  if (!plan_dev) return -2;
  if (h.count == 0) return CA_OK;
  if (!work || lwork < h.work_bytes) return CA_ERR_WORKSPACE;
  const size_t smem = fixed_bytes(h.dtype) + (size_t)h.smem_region;
  BatchArgs a;
  a.items = (const ca_batch_item_t *)((const char *)plan_dev + kHeaderBytes);
  a.count = h.count;
  a.region_elems = (int)(h.smem_region / (h.dtype == CA_DTYPE_F64 ? 8 : 4));
  a.counter = (int *)work;
  a.slots = (char *)work + 256;
  a.slot_bytes = h.slot_bytes;
  if (cudaMemsetAsync(work, 0, 4, stream) != cudaSuccess) return CA_ERR_LAUNCH;
  cudaError_t e;
  {
    ProfScope ps(kClsBatched, stream, h.flops);
    if (h.dtype == CA_DTYPE_F64) {
      e = cudaFuncSetAttribute(batched_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batched_kernel<double><<<h.ctas, kBT, smem, stream>>>(a);
    } else {
      e = cudaFuncSetAttribute(batched_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e == cudaSuccess) batched_kernel<float><<<h.ctas, kBT, smem, stream>>>(a);
    }
  }
  if (e != cudaSuccess) return CA_ERR_LAUNCH;
  return cudaGetLastError() == cudaSuccess ? CA_OK : CA_ERR_LAUNCH;
}

}  // extern "C"
