// panel_lu.cu -- TSLU tournament pivoting and the LU panel steps of CALU.
//
// Tree node = one thread-block cluster of G CTAs (G = 1, 2, 4, 8).  The node's
// rows (a leaf of the panel, or the stacked candidate rows of its children)
// are split in contiguous chunks over the G CTAs' shared memory; GEPP runs on
// the distributed tile: per column, a warp-shuffle argmax inside each CTA,
// the G partial maxima exchanged through distributed shared memory (DSMEM),
// the pivot row read from its owner through DSMEM, then each CTA updates its
// own rows.  This is the paper's reduction operator executed by a group of
// lower-level units (Sec. 3.2: the reduction steps of tournament pivoting,
// each node factored by GEPP; the CALU base case at the leaves).
#include <climits>

#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {

constexpr int kNodeThreads = 256;
constexpr int kNodeWarps = kNodeThreads / 32;
constexpr size_t kNodeSmemBudget = 220 * 1024;

struct TsluNodeArgs {
  const double *P;  // panel (row 0 = first row of the panel), ld lda
  int lda, mk, bk;
  int leaf_rows;
  int is_leaf;      // nodes of this launch are the leaves
  int is_root;      // the single node of this launch is the root
  RoundDesc rd;     // merge round (when !is_leaf)
  const int *cand_in;
  const int *ncand_in;
  int *cand_out;
  int *ncand_out;
  int cand_ld;      // ints per node in the candidate buffers (= b)
  int rloc;         // tile rows per CTA
  // root outputs
  double *lu11;     // bk x bk, ld cand_ld
  int *perm_src, *perm_dst, *perm_cnt;
  int *ipiv_k;      // ipiv + kb
  int ipiv_base;    // kb
  const int *skip;  // nonzero: a stage enqueued ahead that is not needed, do nothing
  int *dev_info;    // [0] info, [1] status
};

struct TsluSmem {
  // layout inside dynamic shared memory
  double *tile;     // rloc x bk, ld rloc | 1 (odd: row accesses across columns hit distinct banks)
  double *prow;     // bk
  double *trow;     // bk
  int *lab;         // rloc labels (panel rows)
  ArgMax *wbest;    // kNodeWarps
  ArgMax *slot;     // 1 (this CTA's partial argmax, read by peers)
  ArgMax *gslot;    // 8 (the cluster's partial maxima, gathered)
  double *scal;     // [0] = 1 / pivot
  int *iscal;       // [0] pivot pos, [1] pivot label, [2] label at j, [3] zero column
  int *work;        // 4 * bk ints (root permutation bookkeeping)
  // published for the peers of the cluster, double-buffered by step parity:
  ArgMax *pkey;     // [2] this CTA's best position of the next column
  double *prow_pub; // [2][bk] that row (every column, as after the step's update)
  double *jrow_pub; // [2][bk] the row at the next diagonal position (its owner only)
  int *plab;        // [2] label of the published best row; [2 + q] label of the published diagonal row
  double *lv;       // rloc multipliers of the current column (nodes held by one CTA)
};

__host__ __device__ inline size_t tslu_smem_bytes(int rloc, int bk) {
  size_t s = (size_t)(rloc | 1) * bk * 8 + 2 * (size_t)bk * 8;
  s += (size_t)rloc * 4 + 16 * (kNodeWarps + 1) + 16 * 8 + 16 + 16 + 4 * (size_t)bk * 4 + 64;
  s += 2 * 16 + 4 * (size_t)bk * 8 + 16 + 64;  // published keys, rows and labels
  s += (size_t)rloc * 8 + 16;                   // multipliers
  return s;
}

__device__ inline TsluSmem tslu_carve(char *base, int rloc, int bk) {
  TsluSmem s;
  s.tile = (double *)base;
  base += (size_t)(rloc | 1) * bk * 8;
  s.prow = (double *)base;
  base += (size_t)bk * 8;
  s.trow = (double *)base;
  base += (size_t)bk * 8;
  s.wbest = (ArgMax *)base;
  base += 16 * kNodeWarps;
  s.slot = (ArgMax *)base;
  base += 16;
  s.gslot = (ArgMax *)base;
  base += 16 * 8;
  s.scal = (double *)base;
  base += 16;
  s.iscal = (int *)base;
  base += 16;
  s.lab = (int *)base;
  base += (size_t)rloc * 4;
  s.work = (int *)base;
  base += 4 * (size_t)bk * 4;
  base = (char *)(((uintptr_t)base + 15) & ~(uintptr_t)15);
  s.pkey = (ArgMax *)base;
  base += 2 * 16;
  s.prow_pub = (double *)base;
  base += 2 * (size_t)bk * 8;
  s.jrow_pub = (double *)base;
  base += 2 * (size_t)bk * 8;
  s.plab = (int *)base;
  base += 16;
  base = (char *)(((uintptr_t)base + 15) & ~(uintptr_t)15);
  s.lv = (double *)base;
  return s;
}

// Split cluster barrier: arrive (release: this CTA's shared-memory writes
// become visible to the peers' reads after their wait), then wait (acquire).
// Every thread of every CTA of the cluster executes both, in the same order.
__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

// Cluster-wide barrier (a plain CTA barrier when the cluster has one CTA).
__device__ __forceinline__ void node_sync(cg::cluster_group &cl, int G) {
  if (G > 1)
    cl.sync();
  else
    __syncthreads();
}

__global__ void __launch_bounds__(kNodeThreads, 1) tslu_node_kernel(TsluNodeArgs a) {
  if (a.skip && *a.skip) return;  // every CTA of the cluster reads the same word
  cg::cluster_group cl = cg::this_cluster();
  const int G = (int)cl.num_blocks();
  const int rank = (int)cl.block_rank();
  const int node = blockIdx.x / G;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int bk = a.bk, rloc = a.rloc;
  const int ldt = rloc | 1;  // tile leading dimension
  extern __shared__ __align__(16) char smem_raw[];
  TsluSmem s = tslu_carve(smem_raw, rloc, bk);

  // ---- node inputs ------------------------------------------------------
  int R;              // total rows of the node
  int start = 0, cnt = 1, midx = 0;
  if (a.is_leaf) {
    int r0 = node * a.leaf_rows;
    R = min(a.leaf_rows, a.mk - r0);
    const int p0 = rank * rloc;
    for (int i = tid; i < rloc; i += kNodeThreads) s.lab[i] = r0 + p0 + i;
  } else {
    round_node(a.rd, node, start, cnt, midx);
    if (cnt == 1) {  // promotion: the candidate set passes through unchanged
      if (rank == 0) {
        int c = a.ncand_in[start];
        for (int i = tid; i < c; i += kNodeThreads)
          a.cand_out[(size_t)node * a.cand_ld + i] = a.cand_in[(size_t)start * a.cand_ld + i];
        if (tid == 0) a.ncand_out[node] = c;
      }
      return;
    }
    R = 0;
    for (int ch = 0; ch < cnt; ++ch) R += a.ncand_in[start + ch];
    const int p0 = rank * rloc;
    for (int i = tid; i < rloc; i += kNodeThreads) {
      int p = p0 + i;
      int lab = -1;
      if (p < R) {
        int off = 0;
        for (int ch = 0; ch < cnt; ++ch) {
          int c = a.ncand_in[start + ch];
          if (p < off + c) {
            lab = a.cand_in[(size_t)(start + ch) * a.cand_ld + (p - off)];
            break;
          }
          off += c;
        }
      }
      s.lab[i] = lab;
    }
  }
  __syncthreads();
  const int p0 = rank * rloc;
  const int myrows = max(0, min(rloc, R - p0));

  // ---- load the node's rows (original panel values) --------------------
  bool bad = false;
  for (int k = warp; k < bk; k += kNodeWarps) {
    const double *col = a.P + (size_t)k * a.lda;
    for (int i = lane; i < myrows; i += 32) {
      double v = col[s.lab[i]];
      bad |= not_finite(v);
      s.tile[i + (size_t)k * ldt] = v;
    }
  }
  if (bad && a.dev_info) atomicOr(a.dev_info + 1, CA_STATUS_NONFINITE);
  __syncthreads();

  // ---- GEPP on the distributed tile ------------------------------------
  const int kmax = min(R, bk);
  // A node held by one CTA: two barriers per column, every row local.
  // Step j reads the pivot p of column j and 1 / a_pj that the previous
  // step left in pkey[j & 1] / scal[j & 1]; phase 1 keeps the old rows p and
  // j (prow, trow) and the multipliers l_i = a_ij / a_pj at their positions
  // after the interchange (lv); phase 2 writes the interchanged rows, the
  // multipliers and the rank-1 update, each element by one thread from those
  // copies, and the warp that updates column j + 1 also finds that column's
  // pivot and its reciprocal.  The arithmetic per element is that of the
  // cluster loop below: the same reciprocal, the same fused multiply-add.
  if (G == 1) {
    double *lv = s.lv;
    // pivot of column c over positions >= c (by warp 0, from the tile), its
    // reciprocal, published into buffer q
    auto publish_pivot = [&](int c, int q, ArgMax b) {
      b = warp_argmax(b);
      __syncwarp();  // the warp's writes of column c are visible to lane 0
      if (lane == 0) {
        s.pkey[q] = b;
        s.scal[q] = (b.key != 0ull) ? 1.0 / s.tile[(b.pos - p0) + (size_t)c * ldt] : 0.0;
      }
    };
    if (kmax > 0 && warp == 0) {
      ArgMax b{0ull, INT_MAX};
      for (int i = lane; i < myrows; i += 32) b = argmax_better(b, ArgMax{absbits(s.tile[i]), i});
      publish_pivot(0, 0, b);
    }
    for (int j = 0; j < kmax; ++j) {
      const int q = j & 1;
      __syncthreads();  // column j's pivot is published; step j - 1 is complete
      const ArgMax gb = s.pkey[q];
      const bool zero = gb.key == 0ull;
      const int p = gb.pos;  // p0 = 0: positions are local rows
      if (zero) {
        if (a.is_root && tid == 0 && a.dev_info) atomicCAS(a.dev_info, 0, a.ipiv_base + j + 1);
        if (j + 1 < kmax && warp == 0) {  // nothing changes: column j + 1 as it stands
          ArgMax b{0ull, INT_MAX};
          const double *c1 = s.tile + (size_t)(j + 1) * ldt;
          for (int i = j + 1 + lane; i < myrows; i += 32) b = argmax_better(b, ArgMax{absbits(c1[i]), i});
          publish_pivot(j + 1, q ^ 1, b);
        }
        continue;
      }
      const double rinv = s.scal[q];
      // phase 1: the old rows p and j, the multipliers, the labels
      for (int k = tid; k < bk; k += kNodeThreads) {
        s.prow[k] = s.tile[p + (size_t)k * ldt];
        s.trow[k] = s.tile[j + (size_t)k * ldt];
      }
      {
        const double *cj = s.tile + (size_t)j * ldt;
        for (int i = j + 1 + tid; i < myrows; i += kNodeThreads) lv[i] = ((i == p) ? cj[j] : cj[i]) * rinv;
      }
      if (tid == 0 && p != j) {
        const int t = s.lab[j];
        s.lab[j] = s.lab[p];
        s.lab[p] = t;
      }
      __syncthreads();
      // phase 2: rows j and p interchanged, the multipliers into column j,
      // the update of columns j + 1 .. from the copies
      for (int k = tid; k < bk; k += kNodeThreads) {
        s.tile[j + (size_t)k * ldt] = s.prow[k];
        if (p != j && k < j) s.tile[p + (size_t)k * ldt] = s.trow[k];
      }
      for (int i = j + 1 + tid; i < myrows; i += kNodeThreads) s.tile[i + (size_t)j * ldt] = lv[i];
      for (int k = j + 1 + warp; k < bk; k += kNodeWarps) {
        const double u = s.prow[k];
        double *ck = s.tile + (size_t)k * ldt;
        const double tk = s.trow[k];
        ArgMax b{0ull, INT_MAX};
        for (int i = j + 1 + lane; i < myrows; i += 32) {
          const double v = fma(-lv[i], u, (i == p) ? tk : ck[i]);
          ck[i] = v;
          if (k == j + 1) b = argmax_better(b, ArgMax{absbits(v), i});
        }
        if (k == j + 1 && j + 1 < kmax) publish_pivot(j + 1, q ^ 1, b);
      }
    }
    __syncthreads();
  } else {
    // One cluster barrier per column.  At the end of step j-1 every CTA has
    // published its best position of column j with that row's values (its
    // columns beyond j computed on the fly exactly as the step's update
    // computes them), and the owner of position j has published the row there;
    // step j reads the G keys, takes the pivot row (and, at the pivot's owner,
    // the row at j) from the peers' published copies, swaps locally, scales
    // column j, updates column j + 1, finds and publishes column j + 1's best
    // row, arrives at the barrier, and only then updates columns j + 2.. while
    // the peers catch up.  The published copies of step j are overwritten two
    // steps later, after a barrier every reader has passed.
    // local best of column c over positions >= c (valid rows of this CTA);
    // publishes it (and, at the owner, the row at position c) into buffer q
    auto find_and_publish = [&](int c, int q, bool upd, int jprev) {
      ArgMax best{0ull, INT_MAX};
      const int i0 = max(c - p0, 0);
      const double *colc = s.tile + (size_t)c * ldt;
      for (int i = i0 + tid; i < myrows; i += kNodeThreads)
        best = argmax_better(best, ArgMax{absbits(colc[i]), p0 + i});
      best = warp_argmax(best);
      if (lane == 0) s.wbest[warp] = best;
      __syncthreads();
      ArgMax b = s.wbest[0];
      for (int w = 1; w < kNodeWarps; ++w) b = argmax_better(b, s.wbest[w]);
      // row values as after step jprev's update: columns > jprev + 1 on the fly
      const double *cjp = upd ? s.tile + (size_t)jprev * ldt : nullptr;
      auto value = [&](int li, int k) -> double {
        const double v = s.tile[li + (size_t)k * ldt];
        return (upd && k > jprev + 1) ? fma(-cjp[li], s.prow[k], v) : v;
      };
      if (b.pos != INT_MAX) {
        const int li = b.pos - p0;
        for (int k = tid; k < bk; k += kNodeThreads) s.prow_pub[q * bk + k] = value(li, k);
        if (tid == 0) s.plab[q] = s.lab[li];
      }
      if (tid == 0) s.pkey[q] = b;
      if (c / rloc == rank) {
        const int lc = c - p0;
        for (int k = tid; k < bk; k += kNodeThreads) s.jrow_pub[q * bk + k] = value(lc, k);
        if (tid == 0) s.plab[2 + q] = s.lab[lc];
      }
      // every read of the tile above is done before any thread updates it
      // (the arrive that follows does not wait)
      __syncthreads();
    };
    if (kmax > 0) find_and_publish(0, 0, false, 0);
    cluster_arrive();
    cluster_wait();
    for (int j = 0; j < kmax; ++j) {
      const int q = j & 1;
      // (a) the cluster's best position of column j
      if (tid < G) s.gslot[tid] = (tid == rank) ? s.pkey[q] : *cl.map_shared_rank(s.pkey + q, tid);
      __syncthreads();
      ArgMax gb = s.gslot[0];
      for (int r = 1; r < G; ++r) gb = argmax_better(gb, s.gslot[r]);
      const int zero = (gb.key == 0ull);
      const int p = gb.pos;
      const int i1 = max(j + 1 - p0, 0);
      double *cj = s.tile + (size_t)j * ldt;
      if (!zero) {
        // (b) the pivot row, and at the pivot's owner the row at position j
        const int op = p / rloc, lp = p - op * rloc;
        const int oj = j / rloc, lj = j - oj * rloc;
        const double *pr = (op == rank) ? s.prow_pub + q * bk : cl.map_shared_rank(s.prow_pub + q * bk, op);
        for (int k = tid; k < bk; k += kNodeThreads) {
          const double v = pr[k];
          s.prow[k] = v;
          if (k == j) s.scal[0] = 1.0 / v;
        }
        if (tid == 0) s.iscal[1] = (op == rank) ? s.plab[q] : *cl.map_shared_rank(s.plab + q, op);
        if (p != j && op == rank) {
          const double *jr = (oj == rank) ? s.jrow_pub + q * bk : cl.map_shared_rank(s.jrow_pub + q * bk, oj);
          for (int k = tid; k < bk; k += kNodeThreads) s.trow[k] = jr[k];
          if (tid == 0) s.iscal[2] = (oj == rank) ? s.plab[2 + q] : *cl.map_shared_rank(s.plab + 2 + q, oj);
        }
        __syncthreads();
        // (c) swap rows j and p (full width), labels with them
        if (oj == rank) {
          for (int k = tid; k < bk; k += kNodeThreads) s.tile[lj + (size_t)k * ldt] = s.prow[k];
          if (tid == 0) s.lab[lj] = s.iscal[1];
        }
        if (p != j && op == rank) {
          for (int k = tid; k < bk; k += kNodeThreads) s.tile[lp + (size_t)k * ldt] = s.trow[k];
          if (tid == 0) s.lab[lp] = s.iscal[2];
        }
        __syncthreads();
        // (d) multipliers l_i = a_ij / a_jj for positions > j
        const double rinv = s.scal[0];
        for (int i = i1 + tid; i < myrows; i += kNodeThreads) cj[i] *= rinv;
        __syncthreads();
        // (e) column j + 1 first
        if (j + 1 < bk) {
          const double u = s.prow[j + 1];
          double *ck = s.tile + (size_t)(j + 1) * ldt;
          for (int i = i1 + tid; i < myrows; i += kNodeThreads) ck[i] = fma(-cj[i], u, ck[i]);
        }
        __syncthreads();
      } else if (a.is_root && rank == 0 && tid == 0 && a.dev_info) {
        atomicCAS(a.dev_info, 0, a.ipiv_base + j + 1);
      }
      // (f) column j + 1's best row, published for the next step
      if (j + 1 < kmax) find_and_publish(j + 1, q ^ 1, !zero, j);
      cluster_arrive();
      // (g) the rest of the rank-1 update while the peers reach the barrier
      if (!zero) {
        for (int k = j + 2 + warp; k < bk; k += kNodeWarps) {
          const double u = s.prow[k];
          double *ck = s.tile + (size_t)k * ldt;
          for (int i = i1 + lane; i < myrows; i += 32) ck[i] = fma(-cj[i], u, ck[i]);
        }
      }
      cluster_wait();
    }
  }

  // ---- outputs: candidates in selection order --------------------------
  int *co = a.cand_out + (size_t)node * a.cand_ld;
  for (int i = tid; i < myrows; i += kNodeThreads)
    if (p0 + i < kmax) co[p0 + i] = s.lab[i];
  if (rank == 0 && tid == 0) a.ncand_out[node] = kmax;
  if (!a.is_root) return;

  // root: L11 \ U11 of the selected rows, and the row permutation
  for (int k = warp; k < bk; k += kNodeWarps)
    for (int i = lane; i < myrows; i += 32)
      if (p0 + i < bk) a.lu11[(p0 + i) + (size_t)k * a.cand_ld] = s.tile[i + (size_t)k * ldt];
  node_sync(cl, G);  // every CTA's labels are final and visible
  if (rank != 0) {
    node_sync(cl, G);  // keep shared memory alive until rank 0 has read it
    return;
  }
  int *sel = s.work;            // bk selected labels
  int *rev_top = s.work + bk;   // position of top label x (>= 0) or -(slot+1)
  int *top_c = s.work + 2 * bk; // label at top position t
  int *far_c = s.work + 3 * bk; // label at far position sel[s] (sel[s] >= bk)
  for (int t = tid; t < bk; t += kNodeThreads) {
    int q = t / rloc, l = t - q * rloc;
    sel[t] = (q == 0) ? s.lab[l] : *cl.map_shared_rank(s.lab + l, q);
  }
  __syncthreads();
  node_sync(cl, G);
  if (tid == 0) {
    for (int t = 0; t < bk; ++t) {
      rev_top[t] = t;
      top_c[t] = t;
      far_c[t] = sel[t];
    }
    // LAPACK swap sequence: at step i, swap position i with the current
    // position of the i-th selected row.
    for (int i = 0; i < bk; ++i) {
      int L = sel[i], pp, fslot = -1;
      if (L < bk) {
        int r = rev_top[L];
        if (r >= 0) {
          pp = r;
        } else {
          fslot = -r - 1;
          pp = sel[fslot];
        }
      } else {
        pp = L;
        fslot = i;
      }
      a.ipiv_k[i] = a.ipiv_base + pp + 1;
      if (pp == i) continue;
      int Ci = top_c[i];
      top_c[i] = L;
      if (pp < bk) {
        top_c[pp] = Ci;
        rev_top[Ci] = pp;
      } else {
        far_c[fslot] = Ci;
        rev_top[Ci] = -(fslot + 1);
      }
      if (L < bk) rev_top[L] = i;
    }
    int n = 0;
    for (int t = 0; t < bk; ++t)
      if (top_c[t] != t) {
        a.perm_dst[n] = t;
        a.perm_src[n] = top_c[t];
        ++n;
      }
    for (int t = 0; t < bk; ++t)
      if (sel[t] >= bk) {
        a.perm_dst[n] = sel[t];
        a.perm_src[n] = far_c[t];
        ++n;
      }
    *a.perm_cnt = n;
  }
}

// ---------------------------------------------------------------------------
// laswp: rows row0 + perm_src[i] -> row0 + perm_dst[i], every column; one warp
// per column, all sources read before any destination is written.
// ---------------------------------------------------------------------------
constexpr int kSwapMax = 2 * kMaxPanel;

__global__ void __launch_bounds__(256) laswp_kernel(int ncols, double *A, int lda, int row0,
                                                    const int *src, const int *dst,
                                                    const int *cnt, const int *skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int col = blockIdx.x * 8 + (threadIdx.x >> 5);
  if (col >= ncols) return;
  const int n = *cnt;
  double *c = A + (size_t)col * lda + row0;
  constexpr int kPer = kSwapMax / 32;
  double v[kPer];
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    int i = lane + 32 * t;
    if (i < n) v[t] = c[src[i]];
  }
  __syncwarp();
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    int i = lane + 32 * t;
    if (i < n) c[dst[i]] = v[t];
  }
}

// ---------------------------------------------------------------------------
// Panel finish: the top bk x bk block <- L11\U11 of the root; the rows below
// get L21 = A21 U11^-1 (Sec. 3.2, block column of L).  Right-looking
// substitution on a tile of rows in shared memory.
// ---------------------------------------------------------------------------
constexpr int kFinThreads = 256;

__global__ void __launch_bounds__(kFinThreads) lu_finish_kernel(int mk, int bk, double *P, int lda,
                                                                const double *lu11, int ldl,
                                                                int rt, const int *skip) {
  extern __shared__ __align__(16) double fsm[];
  if (skip && *skip) return;
  // U's upper triangle packed by rows: row j (columns j .. bk-1) at uoff(j)
  double *U = fsm;
  double *rd = U + (size_t)bk * (bk + 1) / 2;  // reciprocals of U's diagonal
  double *T = rd + bk;                         // rt x bk tile (ld rt)
  auto uoff = [bk](int j) { return j * bk - j * (j - 1) / 2; };
  const int tid = threadIdx.x;
  if (blockIdx.x == 0) {
    for (int k = 0; k < bk; ++k)
      for (int i = tid; i < bk; i += kFinThreads) P[i + (size_t)k * lda] = lu11[i + (size_t)k * ldl];
    return;
  }
  const int r0 = bk + (blockIdx.x - 1) * rt;
  const int rows = min(rt, mk - r0);
  for (int k = 0; k < bk; ++k)
    for (int i = tid; i <= k; i += kFinThreads) U[uoff(i) + (k - i)] = lu11[i + (size_t)k * ldl];
  for (int i = tid; i < bk; i += kFinThreads) rd[i] = 1.0 / lu11[i + (size_t)i * ldl];
  for (int k = 0; k < bk; ++k)
    for (int i = tid; i < rows; i += kFinThreads) T[i + (size_t)k * rt] = P[r0 + i + (size_t)k * lda];
  __syncthreads();
  // thread (r, g): row r, columns k = j + 1 + g (mod ng); rt <= kFinThreads
  const int ng = kFinThreads / rt;
  const int g = tid / rt, r = tid - g * rt;
  for (int j = 0; j < bk; ++j) {
    for (int i = tid; i < rows; i += kFinThreads) T[i + (size_t)j * rt] *= rd[j];
    __syncthreads();
    if (g < ng && r < rows) {
      const double x = T[r + (size_t)j * rt];
      const double *uj = U + uoff(j) - j;  // uj[k] = U(j, k)
      for (int k = j + 1 + g; k < bk; k += ng) T[r + (size_t)k * rt] = fma(-x, uj[k], T[r + (size_t)k * rt]);
    }
    __syncthreads();
  }
  for (int k = 0; k < bk; ++k)
    for (int i = tid; i < rows; i += kFinThreads) P[r0 + i + (size_t)k * lda] = T[i + (size_t)k * rt];
}

// ---------------------------------------------------------------------------
// U12 = L11^-1 A12 (unit lower), one CTA per tile of ct columns.
// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(256) trsm_u12_kernel(int bk, int nt, const double *L, int ldl,
                                                       double *A, int lda, int ct, const int *skip) {
  extern __shared__ __align__(16) double usm[];
  if (skip && *skip) return;
  double *Ls = usm;                   // bk x bk, ld bk
  double *T = Ls + (size_t)bk * bk;   // bk x ct, ld bk
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * ct;
  const int cols = min(ct, nt - c0);
  for (int k = 0; k < bk; ++k)
    for (int i = tid; i < bk; i += 256) Ls[i + (size_t)k * bk] = (i > k) ? L[i + (size_t)k * ldl] : 0.0;
  for (int c = 0; c < cols; ++c)
    for (int i = tid; i < bk; i += 256) T[i + (size_t)c * bk] = A[i + (size_t)(c0 + c) * lda];
  __syncthreads();
  // thread (row group, column): rows i > j updated after row j is final
  for (int j = 0; j < bk - 1; ++j) {
    const int nr = bk - j - 1;
    for (int idx = tid; idx < nr * cols; idx += 256) {
      int c = idx / nr, i = j + 1 + (idx - (idx / nr) * nr);
      T[i + (size_t)c * bk] = fma(-Ls[i + (size_t)j * bk], T[j + (size_t)c * bk], T[i + (size_t)c * bk]);
    }
    __syncthreads();
  }
  for (int c = 0; c < cols; ++c)
    for (int i = tid; i < bk; i += 256) A[i + (size_t)(c0 + c) * lda] = T[i + (size_t)c * bk];
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
size_t lu_panel_ws_bytes(int nleaves_max, int b) {
  size_t s = 0;
  s += 2 * align256((size_t)nleaves_max * b * 4);
  s += 2 * align256((size_t)nleaves_max * 4);
  s += align256((size_t)b * b * 8);
  s += 2 * align256((size_t)2 * b * 4);
  s += align256(4);
  return s;
}

void lu_panel_ws_carve(void *work, int nleaves_max, int b, LuPanelWs &ws) {
  char *p = (char *)work;
  for (int i = 0; i < 2; ++i) {
    ws.cand[i] = (int *)p;
    p += align256((size_t)nleaves_max * b * 4);
  }
  for (int i = 0; i < 2; ++i) {
    ws.ncand[i] = (int *)p;
    p += align256((size_t)nleaves_max * 4);
  }
  ws.lu11 = (double *)p;
  p += align256((size_t)b * b * 8);
  ws.perm_src = (int *)p;
  p += align256((size_t)2 * b * 4);
  ws.perm_dst = (int *)p;
  p += align256((size_t)2 * b * 4);
  ws.perm_cnt = (int *)p;
}

static int pick_cluster(int R, int bk, int nodes, int *rloc) {
  int G = 1;
  while (G < 8 && tslu_smem_bytes((R + G - 1) / G, bk) > kNodeSmemBudget) G *= 2;
  // spread the few nodes of the upper levels over more SMs
  while (G < 8 && nodes * G * 2 <= 152 && (R + 2 * G - 1) / (2 * G) >= 32) G *= 2;
  *rloc = (R + G - 1) / G;
  return (tslu_smem_bytes(*rloc, bk) > kNodeSmemBudget) ? -1 : G;
}

// executed flops of GEPP on an r x c block
static double gepp_flops(double r, double c) {
  double k = r < c ? r : c, f = 0.0;
  for (int j = 0; j < (int)k; ++j) f += 2.0 * (r - j - 1) * (c - j - 1) + (r - j - 1);
  return f;
}

static cudaError_t launch_tslu_node(const TsluNodeArgs &args, int nodes, int G, cudaStream_t st) {
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(tslu_node_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)kNodeSmemBudget + 4096);
  });
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  const double rows = args.is_leaf ? (args.leaf_rows < args.mk ? args.leaf_rows : args.mk)
                                   : (double)args.rd.max_cnt * args.bk;
  ProfScope ps(kClsTsluNode, st, nodes * gepp_flops(rows, args.bk));
  cfg.gridDim = dim3(nodes * G);
  cfg.blockDim = dim3(kNodeThreads);
  cfg.dynamicSmemBytes = tslu_smem_bytes(args.rloc, args.bk);
  cfg.stream = st;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeClusterDimension;
  at[0].val.clusterDim.x = G;
  at[0].val.clusterDim.y = 1;
  at[0].val.clusterDim.z = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, tslu_node_kernel, args);
}

cudaError_t tslu_panel(int mk, int bk, double *P, int lda, int leaf_rows, const Plan &plan,
                       const LuPanelWs &ws, int *ipiv_k, int ipiv_base, int *dev_info,
                       cudaStream_t st, const int *skip) {
  TsluNodeArgs a = {};
  a.skip = skip;
  a.P = P;
  a.lda = lda;
  a.mk = mk;
  a.bk = bk;
  a.leaf_rows = leaf_rows;
  a.cand_ld = bk;
  a.lu11 = ws.lu11;
  a.perm_src = ws.perm_src;
  a.perm_dst = ws.perm_dst;
  a.perm_cnt = ws.perm_cnt;
  a.ipiv_k = ipiv_k;
  a.ipiv_base = ipiv_base;
  a.dev_info = dev_info;
  // leaves
  int R = leaf_rows < mk ? leaf_rows : mk;
  int rloc;
  int G = pick_cluster(R, bk, plan.nleaves, &rloc);
  if (G < 0) return cudaErrorInvalidValue;
  a.is_leaf = 1;
  a.is_root = (plan.nrounds == 0);
  a.rloc = rloc;
  a.cand_in = nullptr;
  a.ncand_in = nullptr;
  a.cand_out = ws.cand[0];
  a.ncand_out = ws.ncand[0];
  cudaError_t e = launch_tslu_node(a, plan.nleaves, G, st);
  if (e != cudaSuccess) return e;
  int buf = 0;
  for (int r = 0; r < plan.nrounds; ++r) {
    const RoundDesc &rd = plan.r[r];
    int Rm = rd.max_cnt * bk;
    G = pick_cluster(Rm, bk, rd.n_out, &rloc);
    if (G < 0) return cudaErrorInvalidValue;
    a.is_leaf = 0;
    a.is_root = (r == plan.nrounds - 1);
    a.rd = rd;
    a.rloc = rloc;
    a.cand_in = ws.cand[buf];
    a.ncand_in = ws.ncand[buf];
    a.cand_out = ws.cand[buf ^ 1];
    a.ncand_out = ws.ncand[buf ^ 1];
    e = launch_tslu_node(a, rd.n_out, G, st);
    if (e != cudaSuccess) return e;
    buf ^= 1;
  }
  return cudaSuccess;
}

cudaError_t laswp_apply(int ncols, double *A, int lda, int row0, const LuPanelWs &ws, int bk,
                        cudaStream_t st, const int *skip) {
  (void)bk;
  if (ncols <= 0) return cudaSuccess;
  ProfScope ps(kClsLaswp, st, 0.0);
  laswp_kernel<<<(ncols + 7) / 8, 256, 0, st>>>(ncols, A, lda, row0, ws.perm_src, ws.perm_dst,
                                                ws.perm_cnt, skip);
  return cudaGetLastError();
}

cudaError_t lu_panel_finish(int mk, int bk, double *P, int lda, const LuPanelWs &ws,
                            cudaStream_t st, const int *skip) {
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(lu_finish_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  if (e != cudaSuccess) return e;
  // row tiles sized so that the rows below the panel's top fill one wave
  // of one CTA per SM where they can (shared memory: packed U plus the tile)
  int sms = 0;
  if ((e = device_sm_count(&sms)) != cudaSuccess) return e;
  const int below = mk - bk;
  const size_t ubytes = ((size_t)bk * (bk + 1) / 2 + bk) * 8;
  int rtmax = (int)((200 * 1024 - ubytes) / ((size_t)bk * 8));
  if (rtmax > kFinThreads / 2) rtmax = kFinThreads / 2;  // at least two threads per row
  int rt = below > 0 ? (below + sms - 1) / sms : 1;
  rt = (rt + 7) / 8 * 8;
  if (rt < 32) rt = 32;
  if (rt > rtmax) rt = rtmax;
  size_t smem = ubytes + (size_t)rt * bk * 8;
  int nblk = 1 + (below > 0 ? (below + rt - 1) / rt : 0);
  ProfScope ps(kClsLuFinish, st, (double)(below > 0 ? below : 0) * bk * bk);
  lu_finish_kernel<<<nblk, kFinThreads, smem, st>>>(mk, bk, P, lda, ws.lu11, bk, rt, skip);
  return cudaGetLastError();
}

cudaError_t trsm_u12(int bk, int nt, const double *L11, int ldl, double *A12, int lda,
                     cudaStream_t st, const int *skip) {
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(trsm_u12_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 220 * 1024);
  });
  if (e != cudaSuccess) return e;
  if (nt <= 0 || bk <= 1) return cudaSuccess;
  // column tiles: as many CTAs as SMs where the columns allow (the look-ahead
  // solve of the next panel's b columns is on the panel chain), at most
  // 8192 / bk columns each
  int sms = 0;
  if ((e = device_sm_count(&sms)) != cudaSuccess) return e;
  int ct = (nt + sms - 1) / sms;
  const int ctmax = 8192 / bk < 128 ? 8192 / bk : 128;
  if (ct > ctmax) ct = ctmax;
  if (ct < 1) ct = 1;
  size_t smem = ((size_t)bk * bk + (size_t)bk * ct) * 8;
  ProfScope ps(kClsTrsmU12, st, (double)bk * bk * nt);
  trsm_u12_kernel<<<(nt + ct - 1) / ct, 256, smem, st>>>(bk, nt, L11, ldl, A12, lda, ct, skip);
  return cudaGetLastError();
}

}  // namespace cagb

namespace cagb {
bool lu_node_feasible(int rows, int bk) {
  int rloc;
  return pick_cluster(rows, bk, 1 << 20, &rloc) > 0;
}
}  // namespace cagb
