/*
 * ca_oracle.c -- plain, slow CPU reference for tree-based LU (CALU, tournament
 * pivoting) and QR (CAQR, TSQR) in IEEE FP64 (the default build) or IEEE
 * FP32 (built with -DORA_REAL=float, for the FP32 form of the batched path,
 * so that pivot decisions are taken in the precision the kernel uses).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness oracle for the GPU
 * library.  Only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark may load it.  It shares no code, header, table or helper with
 * the CUDA path, and it never calls into it.
 *
 * What it computes (Grigori, Jacquelin, Khabou, "Multilevel communication
 * optimal LU and QR factorizations for hierarchical platforms", RR-8270):
 *   - GEPP on a block (the leaf / merge operator of tournament pivoting,
 *     Sec. 3.2 and Algorithm "1D multilevel CALU", with LAPACK getf2 semantics)
 *   - TSLU tournament pivoting over a reduction tree (Sec. 3.2: leaves are
 *     factored by GEPP, candidate sets are stacked two-by-two and GEPP picks
 *     the next set; Algorithm "2D-ML-CALU" reduction steps)
 *   - CALU panel by panel (Algorithm "1D multilevel CALU": permute, block
 *     column of L, block row of U, Schur complement update)
 *   - Householder QR with the compact Y T Y^T representation (Sec. 3.1)
 *   - TSQR over the same reduction tree and CAQR with the leaf update
 *     (UPFACT) and the merge update (UPELIM) of Algorithm ML-CAQR (Sec. 3.1)
 *   - the solves that consume the factors (PA = LU; A = QR, Sec. 3).
 *
 * Everything is plain loops, column-major, no blocking beyond what the
 * algorithms define.  Compile with -O2 -ffp-contract=off so that no fused
 * multiply-add changes the rounding; the result is then deterministic.
 *
 * Conventions (readings of the paper where it is silent; each is listed in
 * the design notes):
 *   - argmax: the first maximum of |a| in the current (swapped) row order;
 *   - a zero pivot column: no swap, no scaling, no update; info records it;
 *   - Householder (LAPACK larfg): for x = [alpha; x2], if ||x2|| = 0 then
 *     tau = 0; else beta = -sign(alpha) ||x||, tau = (beta - alpha) / beta,
 *     v = [1; x2 / (alpha - beta)], with sign(0) = +;
 *   - the tree: fixed leaf_rows with a short last leaf; levels group
 *     consecutive nodes by fan-in, binary style merges pairs repeatedly
 *     (an odd node is promoted unchanged), flat style merges the whole group
 *     at once, and the last level takes all remaining nodes;
 *   - leaf_rows >= panel width (every merge's first child then holds a full
 *     set of b rows, so the merged R fits in its rows).
 *
 * Parity: every exported function is pinned by tests (exact rational GEPP,
 * library QR/LU, closed-form identities); none is "parity unpinned".
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifndef ORA_REAL
#define ORA_REAL double
#endif
typedef ORA_REAL real;

#define ORA_MAXLEV 8
#define ORA_BINARY 0
#define ORA_FLAT 1

typedef struct {
  int leaf_rows;
  int nlevels;
  int fan_in[ORA_MAXLEV];
  int style[ORA_MAXLEV];
  /* reduction operator of the tournament's nodes (CALU only): 0 = GEPP;
   * d = 1, 2: CALU of the node's rows with panel width op_b[0] over leaves
   * of op_leaf_rows[0] rows and a binary tree, whose own nodes use the
   * operator of depth d - 1 with (op_b[1], op_leaf_rows[1]) -- the 2D
   * multilevel CALU reduction (Algorithm 2D-ML-CALU, Sec. 3.2) */
  int op_depth;
  int op_b[2];
  int op_leaf_rows[2];
} ora_tree;

#define AT(M, ld, i, j) (M)[(size_t)(j) * (size_t)(ld) + (size_t)(i)]

/* near-tie threshold: a runner-up within this relative distance of the
 * selected maximum is counted (pivot choice then depends on rounding). */
#define ORA_NEARTIE (sizeof(real) == 4 ? 1e-4 : 1e-10)

/* ------------------------------------------------------------------------ */
/* Reduction tree                                                           */
/* ------------------------------------------------------------------------ */

/* One round of merges: output o merges inputs [start[o], start[o]+cnt[o]). */
typedef struct {
  int nout;
  int *start;
  int *cnt;
} ora_round;

typedef struct {
  int nleaves;
  int nrounds;
  ora_round *r;
} ora_plan;

static void plan_free(ora_plan *p) {
  for (int i = 0; i < p->nrounds; ++i) {
    free(p->r[i].start);
    free(p->r[i].cnt);
  }
  free(p->r);
  p->r = NULL;
  p->nrounds = 0;
}

static int plan_push(ora_plan *p, int nout, const int *start, const int *cnt) {
  int has_merge = 0;
  for (int o = 0; o < nout; ++o)
    if (cnt[o] > 1) has_merge = 1;
  if (!has_merge) return 0; /* a round of pure promotions does nothing */
  ora_round *nr = (ora_round *)realloc(p->r, sizeof(ora_round) * (size_t)(p->nrounds + 1));
  if (!nr) return -1;
  p->r = nr;
  ora_round *rd = &p->r[p->nrounds];
  rd->nout = nout;
  rd->start = (int *)malloc(sizeof(int) * (size_t)nout);
  rd->cnt = (int *)malloc(sizeof(int) * (size_t)nout);
  if (!rd->start || !rd->cnt) return -1;
  memcpy(rd->start, start, sizeof(int) * (size_t)nout);
  memcpy(rd->cnt, cnt, sizeof(int) * (size_t)nout);
  p->nrounds++;
  return 0;
}

/* Build the merge rounds for `nleaves` leaves.  Level l groups consecutive
 * nodes by fan_in[l] (the last level groups all of them); inside a group,
 * binary style merges neighbours pairwise until one node is left, flat style
 * merges the whole group in one step (Sec. 3.1, 3.2: log(Pr) pairwise
 * eliminations per level). */
static int plan_build(int nleaves, const ora_tree *t, ora_plan *p) {
  p->nleaves = nleaves;
  p->nrounds = 0;
  p->r = NULL;
  if (t->nlevels < 1 || t->nlevels > ORA_MAXLEV) return -1;
  int cur = nleaves;
  int *start = (int *)malloc(sizeof(int) * (size_t)(nleaves + 1));
  int *cnt = (int *)malloc(sizeof(int) * (size_t)(nleaves + 1));
  int *gsize = (int *)malloc(sizeof(int) * (size_t)(nleaves + 1));
  if (!start || !cnt || !gsize) return -1;
  for (int l = 0; l < t->nlevels; ++l) {
    int f = (l == t->nlevels - 1) ? cur : t->fan_in[l];
    if (f < 1) f = 1;
    int ngroups = (cur + f - 1) / f;
    if (t->style[l] == ORA_FLAT) {
      for (int g = 0; g < ngroups; ++g) {
        start[g] = g * f;
        cnt[g] = (cur - g * f < f) ? cur - g * f : f;
      }
      if (plan_push(p, ngroups, start, cnt)) return -1;
    } else {
      for (int g = 0; g < ngroups; ++g) gsize[g] = (cur - g * f < f) ? cur - g * f : f;
      for (;;) {
        int any = 0;
        for (int g = 0; g < ngroups; ++g)
          if (gsize[g] > 1) any = 1;
        if (!any) break;
        int nout = 0, off = 0;
        for (int g = 0; g < ngroups; ++g) {
          int s = gsize[g];
          int h = (s + 1) / 2;
          for (int o = 0; o < h; ++o) {
            start[nout] = off + 2 * o;
            cnt[nout] = (s - 2 * o >= 2) ? 2 : 1;
            nout++;
          }
          off += s;
          gsize[g] = h;
        }
        if (plan_push(p, nout, start, cnt)) return -1;
      }
    }
    cur = ngroups;
  }
  free(start);
  free(cnt);
  free(gsize);
  return cur == 1 ? 0 : -1;
}

static int count_merges(const ora_plan *p) {
  int nm = 0;
  for (int r = 0; r < p->nrounds; ++r)
    for (int o = 0; o < p->r[r].nout; ++o)
      if (p->r[r].cnt[o] > 1) nm++;
  return nm;
}

/* Public: number of leaves and merge nodes of the tree over m rows. */
int ora_tree_counts(int m, const ora_tree *t, int *nleaves, int *nmerges) {
  if (m < 1 || t->leaf_rows < 1) return -1;
  int nl = (m + t->leaf_rows - 1) / t->leaf_rows;
  ora_plan p;
  if (plan_build(nl, t, &p)) {
    plan_free(&p);
    return -1;
  }
  *nleaves = nl;
  *nmerges = count_merges(&p);
  plan_free(&p);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* GEPP on an r x c block (LAPACK getf2 semantics)                          */
/* ------------------------------------------------------------------------ */

/* In place on W (ld ldw).  perm[i] is the caller's label of the row now at
 * position i; rows are physically swapped, so after the call perm[0..k) are
 * the labels of the selected pivot rows in selection order, k = min(r, c).
 * Returns the 1-based first step with an exactly zero pivot column, else 0. */
static int gepp_block(int r, int c, real *W, int ldw, int *perm, long *nearties) {
  int info = 0;
  int k = r < c ? r : c;
  for (int j = 0; j < k; ++j) {
    int p = j;
    real amax = fabs(AT(W, ldw, j, j));
    for (int i = j + 1; i < r; ++i) {
      real a = fabs(AT(W, ldw, i, j));
      if (a > amax) {
        amax = a;
        p = i;
      }
    }
    if (nearties && amax > 0.0) {
      real second = -1.0;
      for (int i = j; i < r; ++i) {
        if (i == p) continue;
        real a = fabs(AT(W, ldw, i, j));
        if (a > second) second = a;
      }
      if (second >= amax * (1.0 - ORA_NEARTIE)) (*nearties)++;
    }
    if (AT(W, ldw, p, j) != 0.0) {
      if (p != j) {
        for (int q = 0; q < c; ++q) {
          real tmp = AT(W, ldw, j, q);
          AT(W, ldw, j, q) = AT(W, ldw, p, q);
          AT(W, ldw, p, q) = tmp;
        }
        int ti = perm[j];
        perm[j] = perm[p];
        perm[p] = ti;
      }
      real piv = AT(W, ldw, j, j);
      for (int i = j + 1; i < r; ++i) AT(W, ldw, i, j) = AT(W, ldw, i, j) / piv;
      for (int q = j + 1; q < c; ++q) {
        real u = AT(W, ldw, j, q);
        for (int i = j + 1; i < r; ++i) AT(W, ldw, i, q) = AT(W, ldw, i, q) - AT(W, ldw, i, j) * u;
      }
    } else if (info == 0) {
      info = j + 1;
    }
  }
  return info;
}

/* Public: GEPP of an m x n matrix in place; ipiv is the 1-based LAPACK swap
 * sequence of length min(m, n).  Returns info (0 or first zero pivot). */
int ora_getf2(int m, int n, real *A, int lda, int *ipiv, long *nearties) {
  int k = m < n ? m : n;
  int *perm = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  int *pos = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  if (!perm || !pos) return -1000;
  for (int i = 0; i < m; ++i) perm[i] = i;
  int info = gepp_block(m, n, A, lda, perm, nearties);
  /* the swap sequence that produced perm: replay on identity labels */
  int *cur = (int *)malloc(sizeof(int) * (size_t)(m > 0 ? m : 1));
  for (int i = 0; i < m; ++i) {
    cur[i] = i;
    pos[i] = i;
  }
  for (int i = 0; i < k; ++i) {
    int p = pos[perm[i]];
    ipiv[i] = p + 1;
    int a = cur[i], bb = cur[p];
    cur[i] = bb;
    cur[p] = a;
    pos[bb] = i;
    pos[a] = p;
  }
  free(cur);
  free(perm);
  free(pos);
  return info;
}

/* ------------------------------------------------------------------------ */
/* The reduction operator of a tournament node                              */
/* ------------------------------------------------------------------------ */

int ora_calu(int m, int n, real *A, int lda, int b, const ora_tree *t, int *ipiv, long *nearties);

/* Valid operator spec: depth 0..2, each used level with 1 <= b <= leaf rows. */
static int op_valid(const ora_tree *t) {
  if (t->op_depth < 0 || t->op_depth > 2) return 0;
  for (int d = 0; d < t->op_depth; ++d)
    if (t->op_b[d] < 1 || t->op_leaf_rows[d] < t->op_b[d]) return 0;
  return 1;
}

/* Factors the r x c node block W (ld ldw) in place with the tree's operator
 * and permutes perm with its rows (as gepp_block does): GEPP at depth 0;
 * otherwise CALU of the block (Algorithm 2D-ML-CALU: a node -- a leaf, or
 * the stacked candidate sets of a reduction step -- is factored by the
 * multilevel CALU of the level below, with that level's block size and a
 * binary tree over its row blocks).  The first min(r, c) labels of perm are
 * then the node's pivot rows in pivot order. */
static int node_factor(int r, int c, real *W, int ldw, int *perm, const ora_tree *t, long *nearties) {
  if (t->op_depth <= 0) return gepp_block(r, c, W, ldw, perm, nearties);
  ora_tree in;
  memset(&in, 0, sizeof in);
  in.leaf_rows = t->op_leaf_rows[0];
  in.nlevels = 1;
  in.fan_in[0] = 0;
  in.style[0] = ORA_BINARY;
  in.op_depth = t->op_depth - 1;
  in.op_b[0] = t->op_b[1];
  in.op_leaf_rows[0] = t->op_leaf_rows[1];
  int k = r < c ? r : c;
  int *ipiv = (int *)malloc(sizeof(int) * (size_t)(k > 0 ? k : 1));
  if (!ipiv) return -1000;
  int info = ora_calu(r, c, W, ldw, t->op_b[0], &in, ipiv, nearties);
  for (int i = 0; i < k && info >= 0; ++i) {
    int sw = ipiv[i] - 1; /* the row swapped with row i */
    int ti = perm[i];
    perm[i] = perm[sw];
    perm[sw] = ti;
  }
  free(ipiv);
  return info;
}

/* ------------------------------------------------------------------------ */
/* TSLU: tournament pivoting over the reduction tree                        */
/* ------------------------------------------------------------------------ */

/* Tournament on the m x b panel P (ld ldp, original values are read, never
 * written).  sel[0..k) receives the panel-relative rows chosen by the root,
 * in root selection order, k = min(m, b).  Every leaf is factored by the
 * node operator (GEPP, or the 2D multilevel CALU operator) and yields
 * min(rows, b) candidate rows; every merge stacks its children's candidate
 * rows (original values, child order, each child in its selection order) and
 * the operator picks min(sum, b) of them (Sec. 3.2, reduction steps).
 * Negative returns: -1 bad argument, -2 bad tree, -3 / -1000 out of memory
 * (like the other allocation failures here, nothing is freed on that path). */
int ora_tslu_select(int m, int b, const real *P, int ldp, const ora_tree *t, int *sel,
                    long *nearties) {
  if (m < 1 || b < 1 || t->leaf_rows < b || !op_valid(t)) return -1;
  int L = t->leaf_rows;
  int nl = (m + L - 1) / L;
  ora_plan plan;
  if (plan_build(nl, t, &plan)) {
    plan_free(&plan);
    return -2;
  }
  /* candidate sets of the current round's nodes */
  int **cand = (int **)calloc((size_t)nl, sizeof(int *));
  int *ncand = (int *)calloc((size_t)nl, sizeof(int));
  size_t wmax = (size_t)(L > 2 * b ? L : 2 * b);
  for (int r = 0; r < plan.nrounds; ++r)
    for (int o = 0; o < plan.r[r].nout; ++o)
      if ((size_t)plan.r[r].cnt[o] * b > wmax) wmax = (size_t)plan.r[r].cnt[o] * b;
  real *W = (real *)malloc(sizeof(real) * wmax * (size_t)b);
  int *perm = (int *)malloc(sizeof(int) * wmax);
  if (!cand || !ncand || !W || !perm) return -1000;

  for (int j = 0; j < nl; ++j) {
    int r0 = j * L;
    int rows = (m - r0 < L) ? m - r0 : L;
    for (int q = 0; q < b; ++q)
      for (int i = 0; i < rows; ++i) AT(W, rows, i, q) = AT(P, ldp, r0 + i, q);
    for (int i = 0; i < rows; ++i) perm[i] = r0 + i;
    if (node_factor(rows, b, W, rows, perm, t, nearties) < 0) return -3;
    int c = rows < b ? rows : b;
    cand[j] = (int *)malloc(sizeof(int) * (size_t)c);
    memcpy(cand[j], perm, sizeof(int) * (size_t)c);
    ncand[j] = c;
  }
  int ncur = nl;
  for (int r = 0; r < plan.nrounds; ++r) {
    ora_round *rd = &plan.r[r];
    int **nc = (int **)calloc((size_t)rd->nout, sizeof(int *));
    int *nn = (int *)calloc((size_t)rd->nout, sizeof(int));
    for (int o = 0; o < rd->nout; ++o) {
      int s = rd->start[o], cnt = rd->cnt[o];
      if (cnt == 1) {
        nc[o] = cand[s];
        nn[o] = ncand[s];
        cand[s] = NULL;
        continue;
      }
      int rows = 0;
      for (int ch = s; ch < s + cnt; ++ch) rows += ncand[ch];
      int at = 0;
      for (int ch = s; ch < s + cnt; ++ch)
        for (int i = 0; i < ncand[ch]; ++i) {
          for (int q = 0; q < b; ++q) AT(W, rows, at, q) = AT(P, ldp, cand[ch][i], q);
          perm[at] = cand[ch][i];
          at++;
        }
      if (node_factor(rows, b, W, rows, perm, t, nearties) < 0) return -3;
      int c = rows < b ? rows : b;
      nc[o] = (int *)malloc(sizeof(int) * (size_t)c);
      memcpy(nc[o], perm, sizeof(int) * (size_t)c);
      nn[o] = c;
      for (int ch = s; ch < s + cnt; ++ch) {
        free(cand[ch]);
        cand[ch] = NULL;
      }
    }
    for (int i = 0; i < ncur; ++i) free(cand[i]);
    for (int o = 0; o < rd->nout; ++o) {
      cand[o] = nc[o];
      ncand[o] = nn[o];
    }
    ncur = rd->nout;
    free(nc);
    free(nn);
  }
  int k = ncand[0];
  memcpy(sel, cand[0], sizeof(int) * (size_t)k);
  free(cand[0]);
  free(cand);
  free(ncand);
  free(W);
  free(perm);
  plan_free(&plan);
  return k;
}

/* ------------------------------------------------------------------------ */
/* CALU (Algorithm "1D multilevel CALU", one GPU = one level)               */
/* ------------------------------------------------------------------------ */

/* In place on A (m x n, ld lda).  Panel k covers columns [kb, kb + bk),
 * bk = min(b, min(m, n) - kb).  ipiv gets min(m, n) 1-based row swaps.
 * Returns info: 0, or 1 + the first column whose U diagonal is exactly zero;
 * negative on a bad argument. */
int ora_calu(int m, int n, real *A, int lda, int b, const ora_tree *t, int *ipiv,
             long *nearties) {
  if (m < 0 || n < 0 || lda < (m > 1 ? m : 1) || b < 1 || t->leaf_rows < b || !op_valid(t)) return -1;
  int K = m < n ? m : n;
  int info = 0;
  int *sel = (int *)malloc(sizeof(int) * (size_t)(b + 1));
  int *pos = (int *)malloc(sizeof(int) * (size_t)(m + 1));
  int *who = (int *)malloc(sizeof(int) * (size_t)(m + 1));
  if (!sel || !pos || !who) return -1000;
  for (int kb = 0; kb < K; kb += b) {
    int bk = (K - kb < b) ? K - kb : b;
    int mk = m - kb;
    real *P = &AT(A, lda, kb, kb);
    /* 1. tournament pivoting on the panel */
    int k = ora_tslu_select(mk, bk, P, lda, t, sel, nearties);
    if (k != bk) {
      info = -2;
      break;
    }
    /* 2. move the selected rows to the top, full width (swap rows at left
     *    and right), recording the LAPACK swap sequence */
    for (int i = 0; i < mk; ++i) {
      pos[i] = i;
      who[i] = i;
    }
    for (int i = 0; i < bk; ++i) {
      int p = pos[sel[i]];
      ipiv[kb + i] = kb + p + 1;
      if (p != i) {
        for (int q = 0; q < n; ++q) {
          real tmp = AT(A, lda, kb + i, q);
          AT(A, lda, kb + i, q) = AT(A, lda, kb + p, q);
          AT(A, lda, kb + p, q) = tmp;
        }
        int wi = who[i], wp = who[p];
        who[i] = wp;
        who[p] = wi;
        pos[wp] = i;
        pos[wi] = p;
      }
    }
    /* 3. L11 U11: LU without pivoting of the selected rows, in their order
     *    (the root's GEPP factors of the same rows) */
    for (int j = 0; j < bk; ++j) {
      real piv = AT(A, lda, kb + j, kb + j);
      if (piv == 0.0) {
        if (info == 0) info = kb + j + 1;
        continue;
      }
      for (int i = j + 1; i < bk; ++i) AT(A, lda, kb + i, kb + j) = AT(A, lda, kb + i, kb + j) / piv;
      for (int q = j + 1; q < bk; ++q) {
        real u = AT(A, lda, kb + j, kb + q);
        for (int i = j + 1; i < bk; ++i)
          AT(A, lda, kb + i, kb + q) = AT(A, lda, kb + i, kb + q) - AT(A, lda, kb + i, kb + j) * u;
      }
    }
    /* 4. block column of L: L21 = A21 U11^{-1} (row-wise substitution) */
    for (int i = kb + bk; i < m; ++i)
      for (int j = 0; j < bk; ++j) {
        real s = AT(A, lda, i, kb + j);
        for (int l = 0; l < j; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, kb + j);
        AT(A, lda, i, kb + j) = s / AT(A, lda, kb + j, kb + j);
      }
    /* 5. block row of U: U12 = L11^{-1} A12 (unit lower substitution) */
    for (int q = kb + bk; q < n; ++q)
      for (int i = 0; i < bk; ++i) {
        real s = AT(A, lda, kb + i, q);
        for (int l = 0; l < i; ++l) s = s - AT(A, lda, kb + i, kb + l) * AT(A, lda, kb + l, q);
        AT(A, lda, kb + i, q) = s;
      }
    /* 6. Schur complement: A22 -= L21 U12 */
    for (int q = kb + bk; q < n; ++q)
      for (int i = kb + bk; i < m; ++i) {
        real s = AT(A, lda, i, q);
        for (int l = 0; l < bk; ++l) s = s - AT(A, lda, i, kb + l) * AT(A, lda, kb + l, q);
        AT(A, lda, i, q) = s;
      }
  }
  free(sel);
  free(pos);
  free(who);
  return info;
}

/* Solve A x = B from the CALU (or getf2) factors: row swaps, unit-lower
 * forward substitution, upper back substitution.  B is n x nrhs, in place. */
int ora_getrs(int n, int nrhs, const real *LU, int lda, const int *ipiv, real *B, int ldb) {
  for (int c = 0; c < nrhs; ++c) {
    real *x = &AT(B, ldb, 0, c);
    for (int i = 0; i < n; ++i) {
      int p = ipiv[i] - 1;
      if (p != i) {
        real tmp = x[i];
        x[i] = x[p];
        x[p] = tmp;
      }
    }
    for (int i = 0; i < n; ++i) {
      real s = x[i];
      for (int l = 0; l < i; ++l) s = s - AT(LU, lda, i, l) * x[l];
      x[i] = s;
    }
    for (int i = n - 1; i >= 0; --i) {
      real s = x[i];
      for (int l = i + 1; l < n; ++l) s = s - AT(LU, lda, i, l) * x[l];
      x[i] = s / AT(LU, lda, i, i);
    }
  }
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Householder QR with compact WY (Sec. 3.1: Q = I - Y T Y^T)               */
/* ------------------------------------------------------------------------ */

/* Unblocked Householder QR of the r x c block W (ld ldw) in place, LAPACK
 * geqr2 layout: R on and above the diagonal, v below it (unit diagonal
 * implied).  tau[0..min(r,c)). */
static void geqr2(int r, int c, real *W, int ldw, real *tau) {
  int k = r < c ? r : c;
  for (int j = 0; j < k; ++j) {
    real alpha = AT(W, ldw, j, j);
    real xn2 = 0.0;
    for (int i = j + 1; i < r; ++i) xn2 = xn2 + AT(W, ldw, i, j) * AT(W, ldw, i, j);
    if (xn2 == 0.0) {
      tau[j] = 0.0;
      continue;
    }
    real nrm = sqrt(alpha * alpha + xn2);
    real beta = (alpha >= 0.0) ? -nrm : nrm;
    real tj = (beta - alpha) / beta;
    real scal = (real)1 / (alpha - beta);
    for (int i = j + 1; i < r; ++i) AT(W, ldw, i, j) = AT(W, ldw, i, j) * scal;
    AT(W, ldw, j, j) = beta;
    tau[j] = tj;
    /* apply H_j = I - tau v v^T to the columns on the right */
    for (int q = j + 1; q < c; ++q) {
      real w = AT(W, ldw, j, q);
      for (int i = j + 1; i < r; ++i) w = w + AT(W, ldw, i, j) * AT(W, ldw, i, q);
      w = tj * w;
      AT(W, ldw, j, q) = AT(W, ldw, j, q) - w;
      for (int i = j + 1; i < r; ++i) AT(W, ldw, i, q) = AT(W, ldw, i, q) - AT(W, ldw, i, j) * w;
    }
  }
}

/* LAPACK larft (forward, columnwise): T (k x k, ld ldt) upper triangular with
 * H_0 H_1 ... H_{k-1} = I - V T V^T, V the r x k unit lower trapezoid in W. */
static void larft(int r, int k, const real *V, int ldv, const real *tau, real *T, int ldt) {
  for (int j = 0; j < k; ++j) {
    for (int i = 0; i < k; ++i) AT(T, ldt, i, j) = 0.0;
  }
  for (int j = 0; j < k; ++j) {
    AT(T, ldt, j, j) = tau[j];
    if (tau[j] == 0.0) continue; /* H_j = I: column j of T stays zero above */
    /* z = V(:, 0:j)^T v_j */
    for (int i = 0; i < j; ++i) {
      /* v_j has 1 at row j and V(row, j) below; V(:, i) has 1 at row i */
      real s = AT(V, ldv, j, i); /* row j of v_i times the unit of v_j */
      for (int q = j + 1; q < r; ++q) s = s + AT(V, ldv, q, i) * AT(V, ldv, q, j);
      AT(T, ldt, i, j) = -tau[j] * s;
    }
    /* T(0:j, j) = T(0:j, 0:j) * z  (upper triangular times vector) */
    for (int i = 0; i < j; ++i) {
      real s = 0.0;
      for (int q = i; q < j; ++q) s = s + AT(T, ldt, i, q) * AT(T, ldt, q, j);
      AT(T, ldt, i, j) = s;
    }
  }
}

/* Apply Q^T = I - Y T^T Y^T to C (r x nc, ld ldc); Y is r x k dense (the unit
 * diagonal and the zeros are stored explicitly), T is k x k. */
static void apply_qt_dense(int r, int k, const real *Y, int ldy, const real *T, int ldt,
                           real *C, int ldc, int nc, real *Wk /* k x nc */) {
  for (int q = 0; q < nc; ++q)
    for (int j = 0; j < k; ++j) {
      real s = 0.0;
      for (int i = 0; i < r; ++i) s = s + AT(Y, ldy, i, j) * AT(C, ldc, i, q);
      AT(Wk, k, j, q) = s;
    }
  /* W <- T^T W (T upper, so T^T lower): process rows from the bottom */
  for (int q = 0; q < nc; ++q)
    for (int j = k - 1; j >= 0; --j) {
      real s = 0.0;
      for (int l = 0; l <= j; ++l) s = s + AT(T, ldt, l, j) * AT(Wk, k, l, q);
      AT(Wk, k, j, q) = s;
    }
  for (int q = 0; q < nc; ++q)
    for (int i = 0; i < r; ++i) {
      real s = AT(C, ldc, i, q);
      for (int j = 0; j < k; ++j) s = s - AT(Y, ldy, i, j) * AT(Wk, k, j, q);
      AT(C, ldc, i, q) = s;
    }
}

/* Public: Householder QR of an m x n block in place (geqr2) plus its T
 * (larft), k = min(m, n); T is k x k with ld ldt. */
int ora_geqrt(int m, int n, real *A, int lda, real *T, int ldt) {
  int k = m < n ? m : n;
  real *tau = (real *)malloc(sizeof(real) * (size_t)(k > 0 ? k : 1));
  if (!tau) return -1000;
  geqr2(m, n, A, lda, tau);
  larft(m, k, A, lda, tau, T, ldt);
  free(tau);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* TSQR and CAQR over the reduction tree                                    */
/* ------------------------------------------------------------------------ */

/* Storage (shared convention with the library, documented in its header):
 *  - leaf j of a panel: Householder QR in place on its rows; R in the top
 *    c_j = min(rows_j, bk) rows, Y strictly below the leaf-local diagonal.
 *  - merge node: the stacked R's of its children (child order) are QR
 *    factored; the new R overwrites the first child's R rows (on and above
 *    the diagonal), and child i >= 1's block of Y (upper trapezoidal, c_i x
 *    bk) overwrites child i's R rows on and above the diagonal.  The first
 *    child's block of Y is the identity and is not stored.
 *  - T blocks: per panel, nleaves + nmerges blocks of b x b doubles (ld b),
 *    leaves first, then merges in round order; a block holds its c x c T in
 *    the top-left corner and zeros elsewhere.
 */

/* Stack the R rows of the children [s, s+cnt) of one merge: child ch owns
 * panel rows top[ch] .. top[ch] + c[ch] - 1.  Fills S (rows x bk, ld rows)
 * with the upper trapezoids (zeros below each child's diagonal). */
static void stack_r(const real *P, int ldp, int bk, const int *top, const int *c, int s,
                    int cnt, real *S, int rows) {
  int at = 0;
  for (int ch = s; ch < s + cnt; ++ch) {
    for (int i = 0; i < c[ch]; ++i) {
      for (int q = 0; q < bk; ++q) AT(S, rows, at + i, q) = (q >= i) ? AT(P, ldp, top[ch] + i, q) : 0.0;
    }
    at += c[ch];
  }
}

/* Dense stacked Y of one merge from the stored blocks: identity for the
 * first child, the stored upper trapezoid for the others. */
static void stack_y(const real *P, int ldp, int bk, const int *top, const int *c, int s, int cnt,
                    real *Y, int rows) {
  int at = 0;
  for (int ch = s; ch < s + cnt; ++ch) {
    for (int i = 0; i < c[ch]; ++i)
      for (int q = 0; q < bk; ++q) {
        real v;
        if (ch == s)
          v = (q == i) ? 1.0 : 0.0;
        else
          v = (q >= i) ? AT(P, ldp, top[ch] + i, q) : 0.0;
        AT(Y, rows, at + i, q) = v;
      }
    at += c[ch];
  }
}

/* TSQR of one panel (mk x bk at P, ld ldp) with the tree; T blocks of size
 * b x b go to Tp (leaves then merges). */
static int tsqr_panel(int mk, int bk, int b, real *P, int ldp, const ora_tree *t, real *Tp) {
  int L = t->leaf_rows;
  int nl = (mk + L - 1) / L;
  ora_plan plan;
  if (plan_build(nl, t, &plan)) {
    plan_free(&plan);
    return -2;
  }
  int *top = (int *)malloc(sizeof(int) * (size_t)nl);
  int *c = (int *)malloc(sizeof(int) * (size_t)nl);
  int *ntop = (int *)malloc(sizeof(int) * (size_t)nl);
  int *nc = (int *)malloc(sizeof(int) * (size_t)nl);
  int maxcnt = 2;
  for (int r = 0; r < plan.nrounds; ++r)
    for (int o = 0; o < plan.r[r].nout; ++o)
      if (plan.r[r].cnt[o] > maxcnt) maxcnt = plan.r[r].cnt[o];
  real *S = (real *)malloc(sizeof(real) * (size_t)maxcnt * bk * bk);
  real *tau = (real *)malloc(sizeof(real) * (size_t)bk);
  if (!top || !c || !ntop || !nc || !S || !tau) return -1000;
  size_t bb = (size_t)b * b;
  for (int j = 0; j < nl; ++j) {
    int r0 = j * L;
    int rows = (mk - r0 < L) ? mk - r0 : L;
    real *Tj = Tp + (size_t)j * bb;
    memset(Tj, 0, sizeof(real) * bb);
    ora_geqrt(rows, bk, &AT(P, ldp, r0, 0), ldp, Tj, b);
    top[j] = r0;
    c[j] = rows < bk ? rows : bk;
  }
  int node = nl;
  for (int r = 0; r < plan.nrounds; ++r) {
    ora_round *rd = &plan.r[r];
    for (int o = 0; o < rd->nout; ++o) {
      int s = rd->start[o], cnt = rd->cnt[o];
      if (cnt == 1) {
        ntop[o] = top[s];
        nc[o] = c[s];
        continue;
      }
      int rows = 0;
      for (int ch = s; ch < s + cnt; ++ch) rows += c[ch];
      stack_r(P, ldp, bk, top, c, s, cnt, S, rows);
      geqr2(rows, bk, S, rows, tau);
      int kk = rows < bk ? rows : bk;
      real *Tn = Tp + (size_t)node * bb;
      memset(Tn, 0, sizeof(real) * bb);
      larft(rows, kk, S, rows, tau, Tn, b);
      /* new R into the first child's rows; Y blocks into the others */
      int at = 0;
      for (int ch = s; ch < s + cnt; ++ch) {
        for (int i = 0; i < c[ch]; ++i)
          for (int q = i; q < bk; ++q) AT(P, ldp, top[ch] + i, q) = AT(S, rows, at + i, q);
        at += c[ch];
      }
      ntop[o] = top[s];
      nc[o] = kk;
      node++;
    }
    for (int o = 0; o < rd->nout; ++o) {
      top[o] = ntop[o];
      c[o] = nc[o];
    }
  }
  free(top);
  free(c);
  free(ntop);
  free(nc);
  free(S);
  free(tau);
  plan_free(&plan);
  return node; /* number of T blocks used */
}

/* Apply the Q^T of one factored panel (mk rows, width bk, factors at P) to
 * the mk x nc block C: leaves first (UPFACT), then merges bottom-up
 * (UPELIM).  Tp holds the panel's T blocks (b x b each). */
static int apply_panel_qt(int mk, int bk, int b, const real *P, int ldp, const ora_tree *t,
                          const real *Tp, real *C, int ldc, int ncols) {
  if (ncols <= 0) return 0;
  int L = t->leaf_rows;
  int nl = (mk + L - 1) / L;
  ora_plan plan;
  if (plan_build(nl, t, &plan)) {
    plan_free(&plan);
    return -2;
  }
  int maxcnt = 2;
  for (int r = 0; r < plan.nrounds; ++r)
    for (int o = 0; o < plan.r[r].nout; ++o)
      if (plan.r[r].cnt[o] > maxcnt) maxcnt = plan.r[r].cnt[o];
  size_t ymax = (size_t)(L > maxcnt * bk ? L : maxcnt * bk);
  real *Y = (real *)malloc(sizeof(real) * ymax * bk);
  real *Cs = (real *)malloc(sizeof(real) * ymax * (size_t)ncols);
  real *Wk = (real *)malloc(sizeof(real) * (size_t)bk * ncols);
  int *top = (int *)malloc(sizeof(int) * (size_t)nl);
  int *c = (int *)malloc(sizeof(int) * (size_t)nl);
  int *ntop = (int *)malloc(sizeof(int) * (size_t)nl);
  int *nc = (int *)malloc(sizeof(int) * (size_t)nl);
  if (!Y || !Cs || !Wk || !top || !c || !ntop || !nc) return -1000;
  size_t bb = (size_t)b * b;
  /* leaves (UPFACT) */
  for (int j = 0; j < nl; ++j) {
    int r0 = j * L;
    int rows = (mk - r0 < L) ? mk - r0 : L;
    int kk = rows < bk ? rows : bk;
    for (int q = 0; q < kk; ++q)
      for (int i = 0; i < rows; ++i)
        AT(Y, rows, i, q) = (i > q) ? AT(P, ldp, r0 + i, q) : (i == q ? 1.0 : 0.0);
    apply_qt_dense(rows, kk, Y, rows, Tp + (size_t)j * bb, b, &AT(C, ldc, r0, 0), ldc, ncols, Wk);
    top[j] = r0;
    c[j] = kk;
  }
  /* merges (UPELIM), bottom-up */
  int node = nl;
  for (int r = 0; r < plan.nrounds; ++r) {
    ora_round *rd = &plan.r[r];
    for (int o = 0; o < rd->nout; ++o) {
      int s = rd->start[o], cnt = rd->cnt[o];
      if (cnt == 1) {
        ntop[o] = top[s];
        nc[o] = c[s];
        continue;
      }
      int rows = 0;
      for (int ch = s; ch < s + cnt; ++ch) rows += c[ch];
      int kk = rows < bk ? rows : bk;
      stack_y(P, ldp, bk, top, c, s, cnt, Y, rows);
      int at = 0;
      for (int ch = s; ch < s + cnt; ++ch) {
        for (int i = 0; i < c[ch]; ++i)
          for (int q = 0; q < ncols; ++q) AT(Cs, rows, at + i, q) = AT(C, ldc, top[ch] + i, q);
        at += c[ch];
      }
      apply_qt_dense(rows, kk, Y, rows, Tp + (size_t)node * bb, b, Cs, rows, ncols, Wk);
      at = 0;
      for (int ch = s; ch < s + cnt; ++ch) {
        for (int i = 0; i < c[ch]; ++i)
          for (int q = 0; q < ncols; ++q) AT(C, ldc, top[ch] + i, q) = AT(Cs, rows, at + i, q);
        at += c[ch];
      }
      ntop[o] = top[s];
      nc[o] = kk;
      node++;
    }
    for (int o = 0; o < rd->nout; ++o) {
      top[o] = ntop[o];
      c[o] = nc[o];
    }
  }
  free(Y);
  free(Cs);
  free(Wk);
  free(top);
  free(c);
  free(ntop);
  free(nc);
  plan_free(&plan);
  return 0;
}

/* Public: number of doubles of T storage for CAQR of m x n with width b. */
long long ora_caqr_tcount(int m, int n, int b, const ora_tree *t) {
  int K = m < n ? m : n;
  long long tot = 0;
  for (int kb = 0; kb < K; kb += b) {
    int nl, nm;
    if (ora_tree_counts(m - kb, t, &nl, &nm)) return -1;
    tot += (long long)(nl + nm) * b * b;
  }
  return tot;
}

/* Public: CAQR of A (m x n, m >= n) in place with panel width b and the
 * tree; T receives ora_caqr_tcount doubles.  Per panel: TSQR, then the
 * trailing columns are updated by the leaves' and merges' Q^T (Algorithm
 * ML-CAQR with one level: UPFACT then UPELIM). */
int ora_caqr(int m, int n, real *A, int lda, int b, const ora_tree *t, real *T) {
  if (m < n || n < 0 || lda < (m > 1 ? m : 1) || b < 1 || t->leaf_rows < b || t->op_depth != 0) return -1;
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    int bk = (n - kb < b) ? n - kb : b;
    int mk = m - kb;
    real *P = &AT(A, lda, kb, kb);
    int used = tsqr_panel(mk, bk, b, P, lda, t, T + off);
    if (used < 0) return used;
    int rc = apply_panel_qt(mk, bk, b, P, lda, t, T + off, &AT(A, lda, kb, kb + bk), lda, n - kb - bk);
    if (rc) return rc;
    off += (size_t)used * b * b;
  }
  return 0;
}

/* Public: least-squares solve from the CAQR factors: B (m x nrhs) <- Q^T B
 * panel by panel, then x = R^{-1} (Q^T B)[0:n] in B's top n rows. */
int ora_geqrs(int m, int n, int nrhs, const real *QR, int lda, int b, const ora_tree *t,
              const real *T, real *B, int ldb) {
  if (m < n || b < 1 || t->leaf_rows < b || t->op_depth != 0) return -1;
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    int bk = (n - kb < b) ? n - kb : b;
    int mk = m - kb;
    int nl, nm;
    if (ora_tree_counts(mk, t, &nl, &nm)) return -2;
    int rc = apply_panel_qt(mk, bk, b, &AT(QR, lda, kb, kb), lda, t, T + off, &AT(B, ldb, kb, 0),
                            ldb, nrhs);
    if (rc) return rc;
    off += (size_t)(nl + nm) * b * b;
  }
  for (int c = 0; c < nrhs; ++c)
    for (int i = n - 1; i >= 0; --i) {
      real s = AT(B, ldb, i, c);
      for (int l = i + 1; l < n; ++l) s = s - AT(QR, lda, i, l) * AT(B, ldb, l, c);
      AT(B, ldb, i, c) = s / AT(QR, lda, i, i);
    }
  return 0;
}

/* Public: apply Q^T of a CAQR factorization to C (m x nc) without the solve
 * (used by the tests to rebuild Q). */
int ora_caqr_apply_qt(int m, int n, const real *QR, int lda, int b, const ora_tree *t,
                      const real *T, real *C, int ldc, int nc) {
  size_t off = 0;
  for (int kb = 0; kb < n; kb += b) {
    int bk = (n - kb < b) ? n - kb : b;
    int mk = m - kb;
    int nl, nm;
    if (ora_tree_counts(mk, t, &nl, &nm)) return -2;
    int rc = apply_panel_qt(mk, bk, b, &AT(QR, lda, kb, kb), lda, t, T + off, &AT(C, ldc, kb, 0), ldc, nc);
    if (rc) return rc;
    off += (size_t)(nl + nm) * b * b;
  }
  return 0;
}
