// ir.cu -- FP64 pieces of iterative refinement around the reduced-precision
// factorization: residual R = B - A X, norms, backward error, X += D.
//
// The residual is the one place refinement needs full FP64 (Sec. 5.1 measures
// the normwise backward error ||b - A x|| / (||A|| ||x|| + ||b||), infinity
// norms): one pass over A, FP64 DFMA, column blocks reduced in a fixed order.
// The stop test runs on the device (ir_decide); every kernel of a later step
// reads the stop word first and returns at once when it is set, so a caller
// enqueues the whole loop without waiting for the GPU.
#include "ca_internal.cuh"

namespace cagb {

constexpr int kResRows = 256;    // rows per CTA (one thread per row)
constexpr int kResCols = 1024;   // columns of A per CTA
constexpr int kResMaxRhs = 16;

// partial[cb][j][i] = sum_{c in block cb} A(i, c) X(c, j); NJ right-hand
// sides per pass (1 for a single one, else 4, the last pass padded)
template <int NJ>
__global__ void __launch_bounds__(kResRows) resid_partial_kernel(int n, int ncols, int nrhs, const double *A,
                                                                 int lda, const double *X, int ldx,
                                                                 double *partial, const int *skip) {
  __shared__ double xs[kResCols * NJ];
  if (*skip) return;
  const int i = blockIdx.x * kResRows + threadIdx.x;
  const int c0 = blockIdx.y * kResCols;
  const int nc = min(kResCols, ncols - c0);
  for (int j0 = 0; j0 < nrhs; j0 += NJ) {
    const int nj = min(NJ, nrhs - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nc * NJ; idx += kResRows) {
      int c = idx % nc, j = idx / nc;
      xs[j * kResCols + c] = (j < nj) ? X[(c0 + c) + (size_t)(j0 + j) * ldx] : 0.0;
    }
    __syncthreads();
    double acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = 0.0;
    if (i < n) {
      const double *a = A + i + (size_t)c0 * lda;
#pragma unroll 4
      for (int c = 0; c < nc; ++c) {
        const double v = a[(size_t)c * lda];
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[j] = fma(v, xs[j * kResCols + c], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        if (j < nj) partial[((size_t)blockIdx.y * nrhs + j0 + j) * n + i] = acc[j];
    }
  }
}

// R = B - sum_cb partial[cb]
__global__ void resid_reduce_kernel(int n, int nrhs, int ncb, const double *partial, const double *B, int ldb,
                                    double *R, int ldr, const int *skip) {
  if (*skip) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * nrhs) return;
  const int i = (int)(t % n), j = (int)(t / n);
  double s = 0.0;
  for (int cb = 0; cb < ncb; ++cb) s += partial[((size_t)cb * nrhs + j) * n + i];
  R[i + (size_t)j * ldr] = B[i + (size_t)j * ldb] - s;
}

// rowsum[i] = sum_c |A(i, c)|
__global__ void rowsum_abs_kernel(int n, const double *A, int lda, double *rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < n; ++c) s += fabs(A[i + (size_t)c * lda]);
  rowsum[i] = s;
}

__device__ double block_max(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, off));
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double m = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) m = fmax(m, red[w]);
  return m;
}

// out[0] = ||A||_inf from the row sums (one CTA)
__global__ void max_kernel(int n, const double *v, double *out) {
  double m = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) m = fmax(m, v[i]);
  m = block_max(m);
  if (threadIdx.x == 0) out[0] = m;
}

// berr[j] = ||R_j||_inf / (||A||_inf ||X_j||_inf + ||B_j||_inf), one CTA per column
__global__ void berr_kernel(int n, const double *R, int ldr, const double *X, int ldx, const double *B, int ldb,
                            const double *anorm, double *berr, const int *skip) {
  if (*skip) return;
  const int j = blockIdx.x;
  double r = 0.0, x = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    r = fmax(r, fabs(R[i + (size_t)j * ldr]));
    x = fmax(x, fabs(X[i + (size_t)j * ldx]));
    b = fmax(b, fabs(B[i + (size_t)j * ldb]));
  }
  r = block_max(r);
  x = block_max(x);
  b = block_max(b);
  if (threadIdx.x == 0) {
    const double den = anorm[0] * x + b;
    berr[j] = den > 0.0 ? r / den : 0.0;
  }
}

__global__ void axpy_kernel(int n, int nrhs, const double *D, int ldd, double *X, int ldx, const int *skip) {
  if (*skip) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * nrhs) return;
  const int i = (int)(t % n), j = (int)(t / n);
  X[i + (size_t)j * ldx] += D[i + (size_t)j * ldd];
}

// A refinement phase: a loop of steps (residual, stop test, correction)
// with its own control block.  Phases run one after the other in stream
// order; a phase starts only if the phases before it stopped above tol.

// First phase: control cleared.  slow < 0.5 (AUTO's classic phase): a step
// that reduces the backward error by less than 1/slow ends the phase (the
// next one takes over); otherwise two steps in a row that fail to halve it
// end the loop.
__global__ void begin_kernel(IrCtl *ctl, double slow) {
  ctl->done = 0;
  ctl->ok = 0;
  ctl->ran = 1;
  ctl->stall = 0;
  ctl->iters = 0;
  ctl->iter_base = 0;
  ctl->slow = slow;
  ctl->prev = 0.0;
  ctl->berr = 0.0;
}

// A later phase: runs (ran = 1) only if the previous one ran or was skipped
// without reaching tol; counts corrections on from it.
__global__ void begin_next_kernel(const IrCtl *prev, IrCtl *ctl, double slow) {
  const int skip = prev->ok;
  ctl->done = skip;
  ctl->ok = skip;
  ctl->ran = !skip;
  ctl->stall = 0;
  ctl->iters = 0;
  ctl->iter_base = prev->iter_base + prev->iters;
  ctl->slow = slow;
  ctl->prev = 0.0;
  ctl->berr = prev->berr;
}

__global__ void copy_matrix_kernel(int m, int n, const double *src, int lds, double *dst, int ldd,
                                   const int *skip) {
  if (skip && *skip) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * n) return;
  const int i = (int)(t % m), j = (int)(t / m);
  dst[i + (size_t)j * ldd] = src[i + (size_t)j * lds];
}

// after a refactorization phase that ran: its dev_info replaces the first
// factorization's, with CA_STATUS_REFACTORED
__global__ void merge_info_kernel(const IrCtl *c, const int *info2, int *dev_info) {
  if (!c->ran) return;
  dev_info[0] = info2[0];
  dev_info[1] |= info2[1] | CA_STATUS_REFACTORED;
}

// The stop test of step `it` of a phase (one thread): the largest backward
// error over the right-hand sides; the phase ends at <= tol (ok), at
// it == max_iter, on a slow step (see begin_kernel) or on the second step in
// a row that did not halve the error.
__global__ void decide_kernel(int it, int max_iter, double tol, int nrhs, const double *berr, IrCtl *ctl,
                              double *berr_out, int *iters_out) {
  if (ctl->done) return;
  double be = 0.0;
  for (int j = 0; j < nrhs; ++j) be = berr[j] > be ? berr[j] : be;
  if (be != be) be = berr[0];  // keep a NaN visible
  for (int j = 0; j < nrhs; ++j)
    if (berr[j] != berr[j]) be = berr[j];
  ctl->berr = be;
  ctl->iters = it;
  if (berr_out) *berr_out = be;
  if (iters_out) *iters_out = ctl->iter_base + it;
  bool stop = false;
  if (be <= tol) {
    stop = true;
    ctl->ok = 1;
  } else if (it >= max_iter) {
    stop = true;
  } else if (it > 0 && be > ctl->slow * ctl->prev) {
    stop = true;
  } else if (it > 0 && be > 0.5 * ctl->prev) {
    if (++ctl->stall >= 2) stop = true;
  } else {
    ctl->stall = 0;
  }
  if (!(be == be)) stop = true;  // NaN: nothing more to gain
  ctl->prev = be;
  ctl->done = stop ? 1 : 0;
}

size_t ir_ws_bytes(int n, int nrhs) {
  const int ncb = (n + kResCols - 1) / kResCols;
  return align256((size_t)ncb * nrhs * n * 8) + align256((size_t)n * nrhs * 8) + align256((size_t)n * 8) +
         align256(8) + align256((size_t)nrhs * 8) + kIrPhases * align256(sizeof(IrCtl)) + align256(8) + 256;
}

void ir_ws_carve(void *ws, int n, int nrhs, IrWs &w) {
  const int ncb = (n + kResCols - 1) / kResCols;
  char *p = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  w.partial = (double *)p;
  p += align256((size_t)ncb * nrhs * n * 8);
  w.R = (double *)p;
  p += align256((size_t)n * nrhs * 8);
  w.rowsum = (double *)p;
  p += align256((size_t)n * 8);
  w.anorm = (double *)p;
  p += align256(8);
  w.berr = (double *)p;
  p += align256((size_t)nrhs * 8);
  for (int i = 0; i < kIrPhases; ++i) {
    w.phase[i] = (IrCtl *)p;
    p += align256(sizeof(IrCtl));
  }
  w.ctl = w.phase[0];
  w.info2 = (int *)p;
}

cudaError_t ir_anorm(int n, const double *A, int lda, const IrWs &w, cudaStream_t st) {
  {
    ProfScope ps(kClsRefine, st, (double)n * n);
    rowsum_abs_kernel<<<(n + 255) / 256, 256, 0, st>>>(n, A, lda, w.rowsum);
  }
  ProfScope ps(kClsRefine, st, 0.0);
  max_kernel<<<1, 1024, 0, st>>>(n, w.rowsum, w.anorm);
  return cudaGetLastError();
}

cudaError_t ir_begin(const IrWs &w, double slow, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  begin_kernel<<<1, 1, 0, st>>>(w.ctl, slow);
  return cudaGetLastError();
}

cudaError_t ir_begin_next(const IrCtl *prev, const IrWs &w, double slow, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  begin_next_kernel<<<1, 1, 0, st>>>(prev, w.ctl, slow);
  return cudaGetLastError();
}

cudaError_t copy_matrix(int m, int n, const double *src, int lds, double *dst, int ldd, const int *skip,
                        cudaStream_t st) {
  const long long tot = (long long)m * n;
  if (tot <= 0) return cudaSuccess;
  ProfScope ps(kClsRefine, st, 0.0);
  copy_matrix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, n, src, lds, dst, ldd, skip);
  return cudaGetLastError();
}

cudaError_t ir_merge_info(const IrWs &w, const int *info2, int *dev_info, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  merge_info_kernel<<<1, 1, 0, st>>>(w.ctl, info2, dev_info);  // w.ctl: the refactorization phase
  return cudaGetLastError();
}

cudaError_t ir_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, const IrWs &w, cudaStream_t st) {
  if (nrhs > kResMaxRhs) {
    // wide right-hand sides: R = B, then R -= A X with the FP64 GEMM
    cudaError_t e = cudaMemcpy2DAsync(w.R, (size_t)n * 8, B, (size_t)ldb * 8, (size_t)n * 8, nrhs,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return gemm_minus_f64(n, nrhs, n, A, lda, X, ldx, w.R, n, st, &w.ctl->done);
  }
  const int ncb = (n + kResCols - 1) / kResCols;
  {
    ProfScope ps(kClsRefine, st, 2.0 * n * (double)n * nrhs);
    const dim3 grid((n + kResRows - 1) / kResRows, ncb);
    if (nrhs == 1)
      resid_partial_kernel<1><<<grid, kResRows, 0, st>>>(n, n, nrhs, A, lda, X, ldx, w.partial, &w.ctl->done);
    else
      resid_partial_kernel<4><<<grid, kResRows, 0, st>>>(n, n, nrhs, A, lda, X, ldx, w.partial, &w.ctl->done);
  }
  ProfScope ps(kClsRefine, st, 0.0);
  const long long tot = (long long)n * nrhs;
  resid_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nrhs, ncb, w.partial, B, ldb, w.R, n,
                                                                      &w.ctl->done);
  return cudaGetLastError();
}

cudaError_t ir_berr(int n, int nrhs, const double *X, int ldx, const double *B, int ldb, const IrWs &w,
                    cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  berr_kernel<<<nrhs, 256, 0, st>>>(n, w.R, n, X, ldx, B, ldb, w.anorm, w.berr, &w.ctl->done);
  return cudaGetLastError();
}

cudaError_t ir_decide(int it, int max_iter, double tol, int nrhs, const IrWs &w, double *berr_out,
                      int *iters_out, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  decide_kernel<<<1, 1, 0, st>>>(it, max_iter, tol, nrhs, w.berr, w.ctl, berr_out, iters_out);
  return cudaGetLastError();
}

cudaError_t ir_update(int n, int nrhs, const IrWs &w, double *X, int ldx, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, (double)n * nrhs);
  const long long tot = (long long)n * nrhs;
  axpy_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nrhs, w.R, n, X, ldx, &w.ctl->done);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Least-squares refinement on the corrected semi-normal equations: with R
// the (reduced-precision) triangular factor of A, each step computes
// r = b - A x in double-double (rounded once to FP64), s = A^T r in FP64, and
// corrects x += R^-1 R^-T s.  The contraction per step is about cond(A)
// times the factorization's relative error, as for the LU refinement; the
// fixed point satisfies the least-squares condition A^T (b - A x) = 0 to the
// rounding of s, so its error is of the order of the problem's own
// sensitivity (cond eps + cond^2 eps ||r|| / (||A|| ||x||)), which an FP64
// residual (rounding errors of order eps ||A|| ||x||) would raise to
// cond^2 eps.
// ---------------------------------------------------------------------------
constexpr int kAtrWarps = 8;

// Double-double arithmetic for the least-squares residual (r = b - A x with a
// relative error of order eps^2 (|A||x| + |b|) before its final rounding, so
// that the fixed point of the refinement is governed by the problem's own
// sensitivity and not by the rounding of r).  Knuth's TwoSum and the FMA
// TwoProduct; the _rn intrinsics are never contracted into FMAs.
struct DD {
  double hi, lo;
};
__device__ __forceinline__ DD two_sum(double a, double b) {
  const double s = __dadd_rn(a, b);
  const double bb = __dsub_rn(s, a);
  const double e = __dadd_rn(__dsub_rn(a, __dsub_rn(s, bb)), __dsub_rn(b, bb));
  return DD{s, e};
}
__device__ __forceinline__ DD dd_add_prod(DD acc, double a, double b) {  // acc + a b
  const double p = __dmul_rn(a, b);
  const double pe = fma(a, b, -p);
  const DD s = two_sum(acc.hi, p);
  return DD{s.hi, __dadd_rn(__dadd_rn(acc.lo, pe), s.lo)};
}
__device__ __forceinline__ DD dd_add(DD a, DD b) {
  const DD s = two_sum(a.hi, b.hi);
  return DD{s.hi, __dadd_rn(__dadd_rn(a.lo, b.lo), s.lo)};
}

// partial[(cb * nrhs + j) * m + i] = (hi, lo) of sum_{c in block cb} A(i, c) X(c, j);
// NJ right-hand sides per pass (1 for a single one, else 4)
template <int NJ>
__global__ void __launch_bounds__(kResRows) resid_partial_dd_kernel(int m, int ncols, int nrhs, const double *A,
                                                                    int lda, const double *X, int ldx, DD *partial,
                                                                    const int *skip) {
  __shared__ double xs[kResCols * NJ];
  if (*skip) return;
  const int i = blockIdx.x * kResRows + threadIdx.x;
  const int c0 = blockIdx.y * kResCols;
  const int nc = min(kResCols, ncols - c0);
  for (int j0 = 0; j0 < nrhs; j0 += NJ) {
    const int nj = min(NJ, nrhs - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nc * NJ; idx += kResRows) {
      int c = idx % nc, j = idx / nc;
      xs[j * kResCols + c] = (j < nj) ? X[(c0 + c) + (size_t)(j0 + j) * ldx] : 0.0;
    }
    __syncthreads();
    DD acc[NJ];
#pragma unroll
    for (int j = 0; j < NJ; ++j) acc[j] = DD{0.0, 0.0};
    if (i < m) {
      const double *a = A + i + (size_t)c0 * lda;
      for (int c = 0; c < nc; ++c) {
        const double v = a[(size_t)c * lda];
#pragma unroll
        for (int j = 0; j < NJ; ++j) acc[j] = dd_add_prod(acc[j], v, xs[j * kResCols + c]);
      }
#pragma unroll
      for (int j = 0; j < NJ; ++j)
        if (j < nj) partial[((size_t)blockIdx.y * nrhs + j0 + j) * m + i] = acc[j];
    }
  }
}

// R = B - sum_cb partial[cb], summed and subtracted in double-double, rounded once
__global__ void resid_reduce_dd_kernel(int m, int nrhs, int ncb, const DD *partial, const double *B, int ldb,
                                       double *R, int ldr, const int *skip) {
  if (*skip) return;
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)m * nrhs) return;
  const int i = (int)(t % m), j = (int)(t / m);
  DD s{0.0, 0.0};
  for (int cb = 0; cb < ncb; ++cb) s = dd_add(s, partial[((size_t)cb * nrhs + j) * m + i]);
  const DD r = dd_add(DD{B[i + (size_t)j * ldb], 0.0}, DD{-s.hi, -s.lo});
  R[i + (size_t)j * ldr] = __dadd_rn(r.hi, r.lo);
}

// colsum[j] = sum_i |A(i, j)| (one warp per column)
__global__ void __launch_bounds__(256) colsum_abs_kernel(int m, int n, const double *A, int lda, double *colsum) {
  const int j = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= n) return;
  double s = 0.0;
  for (int i = lane; i < m; i += 32) s += fabs(A[i + (size_t)j * lda]);
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
  if (lane == 0) colsum[j] = s;
}

// rowsum[i] = sum_j |A(i, j)|, i < m
__global__ void rowsum_abs_rect_kernel(int m, int n, const double *A, int lda, double *rowsum) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= m) return;
  double s = 0.0;
  for (int c = 0; c < n; ++c) s += fabs(A[i + (size_t)c * lda]);
  rowsum[i] = s;
}

// S(j, c) = sum_i A(i, j) R(i, c): one warp per column j of A, lanes down the
// rows (coalesced), every right-hand side accumulated per lane, then summed
// across the warp in a fixed order
template <int NC>  // right-hand sides per pass: 1 for a single one, else kResMaxRhs
__global__ void __launch_bounds__(kAtrWarps * 32) atr_kernel(int m, int n, int nrhs, const double *A, int lda,
                                                             const double *R, int ldr, double *S, int lds,
                                                             const int *skip) {
  if (*skip) return;
  const int j = blockIdx.x * kAtrWarps + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (j >= n) return;
  const double *a = A + (size_t)j * lda;
  for (int c0 = 0; c0 < nrhs; c0 += NC) {
    const int nc = min(NC, nrhs - c0);
    double acc[NC];
#pragma unroll
    for (int c = 0; c < NC; ++c) acc[c] = 0.0;
    for (int i = lane; i < m; i += 32) {
      const double v = a[i];
#pragma unroll
      for (int c = 0; c < NC; ++c)
        if (c < nc) acc[c] = fma(v, R[i + (size_t)(c0 + c) * ldr], acc[c]);
    }
#pragma unroll
    for (int c = 0; c < NC; ++c) {
      double v = acc[c];
#pragma unroll
      for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
      if (lane == 0 && c < nc) S[j + (size_t)(c0 + c) * lds] = v;
    }
  }
}

// berr[c] = ||S_c||inf / (||A||_1 (||A||inf ||X_c||inf + ||B_c||inf)), one CTA per column
__global__ void ls_berr_kernel(int m, int n, const double *S, int lds, const double *X, int ldx, const double *B,
                               int ldb, const double *anorm, const double *a1, double *berr, const int *skip) {
  if (*skip) return;
  const int c = blockIdx.x;
  double sv = 0.0, x = 0.0, b = 0.0;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    sv = fmax(sv, fabs(S[i + (size_t)c * lds]));
    x = fmax(x, fabs(X[i + (size_t)c * ldx]));
  }
  for (int i = threadIdx.x; i < m; i += blockDim.x) b = fmax(b, fabs(B[i + (size_t)c * ldb]));
  sv = block_max(sv);
  x = block_max(x);
  b = block_max(b);
  if (threadIdx.x == 0) {
    const double den = a1[0] * (anorm[0] * x + b);
    berr[c] = den > 0.0 ? sv / den : 0.0;
  }
}

// Rt = R^T (n x n, the upper triangle of QR's top n rows, lower triangular)
__global__ void transpose_upper_kernel(int n, const double *QR, int ldq, double *Rt, int ldt, const int *skip) {
  __shared__ double t[32][33];
  if (skip && *skip) return;
  const int bx = blockIdx.x * 32, by = blockIdx.y * 32;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 256 threads: 8 rows per pass
  for (int r = ty; r < 32; r += 8) {
    const int i = by + r, j = bx + tx;  // read R(i, j), i <= j
    t[r][tx] = (i < n && j < n && i <= j) ? QR[i + (size_t)j * ldq] : 0.0;
  }
  __syncthreads();
  for (int r = ty; r < 32; r += 8) {
    const int i = bx + r, j = by + tx;  // write Rt(i, j) = R(j, i)
    if (i < n && j < n) Rt[i + (size_t)j * ldt] = t[tx][r];
  }
}

// dx = max_j ||D_j||inf / ||X_j||inf of the correction D just solved (one CTA)
__global__ void ls_dxnorm_kernel(int n, int nrhs, const double *D, int ldd, const double *X, int ldx, IrCtl *ctl) {
  if (ctl->done) return;
  double best = 0.0;
  for (int j = 0; j < nrhs; ++j) {
    double d = 0.0, x = 0.0;
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
      d = fmax(d, fabs(D[i + (size_t)j * ldd]));
      x = fmax(x, fabs(X[i + (size_t)j * ldx]));
    }
    d = block_max(d);
    x = block_max(x);
    const double r = x > 0.0 ? d / x : d;
    best = (r > best || r != r) ? r : best;
  }
  if (threadIdx.x == 0) ctl->dx = best;
}

// The stop test of least-squares step `it`: the optimality measure
// ||A^T r|| / (||A||_1 (||A||inf ||x|| + ||b||)) alone can be tiny while the
// components of x along small singular directions are still off (it weighs
// them by sigma_min^2), so the loop runs until the corrections themselves
// stop mattering: the last correction is below 4 unit roundoffs of x, or it
// failed to halve twice in a row, or max_iter.  ok: the measure is <= tol.
__global__ void ls_decide_kernel(int it, int max_iter, double tol, int nrhs, const double *berr, IrCtl *ctl,
                                 double *berr_out, int *iters_out) {
  if (ctl->done) return;
  double be = 0.0;
  for (int j = 0; j < nrhs; ++j) be = (berr[j] > be || berr[j] != berr[j]) ? berr[j] : be;
  ctl->berr = be;
  ctl->iters = it;
  ctl->ok = be <= tol;
  if (berr_out) *berr_out = be;
  if (iters_out) *iters_out = ctl->iter_base + it;
  bool stop = false;
  if (it >= max_iter || !(be == be)) {
    stop = true;
  } else if (it > 0) {
    const double dx = ctl->dx;
    if (!(dx > 4.0 * 1.1102230246251565e-16)) {
      stop = true;
    } else if (dx > 0.5 * ctl->prev) {
      if (++ctl->stall >= 2) stop = true;
    } else {
      ctl->stall = 0;
    }
    ctl->prev = dx;
  } else if (be == 0.0) {
    stop = true;
  } else {
    ctl->prev = 1e308;
  }
  ctl->done = stop ? 1 : 0;
}

size_t ls_ws_bytes(int m, int n, int nrhs) {
  const int ncb = (n + kResCols - 1) / kResCols;
  return align256((size_t)ncb * nrhs * m * 16) + align256((size_t)m * nrhs * 8) + align256((size_t)n * nrhs * 8) +
         align256((size_t)n * n * 8) + align256((size_t)(m > n ? m : n) * 8) + 2 * align256(8) +
         align256((size_t)nrhs * 8) + kIrPhases * align256(sizeof(IrCtl)) + align256(8) + 256;
}

void ls_ws_carve(void *ws, int m, int n, int nrhs, LsWs &w) {
  const int ncb = (n + kResCols - 1) / kResCols;
  char *p = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  w.partial = (double *)p;
  p += align256((size_t)ncb * nrhs * m * 16);
  w.R = (double *)p;
  p += align256((size_t)m * nrhs * 8);
  w.S = (double *)p;
  p += align256((size_t)n * nrhs * 8);
  w.Rt = (double *)p;
  p += align256((size_t)n * n * 8);
  w.sums = (double *)p;
  p += align256((size_t)(m > n ? m : n) * 8);
  w.anorm = (double *)p;
  p += align256(8);
  w.a1 = (double *)p;
  p += align256(8);
  w.berr = (double *)p;
  p += align256((size_t)nrhs * 8);
  for (int i = 0; i < kIrPhases; ++i) {
    w.phase[i] = (IrCtl *)p;
    p += align256(sizeof(IrCtl));
  }
  w.ctl = w.phase[0];
  w.info2 = (int *)p;
}

cudaError_t ls_norms(int m, int n, const double *A, int lda, const LsWs &w, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 2.0 * m * (double)n);
  rowsum_abs_rect_kernel<<<(m + 255) / 256, 256, 0, st>>>(m, n, A, lda, w.sums);
  max_kernel<<<1, 1024, 0, st>>>(m, w.sums, w.anorm);
  colsum_abs_kernel<<<(n + 7) / 8, 256, 0, st>>>(m, n, A, lda, w.sums);
  max_kernel<<<1, 1024, 0, st>>>(n, w.sums, w.a1);
  return cudaGetLastError();
}

cudaError_t ls_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, const LsWs &w, cudaStream_t st) {
  const int *skip = &w.ctl->done;
  const int ncb = (n + kResCols - 1) / kResCols;
  DD *part = (DD *)w.partial;
  {
    ProfScope ps(kClsRefine, st, 2.0 * m * (double)n * nrhs);
    const dim3 grid((m + kResRows - 1) / kResRows, ncb);
    if (nrhs == 1)
      resid_partial_dd_kernel<1><<<grid, kResRows, 0, st>>>(m, n, nrhs, A, lda, X, ldx, part, skip);
    else
      resid_partial_dd_kernel<4><<<grid, kResRows, 0, st>>>(m, n, nrhs, A, lda, X, ldx, part, skip);
  }
  ProfScope ps(kClsRefine, st, 0.0);
  const long long tot = (long long)m * nrhs;
  resid_reduce_dd_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(m, nrhs, ncb, part, B, ldb, w.R, m, skip);
  return cudaGetLastError();
}

cudaError_t ls_normal_residual(int m, int n, int nrhs, const double *A, int lda, const double *X, int ldx,
                               const double *B, int ldb, const LsWs &w, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 2.0 * m * (double)n * nrhs);
  const unsigned g = (n + kAtrWarps - 1) / kAtrWarps;
  if (nrhs == 1)
    atr_kernel<1><<<g, kAtrWarps * 32, 0, st>>>(m, n, nrhs, A, lda, w.R, m, w.S, n, &w.ctl->done);
  else
    atr_kernel<kResMaxRhs><<<g, kAtrWarps * 32, 0, st>>>(m, n, nrhs, A, lda, w.R, m, w.S, n, &w.ctl->done);
  ls_berr_kernel<<<nrhs, 256, 0, st>>>(m, n, w.S, n, X, ldx, B, ldb, w.anorm, w.a1, w.berr, &w.ctl->done);
  return cudaGetLastError();
}

cudaError_t ls_transpose_r(int n, const double *QR, int ldq, const LsWs &w, const int *skip, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  dim3 g((n + 31) / 32, (n + 31) / 32);
  transpose_upper_kernel<<<g, 256, 0, st>>>(n, QR, ldq, w.Rt, n, skip);
  return cudaGetLastError();
}

cudaError_t ls_update(int n, int nrhs, const LsWs &w, double *X, int ldx, cudaStream_t st) {
  {
    ProfScope ps(kClsRefine, st, 0.0);
    ls_dxnorm_kernel<<<1, 256, 0, st>>>(n, nrhs, w.S, n, X, ldx, w.ctl);
  }
  ProfScope ps(kClsRefine, st, (double)n * nrhs);
  const long long tot = (long long)n * nrhs;
  axpy_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nrhs, w.S, n, X, ldx, &w.ctl->done);
  return cudaGetLastError();
}

cudaError_t ls_decide(int it, int max_iter, double tol, int nrhs, const LsWs &w, double *berr_out, int *iters_out,
                      cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  ls_decide_kernel<<<1, 1, 0, st>>>(it, max_iter, tol, nrhs, w.berr, w.ctl, berr_out, iters_out);
  return cudaGetLastError();
}

cudaError_t ls_begin(const LsWs &w, const IrCtl *prev, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  if (prev)
    begin_next_kernel<<<1, 1, 0, st>>>(prev, w.ctl, 1e308);
  else
    begin_kernel<<<1, 1, 0, st>>>(w.ctl, 1e308);
  return cudaGetLastError();
}

cudaError_t ls_merge_info(const LsWs &w, int *dev_info, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  merge_info_kernel<<<1, 1, 0, st>>>(w.ctl, w.info2, dev_info);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// GMRES on the preconditioned correction equation (M^-1 A) d = M^-1 r with
// M = P^T L U the reduced-precision factors (GMRES-based iterative
// refinement): x0 = 0, Arnoldi with classical Gram-Schmidt applied twice,
// Givens rotations on the Hessenberg matrix, stop when the preconditioned
// residual has dropped by kGmTol or after kGmMax steps; then d = V y and
// x += d.  All in FP64.  The control block lives in device memory; every
// kernel reads gm->stop (or gm->active) first, so the host enqueues kGmMax
// Arnoldi steps and the ones after convergence do nothing.
// ---------------------------------------------------------------------------
constexpr int kGmRows = 256;  // rows per CTA of the dot-product kernels

__global__ void gm_begin_kernel(const IrCtl *ctl, GmCtl *gm) {
  gm->active = !ctl->done;
  gm->stop = !gm->active;
  gm->k = 0;
  gm->beta = 0.0;
}

// dst = column j of R (the current residual)
__global__ void gm_copy_kernel(int n, const double *src, double *dst, const GmCtl *gm) {
  if (gm->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i];
}

__device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  __syncthreads();
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double s = 0.0;
  for (int w = 0; w < (int)(blockDim.x >> 5); ++w) s += red[w];
  return s;
}

// partial[blk * (kGmMax + 1) + c] = sum over this CTA's rows of V(:, c) w,
// c < ncols (the columns of V, or w itself when V == w and ncols == 1)
__global__ void __launch_bounds__(kGmRows) gm_dots_kernel(int n, int ncols, const double *V, int ldv,
                                                          const double *w, double *partial, const GmCtl *gm) {
  __shared__ double red[kGmRows / 32];
  if (gm->stop) return;
  const int i = blockIdx.x * kGmRows + threadIdx.x;
  const double wi = i < n ? w[i] : 0.0;
  for (int c = 0; c < ncols; ++c) {
    const double v = i < n ? V[i + (size_t)c * ldv] : 0.0;
    const double s = block_sum(v * wi, red);
    if (threadIdx.x == 0) partial[(size_t)blockIdx.x * (kGmMax + 1) + c] = s;
  }
}

// h[c] = sum_blk partial[blk][c] in a fixed order; accumulate: H(:, j) += h
// (second Gram-Schmidt pass) or H(:, j) = h (first); norm: h is ||w||^2.
__global__ void gm_finish_kernel(int nblk, int ncols, const double *partial, GmCtl *gm, int j, int pass) {
  if (gm->stop) return;
  const int c = threadIdx.x;
  if (c >= ncols) return;
  double s = 0.0;
  for (int b = 0; b < nblk; ++b) s += partial[(size_t)b * (kGmMax + 1) + c];
  gm->h[c] = s;
  if (pass == 1) gm->H[c + j * (kGmMax + 1)] = s;
  if (pass == 2) gm->H[c + j * (kGmMax + 1)] += s;
}

// w -= V(:, 0:ncols) h
__global__ void gm_axpy_kernel(int n, int ncols, const double *V, int ldv, double *w, const GmCtl *gm) {
  if (gm->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = w[i];
  for (int c = 0; c < ncols; ++c) s = fma(-V[i + (size_t)c * ldv], gm->h[c], s);
  w[i] = s;
}

// beta = ||M^-1 r|| (from gm->h[0] = its square), g = beta e1; nothing to do
// for a zero residual
__global__ void gm_start_kernel(GmCtl *gm) {
  if (gm->stop) return;
  const double beta = sqrt(gm->h[0]);
  gm->beta = beta;
  for (int i = 0; i <= kGmMax; ++i) gm->g[i] = 0.0;
  gm->g[0] = beta;
  gm->scale = beta > 0.0 ? 1.0 / beta : 0.0;
  if (!(beta > 0.0)) gm->stop = 1;
}

// Arnoldi step j done: H(j+1, j) = ||w|| (gm->h[0] = its square); the
// earlier rotations are applied to H(:, j), a new one zeroes H(j+1, j), g is
// rotated; converged when |g(j+1)| <= tol beta.
__global__ void gm_givens_kernel(GmCtl *gm, int j, double tol) {
  if (gm->stop) return;
  double *H = gm->H + j * (kGmMax + 1);
  const double hn = sqrt(gm->h[0]);
  for (int i = 0; i < j; ++i) {
    const double a = H[i], b = H[i + 1];
    H[i] = gm->cs[i] * a + gm->sn[i] * b;
    H[i + 1] = -gm->sn[i] * a + gm->cs[i] * b;
  }
  const double a = H[j];
  const double r = hypot(a, hn);
  const double c = r > 0.0 ? a / r : 1.0, s = r > 0.0 ? hn / r : 0.0;
  gm->cs[j] = c;
  gm->sn[j] = s;
  H[j] = r;
  H[j + 1] = 0.0;
  gm->g[j + 1] = -s * gm->g[j];
  gm->g[j] = c * gm->g[j];
  gm->k = j + 1;
  gm->scale = hn > 0.0 ? 1.0 / hn : 0.0;
  if (fabs(gm->g[j + 1]) <= tol * gm->beta || j + 1 >= kGmMax || !(hn > 0.0)) gm->stop = 1;
}

// dst = scale * src (the next Arnoldi vector, or the first one)
__global__ void gm_scale_kernel(int n, const double *src, double *dst, const GmCtl *gm) {
  if (gm->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) dst[i] = src[i] * gm->scale;
}

// y = R^-1 g over the k accepted steps (R: the rotated Hessenberg matrix)
__global__ void gm_solve_kernel(GmCtl *gm) {
  if (!gm->active) return;
  const int k = gm->k;
  for (int i = k - 1; i >= 0; --i) {
    double s = gm->g[i];
    for (int c = i + 1; c < k; ++c) s -= gm->H[i + c * (kGmMax + 1)] * gm->y[c];
    gm->y[i] = s / gm->H[i + i * (kGmMax + 1)];
  }
}

// x += V(:, 0:k) y
__global__ void gm_xupdate_kernel(int n, const double *V, int ldv, double *x, const GmCtl *gm) {
  if (!gm->active) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int c = 0; c < gm->k; ++c) s = fma(V[i + (size_t)c * ldv], gm->y[c], s);
  x[i] += s;
}

// w = A v (one thread per row, column blocks reduced in a fixed order)
__global__ void gm_gemv_reduce_kernel(int n, int ncb, const double *partial, double *w, const GmCtl *gm) {
  if (gm->stop) return;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double s = 0.0;
  for (int cb = 0; cb < ncb; ++cb) s += partial[(size_t)cb * n + i];
  w[i] = s;
}

size_t gm_ws_bytes(int n) {
  const int nblk = (n + kGmRows - 1) / kGmRows;
  const int ncb = (n + kResCols - 1) / kResCols;
  return align256((size_t)n * (kGmMax + 1) * 8) + align256((size_t)n * 8) +
         align256((size_t)nblk * (kGmMax + 1) * 8) + align256((size_t)ncb * n * 8) + align256(sizeof(GmCtl)) +
         256;
}

void gm_ws_carve(void *ws, int n, GmWs &g) {
  const int nblk = (n + kGmRows - 1) / kGmRows;
  const int ncb = (n + kResCols - 1) / kResCols;
  char *p = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  g.V = (double *)p;
  p += align256((size_t)n * (kGmMax + 1) * 8);
  g.w = (double *)p;
  p += align256((size_t)n * 8);
  g.partial = (double *)p;
  p += align256((size_t)nblk * (kGmMax + 1) * 8);
  g.mv = (double *)p;
  p += align256((size_t)ncb * n * 8);
  g.ctl = (GmCtl *)p;
}

// The GMRES correction of right-hand side j: x(:, j) += d with
// (M^-1 A) d = M^-1 r_j, M the factors in LU / ipiv.
cudaError_t ir_gmres_correction(int n, const double *A, int lda, const double *LU, int ldlu, const int *ipiv,
                                const IrWs &w, const GmWs &g, int j, double *X, int ldx, const SolveWs &sw,
                                int *status, int status_bit, cudaStream_t st) {
  const int *stop = &g.ctl->stop;
  const int nb = (n + 255) / 256;
  const int nblk = (n + kGmRows - 1) / kGmRows;
  const int ncb = (n + kResCols - 1) / kResCols;
  cudaError_t e;
  auto prec_solve = [&](double *v) -> cudaError_t {  // v <- M^-1 v
    cudaError_t e2 = getrs_swap(n, 1, ipiv, v, n, st, stop);
    if (e2 != cudaSuccess) return e2;
    if ((e2 = trsm_left(true, true, n, 1, LU, ldlu, v, n, sw, status, status_bit, stop, st)) != cudaSuccess)
      return e2;
    return trsm_left(false, false, n, 1, LU, ldlu, v, n, sw, status, status_bit, stop, st);
  };
  auto norm2 = [&](const double *v) -> cudaError_t {  // gm->h[0] = ||v||^2
    gm_dots_kernel<<<nblk, kGmRows, 0, st>>>(n, 1, v, n, v, g.partial, g.ctl);
    gm_finish_kernel<<<1, 32, 0, st>>>(nblk, 1, g.partial, g.ctl, 0, 0);
    return cudaGetLastError();
  };
  {
    ProfScope ps(kClsRefine, st, 0.0);
    gm_begin_kernel<<<1, 1, 0, st>>>(w.ctl, g.ctl);
    gm_copy_kernel<<<nb, 256, 0, st>>>(n, w.R + (size_t)j * n, g.V, g.ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  if ((e = prec_solve(g.V)) != cudaSuccess) return e;
  {
    ProfScope ps(kClsRefine, st, 2.0 * n);
    if ((e = norm2(g.V)) != cudaSuccess) return e;
    gm_start_kernel<<<1, 1, 0, st>>>(g.ctl);
    gm_scale_kernel<<<nb, 256, 0, st>>>(n, g.V, g.V, g.ctl);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
  }
  for (int s = 0; s < kGmMax; ++s) {
    double *vs = g.V + (size_t)s * n;
    {  // w = A v_s
      ProfScope ps(kClsRefine, st, 2.0 * n * (double)n);
      resid_partial_kernel<1><<<dim3((n + kResRows - 1) / kResRows, ncb), kResRows, 0, st>>>(n, n, 1, A, lda, vs,
                                                                                              n, g.mv, stop);
      gm_gemv_reduce_kernel<<<nb, 256, 0, st>>>(n, ncb, g.mv, g.w, g.ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if ((e = prec_solve(g.w)) != cudaSuccess) return e;  // w = M^-1 A v_s
    {
      ProfScope ps(kClsRefine, st, 8.0 * n * (s + 1) + 2.0 * n);
      for (int pass = 1; pass <= 2; ++pass) {  // classical Gram-Schmidt, twice
        gm_dots_kernel<<<nblk, kGmRows, 0, st>>>(n, s + 1, g.V, n, g.w, g.partial, g.ctl);
        gm_finish_kernel<<<1, 32, 0, st>>>(nblk, s + 1, g.partial, g.ctl, s, pass);
        gm_axpy_kernel<<<nb, 256, 0, st>>>(n, s + 1, g.V, n, g.w, g.ctl);
      }
      if ((e = norm2(g.w)) != cudaSuccess) return e;
      gm_givens_kernel<<<1, 1, 0, st>>>(g.ctl, s, kGmTol);
      gm_scale_kernel<<<nb, 256, 0, st>>>(n, g.w, g.V + (size_t)(s + 1) * n, g.ctl);
      if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
  }
  ProfScope ps(kClsRefine, st, 2.0 * n * kGmMax);
  gm_solve_kernel<<<1, 1, 0, st>>>(g.ctl);
  gm_xupdate_kernel<<<nb, 256, 0, st>>>(n, g.V, n, X + (size_t)j * ldx, g.ctl);
  return cudaGetLastError();
}

}  // namespace cagb
