// ir.cu -- FP64 pieces of iterative refinement around the reduced-precision
// factorization: residual R = B - A X, norms, backward error, X += D.
//
// The residual is the one place refinement needs full FP64 (Sec. 5.1 measures
// the normwise backward error ||b - A x|| / (||A|| ||x|| + ||b||), infinity
// norms): one pass over A, FP64 DFMA, column blocks reduced in a fixed order.
#include "ca_internal.cuh"

namespace cagb {

constexpr int kResRows = 256;    // rows per CTA (one thread per row)
constexpr int kResCols = 1024;   // columns of A per CTA
constexpr int kResMaxRhs = 16;

// partial[cb][j][i] = sum_{c in block cb} A(i, c) X(c, j)
__global__ void __launch_bounds__(kResRows) resid_partial_kernel(int n, int ncols, int nrhs, const double *A,
                                                                 int lda, const double *X, int ldx,
                                                                 double *partial) {
  __shared__ double xs[kResCols * 4];
  const int i = blockIdx.x * kResRows + threadIdx.x;
  const int c0 = blockIdx.y * kResCols;
  const int nc = min(kResCols, ncols - c0);
  for (int j0 = 0; j0 < nrhs; j0 += 4) {  // right-hand sides four at a time
    const int nj = min(4, nrhs - j0);
    __syncthreads();
    for (int idx = threadIdx.x; idx < nc * 4; idx += kResRows) {
      int c = idx % nc, j = idx / nc;
      xs[j * kResCols + c] = (j < nj) ? X[(c0 + c) + (size_t)(j0 + j) * ldx] : 0.0;
    }
    __syncthreads();
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
    if (i < n) {
      const double *a = A + i + (size_t)c0 * lda;
#pragma unroll 4
      for (int c = 0; c < nc; ++c) {
        const double v = a[(size_t)c * lda];
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[j] = fma(v, xs[j * kResCols + c], acc[j]);
      }
#pragma unroll
      for (int j = 0; j < 4; ++j)
        if (j < nj) partial[((size_t)blockIdx.y * nrhs + j0 + j) * n + i] = acc[j];
    }
  }
}

// R = B - sum_cb partial[cb]
__global__ void resid_reduce_kernel(int n, int nrhs, int ncb, const double *partial, const double *B, int ldb,
                                    double *R, int ldr) {
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
                            const double *anorm, double *berr) {
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

__global__ void axpy_kernel(int n, int nrhs, const double *D, int ldd, double *X, int ldx) {
  const long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)n * nrhs) return;
  const int i = (int)(t % n), j = (int)(t / n);
  X[i + (size_t)j * ldx] += D[i + (size_t)j * ldd];
}

size_t ir_ws_bytes(int n, int nrhs) {
  const int ncb = (n + kResCols - 1) / kResCols;
  return align256((size_t)ncb * nrhs * n * 8) + align256((size_t)n * nrhs * 8) + align256((size_t)n * 8) +
         align256(8) + align256((size_t)nrhs * 8) + 256;
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

cudaError_t ir_residual(int n, int nrhs, const double *A, int lda, const double *X, int ldx, const double *B,
                        int ldb, const IrWs &w, cudaStream_t st) {
  if (nrhs > kResMaxRhs) {
    // wide right-hand sides: R = B, then R -= A X with the FP64 GEMM
    cudaError_t e = cudaMemcpy2DAsync(w.R, (size_t)n * 8, B, (size_t)ldb * 8, (size_t)n * 8, nrhs,
                                      cudaMemcpyDeviceToDevice, st);
    if (e != cudaSuccess) return e;
    return gemm_minus_f64(n, nrhs, n, A, lda, X, ldx, w.R, n, st);
  }
  const int ncb = (n + kResCols - 1) / kResCols;
  {
    ProfScope ps(kClsRefine, st, 2.0 * n * (double)n * nrhs);
    resid_partial_kernel<<<dim3((n + kResRows - 1) / kResRows, ncb), kResRows, 0, st>>>(n, n, nrhs, A, lda, X,
                                                                                         ldx, w.partial);
  }
  ProfScope ps(kClsRefine, st, 0.0);
  const long long tot = (long long)n * nrhs;
  resid_reduce_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nrhs, ncb, w.partial, B, ldb, w.R, n);
  return cudaGetLastError();
}

cudaError_t ir_berr(int n, int nrhs, const double *X, int ldx, const double *B, int ldb, const IrWs &w,
                    cudaStream_t st) {
  ProfScope ps(kClsRefine, st, 0.0);
  berr_kernel<<<nrhs, 256, 0, st>>>(n, w.R, n, X, ldx, B, ldb, w.anorm, w.berr);
  return cudaGetLastError();
}

cudaError_t ir_update(int n, int nrhs, const IrWs &w, double *X, int ldx, cudaStream_t st) {
  ProfScope ps(kClsRefine, st, (double)n * nrhs);
  const long long tot = (long long)n * nrhs;
  axpy_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, st>>>(n, nrhs, w.R, n, X, ldx);
  return cudaGetLastError();
}

}  // namespace cagb
