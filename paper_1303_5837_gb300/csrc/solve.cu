// solve.cu -- triangular solves and row interchanges that consume the
// factors (PA = LU: swaps, unit-lower forward and upper back substitution;
// A = QR: back substitution with R after Q^T is applied through the tree).
//
// Blocked by kTb rows: the diagonal block is solved by one CTA in shared
// memory, then the rows below (or above) are updated with the FP64 GEMM.
#include "ca_internal.cuh"

namespace cagb {

constexpr int kTb = 128;

// Row interchanges of LAPACK laswp (forward), one CTA per right-hand side;
// the column is staged in shared memory when it fits.
__global__ void __launch_bounds__(32) swap_rows_kernel(int n, const int *ipiv, double *B, int ldb,
                                                       int staged) {
  extern __shared__ __align__(16) double col[];
  double *b = B + (size_t)blockIdx.x * ldb;
  const int lane = threadIdx.x;
  if (staged) {
    for (int i = lane; i < n; i += 32) col[i] = b[i];
    __syncwarp();
    if (lane == 0)
      for (int i = 0; i < n; ++i) {
        int p = ipiv[i] - 1;
        if (p != i) {
          double t = col[i];
          col[i] = col[p];
          col[p] = t;
        }
      }
    __syncwarp();
    for (int i = lane; i < n; i += 32) b[i] = col[i];
  } else if (lane == 0) {
    for (int i = 0; i < n; ++i) {
      int p = ipiv[i] - 1;
      if (p != i) {
        double t = b[i];
        b[i] = b[p];
        b[p] = t;
      }
    }
  }
}

cudaError_t getrs_swap(int n, int nrhs, const int *ipiv, double *B, int ldb, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(swap_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         200 * 1024);
    if (e != cudaSuccess) return e;
    init = true;
  }
  int staged = ((size_t)n * 8 <= 200 * 1024) ? 1 : 0;
  ProfScope ps(kClsSolve, st, 0.0);
  swap_rows_kernel<<<nrhs, 32, staged ? (size_t)n * 8 : 0, st>>>(n, ipiv, B, ldb, staged);
  return cudaGetLastError();
}

// Solve the nb x nb diagonal block T11 X = B1 in place (nb <= kTb) for all
// right-hand sides, one CTA per tile of 32 right-hand sides.
__global__ void __launch_bounds__(256) trsm_diag_kernel(int nb, int nrhs, const double *T, int ldt,
                                                        double *B, int ldb, int lower, int unit) {
  extern __shared__ __align__(16) double tsm[];
  double(*Ts)[kTb + 1] = reinterpret_cast<double(*)[kTb + 1]>(tsm);
  double(*Xs)[33] = reinterpret_cast<double(*)[33]>(tsm + kTb * (kTb + 1));
  const int tid = threadIdx.x;
  const int c0 = blockIdx.x * 32;
  const int nc = min(32, nrhs - c0);
  for (int idx = tid; idx < nb * nb; idx += 256) {
    int i = idx % nb, k = idx / nb;
    Ts[i][k] = T[i + (size_t)k * ldt];
  }
  for (int idx = tid; idx < nb * nc; idx += 256) {
    int i = idx % nb, c = idx / nb;
    Xs[i][c] = B[i + (size_t)(c0 + c) * ldb];
  }
  __syncthreads();
  // column-oriented substitution: finalize x_j, then update the rest
  for (int s = 0; s < nb; ++s) {
    const int j = lower ? s : nb - 1 - s;
    if (!unit) {
      const double d = Ts[j][j];
      for (int c = tid; c < nc; c += 256) Xs[j][c] = Xs[j][c] / d;
      __syncthreads();
    }
    const int lo = lower ? j + 1 : 0, hi = lower ? nb : j;
    const int nr = hi - lo;
    for (int idx = tid; idx < nr * nc; idx += 256) {
      int i = lo + idx % nr, c = idx / nr;
      Xs[i][c] = fma(-Ts[i][j], Xs[j][c], Xs[i][c]);
    }
    __syncthreads();
  }
  for (int idx = tid; idx < nb * nc; idx += 256) {
    int i = idx % nb, c = idx / nb;
    B[i + (size_t)(c0 + c) * ldb] = Xs[i][c];
  }
}

cudaError_t trsm_left(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B,
                      int ldb, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  const size_t smem = ((size_t)kTb * (kTb + 1) + (size_t)kTb * 33) * 8;
  static bool init = false;
  if (!init) {
    cudaError_t e = cudaFuncSetAttribute(trsm_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    init = true;
  }
  const int nblk = (n + kTb - 1) / kTb;
  const dim3 g((nrhs + 31) / 32);
  for (int s = 0; s < nblk; ++s) {
    const int blk = lower ? s : nblk - 1 - s;
    const int r0 = blk * kTb;
    const int nb = min(kTb, n - r0);
    {
      ProfScope ps(kClsSolve, st, (double)nb * nb * nrhs);
      trsm_diag_kernel<<<g, 256, smem, st>>>(nb, nrhs, T + r0 + (size_t)r0 * ldt, ldt, B + r0, ldb,
                                          lower ? 1 : 0, unit ? 1 : 0);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (lower) {
      const int rest = n - r0 - nb;
      e = gemm_minus_f64(rest, nrhs, nb, T + (r0 + nb) + (size_t)r0 * ldt, ldt, B + r0, ldb,
                         B + r0 + nb, ldb, st);
    } else {
      e = gemm_minus_f64(r0, nrhs, nb, T + (size_t)r0 * ldt, ldt, B + r0, ldb, B, ldb, st);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cagb
