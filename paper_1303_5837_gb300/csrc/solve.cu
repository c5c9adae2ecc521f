// solve.cu -- triangular solves and row interchanges that consume the
// factors (PA = LU: swaps, unit-lower forward and upper back substitution;
// A = QR: back substitution with R after Q^T is applied through the tree).
//
// Blocked by kTb rows: the diagonal block is solved by one CTA in shared
// memory, then the rows below (or above) are updated -- for few right-hand
// sides in one cooperative launch, otherwise with one launch per block and
// the FP64 GEMM.
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

// ---------------------------------------------------------------------------
// Few right-hand sides: one cooperative launch over every SM.
//   Phase 0: CTA c inverts diagonal block c of T in place in its shared memory
//            (LAPACK trti2 order, unit lower or non-unit upper), so no block
//            step needs a serial substitution chain.
//   Per block (forward for L, backward for U): the owning CTA computes
//            x_i = T_ii^-1 b_i (a GEMV from shared memory); grid-wide sync;
//            every CTA updates its share of the rows below / above
//            (b_r -= T(r, block) x_i, rows coalesced); grid-wide sync.
// Needs one CTA per diagonal block: n <= gridDim.x * kTb.
// ---------------------------------------------------------------------------
constexpr int kCoopMaxRhs = 16;
constexpr int kLdI = kTb + 1;

__global__ void __launch_bounds__(256, 1) trsv_coop_kernel(int n, int nrhs, const double *T, int ldt, double *B,
                                                           int ldb, int lower, int unit) {
  cg::grid_group grid = cg::this_grid();
  extern __shared__ __align__(16) double csm[];
  double *Ti = csm;                      // the inverted diagonal block, ld kLdI
  double *tmp = Ti + kTb * kLdI;         // kTb column buffer
  double *xs = tmp + kTb;                // kTb x nrhs solved block
  const int tid = threadIdx.x;
  const int nblk = (n + kTb - 1) / kTb;
  const long long nthreads = (long long)gridDim.x * blockDim.x;
  const long long gtid = (long long)blockIdx.x * blockDim.x + tid;

  // ---- phase 0: invert my diagonal block ----------------------------------
  const int myblk = blockIdx.x;
  if (myblk < nblk) {
    const int r0 = myblk * kTb, nb = min(kTb, n - r0);
    for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
      const int i = idx % nb, k = idx / nb;
      const bool keep = lower ? (i >= k) : (i <= k);
      Ti[i + k * kLdI] = keep ? T[(r0 + i) + (size_t)(r0 + k) * ldt] : 0.0;
    }
    __syncthreads();
    if (lower) {
      // unit lower: columns right to left; X(j+1:, j) = -X(j+1:, j+1:) T(j+1:, j)
      for (int j = nb - 1; j >= 0; --j) {
        for (int i = j + 1 + tid; i < nb; i += blockDim.x) {
          double acc = 0.0;
          for (int k = j + 1; k <= i; ++k) acc = fma(Ti[i + k * kLdI], Ti[k + j * kLdI], acc);
          tmp[i] = -acc;
        }
        __syncthreads();
        for (int i = j + 1 + tid; i < nb; i += blockDim.x) Ti[i + j * kLdI] = tmp[i];
        if (tid == 0) Ti[j + j * kLdI] = 1.0;
        __syncthreads();
      }
    } else {
      // non-unit upper: columns left to right; X(j, j) = 1 / T(j, j),
      // X(0:j, j) = -X(j, j) X(0:j, 0:j) T(0:j, j)
      for (int i = tid; i < nb; i += blockDim.x) xs[i] = 1.0 / Ti[i + i * kLdI];  // all pivots at once
      __syncthreads();
      for (int j = 0; j < nb; ++j) {
        const double djj = xs[j];
        for (int i = tid; i < j; i += blockDim.x) {
          double acc = 0.0;
          for (int k = i; k < j; ++k) acc = fma(Ti[i + k * kLdI], Ti[k + j * kLdI], acc);
          tmp[i] = -djj * acc;
        }
        __syncthreads();
        for (int i = tid; i < j; i += blockDim.x) Ti[i + j * kLdI] = tmp[i];
        if (tid == 0) Ti[j + j * kLdI] = djj;
        __syncthreads();
      }
    }
  }
  grid.sync();

  for (int s = 0; s < nblk; ++s) {
    const int blk = lower ? s : nblk - 1 - s;
    const int r0 = blk * kTb;
    const int nb = min(kTb, n - r0);
    // x_blk = T_ii^-1 b_blk by the CTA that holds the inverse
    if (blockIdx.x == blk) {
      for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
        const int k = idx % nb, c = idx / nb;
        xs[k + c * kTb] = B[(r0 + k) + (size_t)c * ldb];
      }
      __syncthreads();
      for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
        const int i = idx % nb, c = idx / nb;
        double acc = 0.0;
        for (int k = 0; k < nb; ++k) acc = fma(Ti[i + k * kLdI], xs[k + c * kTb], acc);
        B[(r0 + i) + (size_t)c * ldb] = acc;
      }
    }
    grid.sync();
    // rows outside the block: below it (lower) or above it (upper)
    const int rlo = lower ? r0 + nb : 0, rhi = lower ? n : r0;
    if (rhi > rlo) {
      for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
        const int k = idx % nb, c = idx / nb;
        xs[k + c * kTb] = B[(r0 + k) + (size_t)c * ldb];
      }
      __syncthreads();
      for (long long r = rlo + gtid; r < rhi; r += nthreads) {
        double acc[kCoopMaxRhs];
#pragma unroll
        for (int c = 0; c < kCoopMaxRhs; ++c) acc[c] = 0.0;
        const double *tr = T + r + (size_t)r0 * ldt;
#pragma unroll 16
        for (int k = 0; k < nb; ++k) {  // unrolled: many loads of T in flight per thread
          const double tv = tr[(size_t)k * ldt];
#pragma unroll
          for (int c = 0; c < kCoopMaxRhs; ++c)
            if (c < nrhs) acc[c] = fma(tv, xs[k + c * kTb], acc[c]);
        }
#pragma unroll
        for (int c = 0; c < kCoopMaxRhs; ++c)
          if (c < nrhs) B[r + (size_t)c * ldb] -= acc[c];
      }
    }
    grid.sync();
  }
}

// one CTA per SM, one diagonal block per CTA
static int coop_max_n() {
  static int sms = 0;
  if (sms == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      sms = 1;
  }
  return sms * kTb;
}

static cudaError_t trsm_left_coop(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B,
                                  int ldb, cudaStream_t st) {
  static int grid = 0;
  const size_t smem = ((size_t)kTb * kLdI + kTb + (size_t)kTb * kCoopMaxRhs) * 8;
  if (grid == 0) {
    cudaError_t e = cudaFuncSetAttribute(trsv_coop_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, trsv_coop_kernel, 256, smem)) != cudaSuccess)
      return e;
    if (per < 1) return cudaErrorInvalidConfiguration;
    grid = sms;  // one CTA per SM: every CTA resident, as the grid-wide sync requires
  }
  int lo = lower ? 1 : 0, un = unit ? 1 : 0;
  void *args[] = {&n, &nrhs, (void *)&T, &ldt, &B, &ldb, &lo, &un};
  ProfScope ps(kClsSolve, st, (double)n * n * nrhs);
  return cudaLaunchCooperativeKernel((void *)trsv_coop_kernel, dim3(grid), dim3(256), args, smem, st);
}

cudaError_t trsm_left(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B,
                      int ldb, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs <= kCoopMaxRhs && n > kTb && n <= coop_max_n()) return trsm_left_coop(lower, unit, n, nrhs, T, ldt, B, ldb, st);
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
