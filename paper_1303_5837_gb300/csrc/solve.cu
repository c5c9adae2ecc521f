// solve.cu -- triangular solves and row interchanges that consume the
// factors (PA = LU: swaps, unit-lower forward and upper back substitution;
// A = QR: back substitution with R after Q^T is applied through the tree).
//
// Blocked by kTb rows: for few right-hand sides one cooperative launch with
// one CTA per diagonal block, ordered by ready flags; otherwise the diagonal
// block is solved by one CTA in shared memory and the rows below (or above)
// are updated with the FP64 GEMM, one launch per block.
#include <mutex>

#include "ca_internal.cuh"
#include "device_once.cuh"

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
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(swap_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e != cudaSuccess) return e;
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
// Few right-hand sides: one cooperative launch, one CTA per diagonal block,
// ordered by per-block ready flags instead of grid-wide barriers.
//   Phase 0: CTA c inverts diagonal block c of T in its shared memory
//            (LAPACK trti2 order, unit lower or non-unit upper).
//   Then CTA c takes the blocks it depends on in order (the ones before it
//   for L, after it for U): it waits until block j's solution is published
//   (flag j), subtracts T(c, j) x_j from its right-hand sides, and after the
//   last one computes x_c = T_cc^-1 b_c, writes it to B and publishes flag c.
//   The chain of dependent steps is one GEMV of a 128 x 128 block and one
//   small triangular multiply per block; the earlier GEMVs of a CTA overlap
//   with the chain.  The cooperative launch makes every CTA resident, as the
//   waits require; every wait is bounded (about 2 s of SM clock), after
//   which the CTA records the timeout in the flag word after the last block
//   and leaves.
// Needs one CTA per diagonal block: n <= SMs * kTb.
// ---------------------------------------------------------------------------
constexpr int kCoopMaxRhs = 16;
constexpr int kLdI = kTb + 1;
constexpr int kMaxFlagBlocks = 1024;            // flag words per stream (covers any SM count here)
constexpr long long kSolveWaitLimit = 4000000000ll;

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

__global__ void __launch_bounds__(256, 1) trsv_flag_kernel(int n, int nrhs, const double *T, int ldt, double *B,
                                                           int ldb, int lower, int unit, int *flags) {
  extern __shared__ __align__(16) double csm[];
  double *Ti = csm;                          // the inverted diagonal block, ld kLdI
  double *tmp = Ti + kTb * kLdI;             // kTb column buffer
  double *sb = tmp + kTb;                    // kTb x nrhs: my right-hand sides being reduced
  double *xj = sb + kTb * kCoopMaxRhs;       // kTb x nrhs: a published solution block
  double *part = xj + kTb * kCoopMaxRhs;     // 2 x kTb x nrhs: half-row partial sums
  __shared__ int abort_flag;
  const int tid = threadIdx.x;
  const int nblk = (n + kTb - 1) / kTb;
  const int blk = blockIdx.x;
  if (blk >= nblk) return;
  const int r0 = blk * kTb, nb = min(kTb, n - r0);

  // ---- phase 0: invert my diagonal block ----------------------------------
  for (int idx = tid; idx < nb * nb; idx += blockDim.x) {
    const int i = idx % nb, k = idx / nb;
    const bool keep = lower ? (i >= k) : (i <= k);
    Ti[i + k * kLdI] = keep ? T[(r0 + i) + (size_t)(r0 + k) * ldt] : 0.0;
  }
  for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
    const int k = idx % nb, c = idx / nb;
    sb[k + c * kTb] = B[(r0 + k) + (size_t)c * ldb];
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
    for (int i = tid; i < nb; i += blockDim.x) xj[i] = 1.0 / Ti[i + i * kLdI];  // all pivots at once
    __syncthreads();
    for (int j = 0; j < nb; ++j) {
      const double djj = xj[j];
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

  // ---- the blocks this one depends on, in order ----------------------------
  const int ndep = lower ? blk : nblk - 1 - blk;
  const int r = tid & (kTb - 1), half = tid >> 7;  // row of my block, half of the columns
  for (int t = 0; t < ndep; ++t) {
    const int j = lower ? t : nblk - 1 - t;
    const int c0 = j * kTb, nbj = min(kTb, n - c0);
    // prefetch this thread's half row of T(blk, j) while waiting
    double trow[kTb / 2];
    const int k0 = half * (kTb / 2);
#pragma unroll
    for (int k = 0; k < kTb / 2; ++k)
      trow[k] = (r < nb && k0 + k < nbj) ? T[(r0 + r) + (size_t)(c0 + k0 + k) * ldt] : 0.0;
    if (tid == 0) {
      const long long tstart = clock64();
      int ok = 1;
      while (ld_acquire_gpu(flags + j) == 0) {
        if (clock64() - tstart > kSolveWaitLimit) {
          ok = 0;
          atomicOr(flags + kMaxFlagBlocks, 1);  // the timeout word
          break;
        }
      }
      abort_flag = !ok;
    }
    __syncthreads();
    if (abort_flag) return;
    for (int idx = tid; idx < nbj * nrhs; idx += blockDim.x) {
      const int k = idx % nbj, c = idx / nbj;
      xj[k + c * kTb] = __ldcg(B + (c0 + k) + (size_t)c * ldb);
    }
    __syncthreads();
    if (nrhs == 1) {  // one right-hand side: four independent partial sums
      double a4[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int k = 0; k < kTb / 2; ++k) a4[k & 3] = fma(trow[k], xj[k0 + k], a4[k & 3]);
      part[half * kTb * kCoopMaxRhs + r] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    } else {
      double acc[kCoopMaxRhs];
#pragma unroll
      for (int c = 0; c < kCoopMaxRhs; ++c) acc[c] = 0.0;
#pragma unroll
      for (int k = 0; k < kTb / 2; ++k) {
        const double tv = trow[k];
#pragma unroll
        for (int c = 0; c < kCoopMaxRhs; ++c)
          if (c < nrhs) acc[c] = fma(tv, xj[k0 + k + c * kTb], acc[c]);
      }
#pragma unroll
      for (int c = 0; c < kCoopMaxRhs; ++c)
        if (c < nrhs) part[half * kTb * kCoopMaxRhs + r + c * kTb] = acc[c];
    }
    __syncthreads();
    for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
      const int i = idx % nb, c = idx / nb;
      sb[i + c * kTb] -= part[i + c * kTb] + part[kTb * kCoopMaxRhs + i + c * kTb];
    }
    __syncthreads();
  }

  // ---- x = T_blk^-1 b_blk, published ---------------------------------------
  for (int idx = tid; idx < nb * nrhs; idx += blockDim.x) {
    const int i = idx % nb, c = idx / nb;
    double acc = 0.0;
    for (int k = 0; k < nb; ++k) acc = fma(Ti[i + k * kLdI], sb[k + c * kTb], acc);
    B[(r0 + i) + (size_t)c * ldb] = acc;
  }
  __threadfence();
  __syncthreads();
  if (tid == 0) st_release_gpu(flags + blk, 1);
}

// Flag words of the dependency-driven solve: one array per (device, caller
// stream), created on first use (make the first solve on a stream before
// capturing it in a graph) and kept until the process exits.
struct FlagPool {
  struct Entry {
    int dev;
    cudaStream_t st;
    int *flags;
  };
  std::mutex mu;
  Entry pool[64];
  int used = 0;
};

static FlagPool &flag_pool() {
  static FlagPool p;
  return p;
}

// The flag array of (current device, st), or nullptr if none exists and
// `create` is false (or it cannot be created).
static int *solve_flags_lookup(cudaStream_t st, bool create) {
  FlagPool &fp = flag_pool();
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return nullptr;
  std::lock_guard<std::mutex> g(fp.mu);
  for (int i = 0; i < fp.used; ++i)
    if (fp.pool[i].dev == dev && fp.pool[i].st == st) return fp.pool[i].flags;
  if (!create || fp.used == 64) return nullptr;
  int *f = nullptr;
  if (cudaMalloc(&f, (kMaxFlagBlocks + 1) * sizeof(int)) != cudaSuccess) return nullptr;
  if (cudaMemset(f, 0, (kMaxFlagBlocks + 1) * sizeof(int)) != cudaSuccess) return nullptr;
  fp.pool[fp.used] = {dev, st, f};
  return fp.pool[fp.used++].flags;
}

static int *solve_flags_for(cudaStream_t st) { return solve_flags_lookup(st, true); }

// Whether a flag wait of a solve on `st` gave up since the last call: waits
// for the stream, reads the timeout word and clears it.
cudaError_t solve_timeout_read(cudaStream_t st, int *timed_out) {
  *timed_out = 0;
  int *flags = solve_flags_lookup(st, false);
  if (!flags) return cudaSuccess;  // no dependency-ordered solve ran on st
  cudaError_t e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return e;
  int word = 0;
  if ((e = cudaMemcpy(&word, flags + kMaxFlagBlocks, sizeof(int), cudaMemcpyDeviceToHost)) != cudaSuccess)
    return e;
  if (word != 0) {  // cleared in the stream's order, before its later solves
    if ((e = cudaMemsetAsync(flags + kMaxFlagBlocks, 0, sizeof(int), st)) != cudaSuccess) return e;
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return e;
  }
  *timed_out = word != 0;
  return cudaSuccess;
}

// one CTA per SM, one diagonal block per CTA
static int coop_max_n() {
  int sms = 1;
  if (device_sm_count(&sms) != cudaSuccess) sms = 1;
  return (sms < kMaxFlagBlocks ? sms : kMaxFlagBlocks) * kTb;
}

// 0: launched; 1: not available here (use the per-block path); <0 error
static int trsm_left_flags(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B, int ldb,
                           cudaStream_t st, cudaError_t *err) {
  static std::atomic<unsigned long long> init{0};
  const size_t smem = ((size_t)kTb * kLdI + kTb + 4 * (size_t)kTb * kCoopMaxRhs) * 8;
  cudaError_t e = once_per_device(init, [smem] {
    return cudaFuncSetAttribute(trsv_flag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) {
    *err = e;
    return -1;
  }
  int *flags = solve_flags_for(st);
  if (!flags) return 1;
  const int nblk = (n + kTb - 1) / kTb;
  e = cudaMemsetAsync(flags, 0, (size_t)nblk * sizeof(int), st);
  if (e != cudaSuccess) {
    *err = e;
    return -1;
  }
  int lo = lower ? 1 : 0, un = unit ? 1 : 0;
  void *args[] = {&n, &nrhs, (void *)&T, &ldt, &B, &ldb, &lo, &un, &flags};
  ProfScope ps(kClsSolve, st, (double)n * n * nrhs);
  e = cudaLaunchCooperativeKernel((void *)trsv_flag_kernel, dim3(nblk), dim3(256), args, smem, st);
  if (e != cudaSuccess) {
    *err = e;
    return -1;
  }
  return 0;
}

cudaError_t trsm_left(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B,
                      int ldb, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs <= kCoopMaxRhs && n > kTb && n <= coop_max_n()) {
    cudaError_t err = cudaSuccess;
    const int rc = trsm_left_flags(lower, unit, n, nrhs, T, ldt, B, ldb, st, &err);
    if (rc == 0) return cudaSuccess;
    if (rc < 0) return err;
  }
  const size_t smem = ((size_t)kTb * (kTb + 1) + (size_t)kTb * 33) * 8;
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [smem] {
    return cudaFuncSetAttribute(trsm_diag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
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
