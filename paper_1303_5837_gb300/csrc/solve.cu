// solve.cu -- triangular solves and row interchanges that consume the
// factors (PA = LU: swaps, unit-lower forward and upper back substitution;
// A = QR: back substitution with R after Q^T is applied through the tree).
//
// Blocked by kTb rows: for few right-hand sides one cooperative launch with
// one CTA per diagonal block, ordered by ready flags; otherwise the diagonal
// block is solved by one CTA in shared memory and the rows below (or above)
// are updated with the FP64 GEMM, one launch per block.
#include <atomic>

#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {

constexpr int kTb = 128;

// Row interchanges of LAPACK laswp (forward), one CTA per right-hand side;
// the column is staged in shared memory when it fits.
__global__ void __launch_bounds__(32) swap_rows_kernel(int n, const int *ipiv, double *B, int ldb,
                                                       int staged, const int *skip) {
  extern __shared__ __align__(16) double col[];
  if (skip && *skip) return;
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

cudaError_t getrs_swap(int n, int nrhs, const int *ipiv, double *B, int ldb, cudaStream_t st, const int *skip) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  static std::atomic<unsigned long long> init{0};
  cudaError_t e = once_per_device(init, [] {
    return cudaFuncSetAttribute(swap_rows_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
  });
  if (e != cudaSuccess) return e;
  int staged = ((size_t)n * 8 <= 200 * 1024) ? 1 : 0;
  ProfScope ps(kClsSolve, st, 0.0);
  swap_rows_kernel<<<nrhs, 32, staged ? (size_t)n * 8 : 0, st>>>(n, ipiv, B, ldb, staged, skip);
  return cudaGetLastError();
}

// Solve the nb x nb diagonal block T11 X = B1 in place (nb <= kTb) for all
// right-hand sides, one CTA per tile of 32 right-hand sides.
__global__ void __launch_bounds__(256) trsm_diag_kernel(int nb, int nrhs, const double *T, int ldt,
                                                        double *B, int ldb, int lower, int unit,
                                                        const int *skip) {
  extern __shared__ __align__(16) double tsm[];
  if (skip && *skip) return;
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
//   waits require; every wait is bounded (wait_limit cycles of SM clock,
//   about 2 s by default), after which the CTA ORs status_bit into *status
//   and leaves.  The flags live in the caller's workspace (SolveWs) and are
//   cleared before every launch.  withhold_blk >= 0 is a test hook: that
//   block never publishes its flag, so every wait on it runs out.
// Needs one CTA per diagonal block: n <= SMs * kTb.
// ---------------------------------------------------------------------------
constexpr int kCoopMaxRhs = 16;
constexpr int kLdI = kTb + 1;
constexpr int kMaxFlagBlocks = 1024;            // flag words of a solve workspace (covers any SM count here)
constexpr long long kSolveWaitLimit = 4000000000ll;

// Test hook state (host): the wait limit and the withheld block of the next
// dependency-ordered solves (kSolveWaitLimit and -1 unless a test set them).
static std::atomic<long long> g_wait_limit{kSolveWaitLimit};
static std::atomic<int> g_withhold{-1};

__device__ __forceinline__ int ld_acquire_gpu(const int *p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_gpu(int *p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

struct FlagArgs {
  int *flags;            // nblk ready flags, zero at launch
  int *status;           // gets status_bit when a wait gives up
  int status_bit;
  const int *skip;       // refinement: nonzero = the loop has stopped, do nothing
  long long wait_limit;  // cycles
  int withhold_blk;      // test hook (-1: off)
};

__global__ void __launch_bounds__(256, 1) trsv_flag_kernel(int n, int nrhs, const double *T, int ldt, double *B,
                                                           int ldb, int lower, int unit, FlagArgs fa) {
  extern __shared__ __align__(16) double csm[];
  double *Ti = csm;                          // the inverted diagonal block, ld kLdI
  double *tmp = Ti + kTb * kLdI;             // kTb column buffer
  double *sb = tmp + kTb;                    // kTb x nrhs: my right-hand sides being reduced
  double *xj = sb + kTb * kCoopMaxRhs;       // kTb x nrhs: a published solution block
  double *part = xj + kTb * kCoopMaxRhs;     // 2 x kTb x nrhs: half-row partial sums
  __shared__ int abort_flag;
  if (fa.skip && *fa.skip) return;
  int *flags = fa.flags;
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
    // lower: columns right to left; X(j, j) = 1 / T(j, j) (1 when unit),
    // X(j+1:, j) = -X(j+1:, j+1:) T(j+1:, j) X(j, j)
    for (int i = tid; i < nb; i += blockDim.x) xj[i] = unit ? 1.0 : 1.0 / Ti[i + i * kLdI];
    __syncthreads();
    for (int j = nb - 1; j >= 0; --j) {
      const double djj = xj[j];
      for (int i = j + 1 + tid; i < nb; i += blockDim.x) {
        double acc = 0.0;
        for (int k = j + 1; k <= i; ++k) acc = fma(Ti[i + k * kLdI], Ti[k + j * kLdI], acc);
        tmp[i] = -acc * djj;
      }
      __syncthreads();
      for (int i = j + 1 + tid; i < nb; i += blockDim.x) Ti[i + j * kLdI] = tmp[i];
      if (tid == 0) Ti[j + j * kLdI] = djj;
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
        if (clock64() - tstart > fa.wait_limit) {
          ok = 0;
          atomicOr(fa.status, fa.status_bit);  // the timeout record
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
  if (tid == 0 && blk != fa.withhold_blk) st_release_gpu(flags + blk, 1);
}

// Solve workspace (caller memory): word 0 is the timeout record of the
// library's solves that use it, the ready flags start at word 32.
size_t solve_ws_bytes(int n) {
  const int nblk = (n + kTb - 1) / kTb;
  return align256((size_t)(32 + (nblk < 1 ? 1 : nblk)) * sizeof(int));
}

void solve_ws_carve(void *w, int n, SolveWs &s) {
  (void)n;
  s.status = (int *)w;
  s.flags = (int *)w + 32;
}

void solve_test_hook(long long wait_cycles, int withhold_blk) {
  g_wait_limit.store(wait_cycles > 0 ? wait_cycles : kSolveWaitLimit);
  g_withhold.store(withhold_blk);
}

// one CTA per SM, one diagonal block per CTA
static int coop_max_n() {
  int sms = 1;
  if (device_sm_count(&sms) != cudaSuccess) sms = 1;
  return (sms < kMaxFlagBlocks ? sms : kMaxFlagBlocks) * kTb;
}

static cudaError_t trsm_left_flags(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B,
                                   int ldb, const SolveWs &ws, int *status, int status_bit, const int *skip,
                                   cudaStream_t st) {
  static std::atomic<unsigned long long> init{0};
  const size_t smem = ((size_t)kTb * kLdI + kTb + 4 * (size_t)kTb * kCoopMaxRhs) * 8;
  cudaError_t e = once_per_device(init, [smem] {
    return cudaFuncSetAttribute(trsv_flag_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  });
  if (e != cudaSuccess) return e;
  const int nblk = (n + kTb - 1) / kTb;
  e = cudaMemsetAsync(ws.flags, 0, (size_t)nblk * sizeof(int), st);
  if (e != cudaSuccess) return e;
  FlagArgs fa;
  fa.flags = ws.flags;
  fa.status = status;
  fa.status_bit = status_bit;
  fa.skip = skip;
  fa.wait_limit = g_wait_limit.load();
  fa.withhold_blk = g_withhold.load();
  if (fa.withhold_blk >= 0) fa.withhold_blk = lower ? 0 : nblk - 1;  // the block nothing else precedes
  int lo = lower ? 1 : 0, un = unit ? 1 : 0;
  void *args[] = {&n, &nrhs, (void *)&T, &ldt, &B, &ldb, &lo, &un, &fa};
  ProfScope ps(kClsSolve, st, (double)n * n * nrhs);
  return cudaLaunchCooperativeKernel((void *)trsv_flag_kernel, dim3(nblk), dim3(256), args, smem, st);
}

cudaError_t trsm_left(bool lower, bool unit, int n, int nrhs, const double *T, int ldt, double *B, int ldb,
                      const SolveWs &ws, int *status, int status_bit, const int *skip, cudaStream_t st) {
  if (n <= 0 || nrhs <= 0) return cudaSuccess;
  if (nrhs <= kCoopMaxRhs && n > kTb && n <= coop_max_n())
    return trsm_left_flags(lower, unit, n, nrhs, T, ldt, B, ldb, ws, status, status_bit, skip, st);
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
                                             lower ? 1 : 0, unit ? 1 : 0, skip);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    if (lower) {
      const int rest = n - r0 - nb;
      e = gemm_minus_f64(rest, nrhs, nb, T + (r0 + nb) + (size_t)r0 * ldt, ldt, B + r0, ldb,
                         B + r0 + nb, ldb, st, skip);
    } else {
      e = gemm_minus_f64(r0, nrhs, nb, T + (size_t)r0 * ldt, ldt, B + r0, ldb, B, ldb, st, skip);
    }
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

}  // namespace cagb
