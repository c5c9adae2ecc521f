// gemm_fp64.cu -- C -= A B in FP64 on the DFMA pipe: the Schur-complement
// update A22 -= L21 U12 of CALU (Sec. 3.2; the dominant 2n^3/3 flops).
//
// On GB300 the FP64 pipe retires about two DFMA per SM per clock, so the
// kernel is bound by the FP64 pipe, not by memory: a register-tiled
// (8 x 8 or 4 x 4 per thread) block of C, A and B chunks staged in shared
// memory, one CTA of 256 threads per tile.
#include "ca_internal.cuh"

namespace cagb {

template <int BM, int BN, int BK>
__global__ void __launch_bounds__(256) gemm_minus_kernel(int m, int n, int k, const double *__restrict__ A,
                                                         int lda, const double *__restrict__ B, int ldb,
                                                         double *__restrict__ C, int ldc, const int *skip) {
  constexpr int TM = BM / 16, TN = BN / 16;
  __shared__ double As[BK][BM];
  __shared__ double Bs[BK][BN];
  if (skip && *skip) return;  // a refinement loop that has already stopped
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  const int i0 = blockIdx.x * BM, j0 = blockIdx.y * BN;
  double acc[TM][TN];
#pragma unroll
  for (int a = 0; a < TM; ++a)
#pragma unroll
    for (int b = 0; b < TN; ++b) acc[a][b] = 0.0;

  // software pipeline: the next K chunk of A and B is loaded into registers
  // while the current one is multiplied from shared memory
  constexpr int PA = BK * BM / 256, PB = BK * BN / 256;
  double ra[PA], rb[PB];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int idx = tid + 256 * t;
      const int i = idx % BM, kk = idx / BM;
      const int gi = i0 + i, gk = k0 + kk;
      ra[t] = (gi < m && gk < k) ? A[gi + (size_t)gk * lda] : 0.0;
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int idx = tid + 256 * t;
      const int kk = idx % BK, j = idx / BK;
      const int gj = j0 + j, gk = k0 + kk;
      rb[t] = (gj < n && gk < k) ? B[gk + (size_t)gj * ldb] : 0.0;
    }
  };
  load(0);
  for (int k0 = 0; k0 < k; k0 += BK) {
#pragma unroll
    for (int t = 0; t < PA; ++t) {
      const int idx = tid + 256 * t;
      As[idx / BM][idx % BM] = ra[t];
    }
#pragma unroll
    for (int t = 0; t < PB; ++t) {
      const int idx = tid + 256 * t;
      Bs[idx % BK][idx / BK] = rb[t];
    }
    __syncthreads();
    if (k0 + BK < k) load(k0 + BK);
#pragma unroll 4
    for (int kk = 0; kk < BK; ++kk) {
      double af[TM], bf[TN];
#pragma unroll
      for (int a = 0; a < TM; ++a) af[a] = As[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < TN; ++b) bf[b] = Bs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < TM; ++a)
#pragma unroll
        for (int b = 0; b < TN; ++b) acc[a][b] = fma(af[a], bf[b], acc[a][b]);
    }
    __syncthreads();
  }
  // per column: the TM loads of C in flight before the stores
#pragma unroll
  for (int b = 0; b < TN; ++b) {
    const int gj = j0 + ty + 16 * b;
    double cv[TM];
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int gi = i0 + tx + 16 * a;
      cv[a] = (gi < m && gj < n) ? C[gi + (size_t)gj * ldc] : 0.0;
    }
#pragma unroll
    for (int a = 0; a < TM; ++a) {
      const int gi = i0 + tx + 16 * a;
      if (gi < m && gj < n) C[gi + (size_t)gj * ldc] = cv[a] - acc[a][b];
    }
  }
}

cudaError_t gemm_minus_f64(int m, int n, int k, const double *A, int lda, const double *B, int ldb,
                           double *C, int ldc, cudaStream_t st, const int *skip) {
  if (m <= 0 || n <= 0 || k <= 0) return cudaSuccess;
  ProfScope ps(kClsGemm, st, 2.0 * m * (double)n * k);
  long long big = (long long)((m + 127) / 128) * ((n + 127) / 128);
  if (big >= 2 * 152) {
    dim3 grid((m + 127) / 128, (n + 127) / 128);
    gemm_minus_kernel<128, 128, 16><<<grid, 256, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, skip);
  } else {
    dim3 grid((m + 63) / 64, (n + 63) / 64);
    gemm_minus_kernel<64, 64, 16><<<grid, 256, 0, st>>>(m, n, k, A, lda, B, ldb, C, ldc, skip);
  }
  return cudaGetLastError();
}

}  // namespace cagb
