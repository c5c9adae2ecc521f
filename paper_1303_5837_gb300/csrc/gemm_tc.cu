// gemm_tc.cu -- C -= A B with FP64 operands on the tcgen05 tensor cores.
//
// The trailing updates of CALU / CAQR are the dense contractions of the
// method (Sec. 3: the Schur complement A22 -= L21 U12 and the compact-WY
// Q^T C).  On GB300 the FP64 pipe retires ~1.2 TFLOP/s while the bf16 tensor
// cores retire ~1.9 PFLOP/s, so the reduced-precision form of the update runs
// there:
//   * split: every row of A (every column of B) is scaled by a power of two,
//     2^-e with |x| < 2^e, and cut into S signed base-256 digits
//     t = sum_k d_k 2^(-8k), |d_1| <= 256, |d_k| <= 128 -- exact FP64 steps.
//     Digit k is stored in bf16 as d_k 2^(-8(k-1)), which bf16 holds exactly;
//   * tcgen05.mma (kind::f16, bf16 x bf16 -> FP32 in tensor memory) sums the
//     digit products d_k d'_l with k + l <= S + 1 for one 128 x 128 tile;
//     operand tiles arrive by TMA (cp.async.bulk.tensor, 128-byte swizzle);
//   * the epilogue reads the accumulator with tcgen05.ld and applies
//     C -= 2^(e_i + f_j - 16) acc in FP64.
// Fused mode: one FP32 accumulator with pre-scaled digits, accurate to about
// 2^-20 relative to max|row of A| max|column of B|; FP64 iterative refinement
// recovers the rest.  Exact mode: integer digits, one accumulator per digit
// diagonal; every diagonal sum is an integer below 2^24 (k <= 128), so the
// tensor cores' FP32 sums are exact and the only error is the dropped digits,
// 2^(-8 S) relative (7 digits: the FP64 level).
//   diagonal k + l = D, digits |d_1| <= 256, |d_k| <= 128, k = 128:
//   D = 2: 2^23, 3: 2^23, 4: 1.25 2^23, 5: 1.5 2^23, 6: 1.75 2^23, 7: 2^24,
//   D = 8: 2.25 2^23 per K block of 64 (so split by K block).
//
// Every wait on an mbarrier is bounded by a clock limit; on a timeout the CTA
// raises a status bit, waits (bounded) for its own copies and MMAs, frees its
// tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>

#include "ca_internal.cuh"
#include "device_once.cuh"

namespace cagb {

// --------------------------------------------------------------------------
// PTX wrappers
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

// Waits for the phase with parity `parity`; false after ~`limit` SM cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, long long limit) {
  const uint32_t addr = smem_u32(bar);
  const long long t0 = clock64();
  while (true) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(addr), "r"(parity)
        : "memory");
    if (done) return true;
    if (clock64() - t0 > limit) return false;
  }
}

__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x,
                                            int y) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], "
      "[%2];" ::"r"(smem_u32(dst)),
      "l"((uint64_t)map), "r"(smem_u32(bar)), "r"(x), "r"(y)
      : "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                       uint32_t accumulate) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// 32 TMEM lanes x 32 consecutive 32-bit columns; thread i of the warp gets
// lane (lane base + i).
__device__ __forceinline__ void tmem_ld_32x32(uint32_t taddr, uint32_t (&r)[32]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
      "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// 32 TMEM lanes x 8 consecutive 32-bit columns.
__device__ __forceinline__ void tmem_ld_32x8(uint32_t taddr, uint32_t (&r)[8]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 "
      "{%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

// Shared-memory matrix descriptor of a K-major operand written by TMA with a
// 128-byte swizzle (rows of 128 bytes, groups of 8 rows = 1024 bytes, layout
// type 2) or a 64-byte swizzle (rows of 64 bytes, groups of 8 = 512 bytes,
// layout type 4); sm_100 descriptor version.
__device__ __forceinline__ uint64_t sw_desc(uint32_t saddr, int swz) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)1 << 16;                              // leading byte offset (unused, swizzled K-major)
  d |= (uint64_t)((swz == 2 ? 1024 : 512) >> 4) << 32;  // stride byte offset
  d |= (uint64_t)1 << 46;                              // version
  d |= (uint64_t)swz << 61;                            // layout type
  return d;
}

// Instruction descriptor, kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// 2^k as a double for -1022 <= k <= 1023 (IEEE binary64 exponent field).
__device__ __forceinline__ double pow2i(int k) {
  k = k < -1022 ? -1022 : (k > 1023 ? 1023 : k);
  return __longlong_as_double((long long)(k + 1023) << 52);
}

// v * 2^e2 as a double, from the integer bits (round to nearest even) -- no
// FP64-pipe instruction; exact when |v| < 2^53.  The results here stay far
// inside the normal range.
__device__ __forceinline__ double i64_scaled_to_double(long long v, int e2) {
  if (v == 0) return 0.0;
  const unsigned long long sign = v < 0 ? (1ull << 63) : 0ull;
  unsigned long long u = v < 0 ? (unsigned long long)(-v) : (unsigned long long)v;
  const int nbits = 64 - __clzll((long long)u);  // significant bits
  int sh = nbits - 53;
  unsigned long long m;
  if (sh <= 0) {
    m = u << (-sh);
  } else {
    m = u >> sh;
    const unsigned long long rem = u & ((1ull << sh) - 1), half = 1ull << (sh - 1);
    if (rem > half || (rem == half && (m & 1ull))) ++m;
    if (m >> 53) {
      m >>= 1;
      ++sh;
    }
  }
  const long long E = 52 + sh + e2 + 1023;  // m in [2^52, 2^53)
  if (E >= 2047) return __longlong_as_double((long long)(sign | (0x7ffull << 52)));  // overflow: infinity
  if (E <= 0) {
    // subnormal or zero: m 2^(E - 1075) = (m >> (1 - E)) 2^-1074, rounded to
    // nearest even (a carry into bit 52 gives the smallest normal number)
    const int s2 = 1 - (int)E;
    if (s2 > 53) return __longlong_as_double((long long)sign);
    unsigned long long q = m >> s2;
    const unsigned long long rem = m & ((1ull << s2) - 1), half = 1ull << (s2 - 1);
    if (rem > half || (rem == half && (q & 1ull))) ++q;
    return __longlong_as_double((long long)(sign | q));
  }
  return __longlong_as_double((long long)(sign | ((unsigned long long)E << 52) | (m & ((1ull << 52) - 1))));
}

// v * 2^e2 as a double, rounded to nearest even: CUDA's correctly rounded
// conversion of v, then the scale added to its exponent field (exact while
// the result stays normal); zero and results outside the normal range take
// the integer path above.
__device__ __forceinline__ double scaled_rn(long long v, int e2) {
  const long long bits = __double_as_longlong(__ll2double_rn(v));
  const int E = (int)((bits >> 52) & 0x7ff) + e2;
  if (v != 0 && E > 0 && E < 2047) return __longlong_as_double(bits + ((long long)e2 << 52));
  return i64_scaled_to_double(v, e2);
}

// Digits of x for the split: F = round(|x| 2^(8S - e)) (|x| < 2^e), as a
// signed integer with at most 8 S + 1 bits, from the FP64 bit pattern.
__device__ __forceinline__ long long fixed_point_digits(double x, int e, int S) {
  const unsigned long long bits = (unsigned long long)__double_as_longlong(x);
  const int E = (int)((bits >> 52) & 0x7ff);
  if (E == 0) return 0;  // zero or subnormal: below every digit
  const unsigned long long mant = (bits & ((1ull << 52) - 1)) | (1ull << 52);
  // |x| = mant 2^(E - 1075); F = mant 2^(E - 1075 + 8 S - e)
  const int sh = E - 1075 + 8 * S - e;
  unsigned long long F;
  if (sh >= 0) {
    F = mant << sh;  // |x| < 2^e keeps F < 2^(8S) <= 2^56
  } else if (sh > -64) {
    F = mant >> (-sh);
    const unsigned long long rem = mant & ((1ull << (-sh)) - 1), half = 1ull << (-sh - 1);
    if (rem > half || (rem == half && (F & 1ull))) ++F;
  } else {
    F = 0;
  }
  return (bits >> 63) ? -(long long)F : (long long)F;
}

constexpr int kTcBM = 128;
constexpr int kTcKpad = 64;                      // K is padded to a multiple of 64
constexpr long long kWaitLimit = 4000000000ll;   // ~2 s of SM clock
constexpr size_t kTcSmemBudget = 224 * 1024;
constexpr size_t kTcSmemHalf = 110 * 1024;  // per CTA when two share an SM

struct TcArgs {
  int kblocks, S, mpad, npad, bn;
  int bk, swz;   // K block (32 or 64 bf16) and its swizzle layout (4: 64 B, 2: 128 B)
  int exact;     // 1: one accumulator per digit diagonal (exact FP32 sums)
  int nstages;   // operand stages in shared memory (1 or 2)
  int tmem_cols;
  int nacc;      // TMEM accumulators (1, S, or 8 when the last of 7 diagonals is split)
  int nbatch;    // batch items (grid z)
  // valid rows / columns of item b: m_item[b] (or m, and m_last for the last item)
  int m, m_last, n, n_last;
  const int *m_item, *n_item;
  const int *ea, *eb;  // exponents, [item][mpad] and [item][npad]
  double *C;           // item b: C + b * sbc + coff[b], ld ldc
  int ldc;
  long long sbc;
  const int *coff;
  int sign;            // C -= sign * A B, sign = +1 or -1
  int *status;
  const int *skip;     // nonzero: a stage enqueued ahead that is not needed, do nothing
};

// Operand tiles for one K block: S boxes of A digits (128 x bk) then S boxes
// of B digits (bn x bk).
__host__ __device__ inline size_t tc_stage_bytes(int S, int bn, int bk) {
  return (size_t)S * (kTcBM + bn) * bk * 2;
}

__global__ void __launch_bounds__(256, 2)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap mapA, const __grid_constant__ CUtensorMap mapB,
                   TcArgs a) {
  extern __shared__ uint8_t smem_raw[];
  if (a.skip && *a.skip) return;  // before any barrier, copy or tensor-memory allocation
  uint8_t *base = (uint8_t *)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  const size_t stage_bytes = tc_stage_bytes(a.S, a.bn, a.bk);
  const int boxA = kTcBM * a.bk * 2;
  const int boxB = a.bn * a.bk * 2;
  uint64_t *full = (uint64_t *)(base + (size_t)a.nstages * stage_bytes);  // [2]
  uint64_t *empty = full + 2;                                            // [2]
  uint64_t *done = empty + 2;                                            // [1]
  uint32_t *tslot = (uint32_t *)(done + 1);
  volatile int *abort_flag = (volatile int *)(tslot + 1);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.x * kTcBM, n0 = blockIdx.y * a.bn;
  const int item = blockIdx.z;
  const bool last = item == a.nbatch - 1;
  const int mv = a.m_item ? a.m_item[item] : (last ? a.m_last : a.m);
  const int nvv = a.n_item ? a.n_item[item] : (last ? a.n_last : a.n);
  if (m0 >= mv || n0 >= nvv) return;  // an empty tile of a short batch item (uniform per CTA)

  if (threadIdx.x == 0) {
    for (int i = 0; i < 2; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(done, 1);
    *abort_flag = 0;
    fence_mbar_init();
  }
  if (warp == 0) {
    tmem_alloc(tslot, (uint32_t)a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  int issued0 = 0, issued1 = 0;  // loads issued into stage 0 / 1

  if (threadIdx.x == 0) {
    // ---- producer: TMA loads of the digit tiles, one K block per stage ----
    for (int kb = 0; kb < a.kblocks; ++kb) {
      const int st = kb % a.nstages, round = kb / a.nstages;
      if (round > 0 && !mbar_wait(&empty[st], (round - 1) & 1, kWaitLimit)) {
        *abort_flag = 1;
        atomicOr(a.status, 2);
        break;
      }
      if (*abort_flag) break;
      uint8_t *sa = base + (size_t)st * stage_bytes;
      uint8_t *sb = sa + (size_t)a.S * boxA;
      mbar_expect_tx(&full[st], (uint32_t)stage_bytes);
      for (int s = 0; s < a.S; ++s) {
        tma_load_2d(sa + (size_t)s * boxA, &mapA, &full[st], kb * a.bk, (item * a.S + s) * a.mpad + m0);
        tma_load_2d(sb + (size_t)s * boxB, &mapB, &full[st], kb * a.bk, (item * a.S + s) * a.npad + n0);
      }
      if (st == 0)
        ++issued0;
      else
        ++issued1;
    }
  } else if (threadIdx.x == 32) {
    // ---- MMA issuer: digit products d_k d'_l with k + l <= S + 1 ----------
    const uint32_t idesc = idesc_bf16_f32(kTcBM, a.bn);
    uint32_t started = 0;  // bit acc: accumulator acc already holds a product
    for (int kb = 0; kb < a.kblocks; ++kb) {
      const int st = kb % a.nstages;
      if (!mbar_wait(&full[st], (kb / a.nstages) & 1, kWaitLimit)) {
        *abort_flag = 1;
        atomicOr(a.status, 4);
        break;
      }
      tc_fence_after();
      uint8_t *sa = base + (size_t)st * stage_bytes;
      uint8_t *sb = sa + (size_t)a.S * boxA;
      const int khalf = (kb * a.bk >= 64) ? 1 : 0;  // which 64-wide half of K
      for (int ka = 0; ka < a.S; ++ka)
        for (int kq = 0; ka + kq < a.S; ++kq) {
          // accumulator: the digit diagonal ka + kq; with 7 digits the last
          // diagonal (7 products) is split by K block to stay below 2^24
          int acc = a.exact ? ka + kq : 0;
          if (a.nacc == 8 && acc == 6) acc = 6 + khalf;
          const uint32_t d = tmem + (uint32_t)(acc * a.bn);
          const uint64_t ad = sw_desc(smem_u32(sa + (size_t)ka * boxA), a.swz);
          const uint64_t bd = sw_desc(smem_u32(sb + (size_t)kq * boxB), a.swz);
          for (int ks = 0; ks < a.bk / 16; ++ks) {  // +32 bytes of K per step
            tc_mma(d, ad + 2 * ks, bd + 2 * ks, idesc, (started >> acc) & 1u);
            started |= 1u << acc;
          }
        }
      tc_commit(&empty[st]);  // the stage may be refilled once these MMAs are done
    }
    tc_commit(done);
  }
  __syncthreads();
  // ---- epilogue: C -= 2^(e_i + f_j - 16) sum_d 2^(-8 d) acc_d -------------
  bool ok = mbar_wait(done, 0, kWaitLimit) && (*abort_flag == 0);
  if (!ok && lane == 0) atomicOr(a.status, 8);
  tc_fence_after();
  const int nacc = a.nacc;
  if (ok) {
    // 8 warps: warp w reads TMEM lanes 32 (w % 4) .. + 31, column chunks
    // alternate between warps w and w + 4
    const int quad = warp & 3, half = warp >> 2;
    const int row = m0 + 32 * quad + lane;
    const bool rin = row < mv;
    const int er = rin ? a.ea[(size_t)item * a.mpad + row] : 0;
    const int *ebi = a.eb + (size_t)item * a.npad;
    double *Cb = a.C + (size_t)item * a.sbc + (a.coff ? a.coff[item] : 0);
    // exact mode: the digit diagonals D = 0 .. S-1 (weights 2^(-8 D)) are
    // integers below 2^24; combine them in integer arithmetic,
    //   T_hi = sum_{D <= 4} acc_D 2^(8 (4 - D)),  T_lo = sum_{D > 4} acc_D 2^(8 (6 - D)),
    // and turn each into a double by one correctly rounded conversion and an
    // exponent add (FP64 pipe: the conversion and the subtraction from C).
    const int dmax = a.exact ? a.S - 1 : 0;
    constexpr int kEp = 8;  // columns per epilogue step
    for (int c0 = half * kEp; c0 < a.bn; c0 += 2 * kEp) {
      long long thi[kEp], tlo[kEp];
#pragma unroll
      for (int j = 0; j < kEp; ++j) thi[j] = tlo[j] = 0;
      float vf[kEp];
      // unrolled over the at most 8 accumulators: constant shifts
#pragma unroll
      for (int d = 0; d < 8; ++d) {
        if (d >= nacc) break;
        uint32_t r[kEp];
        tmem_ld_32x8(tmem + ((uint32_t)(32 * quad) << 16) + (uint32_t)(d * a.bn + c0), r);
        if (!a.exact) {
#pragma unroll
          for (int j = 0; j < kEp; ++j) vf[j] = __uint_as_float(r[j]);
          continue;
        }
        const int D = d < 7 ? d : 6;  // accumulator 7 is the second half of diagonal 6
#pragma unroll
        for (int j = 0; j < kEp; ++j) {
          const long long q = (long long)__float2int_rn(__uint_as_float(r[j]));
          if (D <= 4)
            thi[j] += q << (8 * (4 - D));
          else
            tlo[j] += q << (8 * (6 - D));
        }
      }
      if (!rin) continue;
      // all loads of C in flight before any store
      double cv[kEp];
      int ec[kEp];
#pragma unroll
      for (int j = 0; j < kEp; ++j) {
        const int col = n0 + c0 + j;
        const bool ok_c = col < nvv;
        cv[j] = ok_c ? __ldcg(Cb + row + (size_t)col * a.ldc) : 0.0;
        ec[j] = ok_c ? __ldg(ebi + col) : 0;
      }
#pragma unroll
      for (int j = 0; j < kEp; ++j) {
        const int col = n0 + c0 + j;
        if (col >= nvv) continue;
        const int sc = er + ec[j] - 16;  // C -= sign 2^sc value
        double c = cv[j];
        if (a.exact) {
          // value = T_hi 2^(8 (4 - dmax)) ... written relative to diagonal dmax:
          // sum_D acc_D 2^(-8 D) = T_hi 2^(-32) + T_lo 2^(-48)
          c -= scaled_rn(a.sign > 0 ? thi[j] : -thi[j], sc - 32);
          if (dmax > 4) c -= scaled_rn(a.sign > 0 ? tlo[j] : -tlo[j], sc - 48);
        } else {
          c = fma((double)(-a.sign * vf[j]), pow2i(sc), c);
        }
        Cb[row + (size_t)col * a.ldc] = c;
      }
    }
  }
  // every copy this CTA issued has landed before shared memory goes away
  if (threadIdx.x == 0) {
    if (issued0 > 0) mbar_wait(&full[0], (issued0 - 1) & 1, kWaitLimit);
    if (issued1 > 0) mbar_wait(&full[1], (issued1 - 1) & 1, kWaitLimit);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, (uint32_t)a.tmem_cols);
}

// --------------------------------------------------------------------------
// split: the vectors of an operand (rows of A, columns of B) -> S bf16 digit
// slices, one warp per vector, K <= 256.  Item b, vector v, position k reads
// element (v, k) of the source: X[b * sb + off[b] + v * sv + k * sk], through
// the structure rule on (r, q) = (row, column) of the source:
// shape 0 dense, 1 unit lower (r > q stored, r == q is one, r < q zero),
// 2 upper (r <= q stored); (r, q) = (v + roff, k) or, transposed, (k + roff, v).
// Output: out[((b * S + s) * vpad + v) * kpad + k], exponent ex[b * vpad + v].
// --------------------------------------------------------------------------
__global__ void __launch_bounds__(256) split_kernel(TcOperand o, int nbatch, int S, int vpad, int kpad, int exact,
                                                    __nv_bfloat16 *__restrict__ out, int *__restrict__ ex,
                                                    const int *skip) {
  if (skip && *skip) return;
  const int lane = threadIdx.x & 31;
  const int v = blockIdx.x * 8 + (threadIdx.x >> 5);
  const int b = blockIdx.y;
  if (v >= vpad) return;
  const bool last = b == nbatch - 1;
  const int nv = o.nv_item ? o.nv_item[b] : (last ? o.nv_last : o.nv);
  const int K = o.K_item ? o.K_item[b] : (last ? o.K_last : o.K);
  const double *X = o.X + (long long)b * o.sb + (o.off ? o.off[b] : 0);
  constexpr int kPer = 8;  // K <= 256
  double x[kPer];
  unsigned long long mx = 0;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = lane + 32 * t;
    double val = 0.0;
    if (v < nv && k < K) {
      const int r = (o.trans ? k : v) + o.roff, q = o.trans ? v : k;
      if (o.shape == 0 || (o.shape == 1 && r > q) || (o.shape == 2 && r <= q))
        val = X[(long long)v * o.sv + (long long)k * o.sk];
      else if (o.shape == 1 && r == q)
        val = 1.0;
    }
    x[t] = val;
    const unsigned long long bits = absbits(val);
    mx = bits > mx ? bits : mx;
  }
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    const unsigned long long ot = __shfl_xor_sync(0xffffffffu, mx, off);
    mx = ot > mx ? ot : mx;
  }
  // |x| < 2^e; e from the exponent field of the largest magnitude
  int e = 0;
  if (mx != 0) {
    const int E = (int)(mx >> 52);
    e = (E == 0) ? -1021 : E - 1022;
  }
  if (lane == 0) ex[(long long)b * vpad + v] = e;
#pragma unroll
  for (int t = 0; t < kPer; ++t) {
    const int k = lane + 32 * t;
    if (k >= kpad) continue;
    // F = round(x 2^(8S - e)) = sum_s d_s 256^(S-1-s), balanced digits
    // d_s in [-128, 127] for s >= 1 and |d_0| <= 256, all integer arithmetic
    long long F = fixed_point_digits(x[t], e, S);
    int dg[8];
#pragma unroll
    for (int s = 7; s >= 1; --s) {
      if (s >= S) continue;
      int d = (int)(F & 255);
      if (d >= 128) d -= 256;
      dg[s] = d;
      F = (F - d) >> 8;
    }
    dg[0] = (int)F;
#pragma unroll
    for (int s = 0; s < 8; ++s) {
      if (s >= S) break;
      // stored value: d_s (exact mode) or d_s 2^(-8 s) (fused mode), exact in bf16
      // 2^(-8 s) as a float from its exponent field (s <= 7: a normal number)
      const float w = exact ? 1.0f : __int_as_float((127 - 8 * s) << 23);
      const float val = (float)dg[s] * w;
      out[(((long long)b * S + s) * vpad + v) * kpad + k] = __float2bfloat16_rn(val);
    }
  }
}

// --------------------------------------------------------------------------
// host side
// --------------------------------------------------------------------------
static inline int rup(int x, int q) { return (x + q - 1) / q * q; }

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                   const cuuint64_t *, const cuuint32_t *, const cuuint32_t *,
                                   CUtensorMapInterleave, CUtensorMapSwizzle, CUtensorMapL2promotion,
                                   CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
  static EncodeTiledFn fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void *p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (EncodeTiledFn)p;
  }
  return fn;
}

static bool make_map(CUtensorMap *map, void *base, int kpad, int rows, int box_rows, int bk) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  cuuint64_t dims[2] = {(cuuint64_t)kpad, (cuuint64_t)rows};
  cuuint64_t strides[1] = {(cuuint64_t)kpad * 2};
  cuuint32_t box[2] = {(cuuint32_t)bk, (cuuint32_t)box_rows};
  cuuint32_t estr[2] = {1, 1};
  return fn(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, bk == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : CU_TENSOR_MAP_SWIZZLE_64B,
            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// Accumulators: one (fused), one per digit diagonal (exact), and with 7
// digits over K > 64 the 7-product diagonal gets one per 64-wide half of K.
static int tc_nacc(int S, int exact, int kpad) {
  return exact ? ((S == 7 && kpad > 64) ? 8 : S) : 1;
}

static int pow2_at_least(int x) {
  int p = 32;
  while (p < x) p *= 2;
  return p;
}

struct TcCfg {
  int bn, bk, swz, nstages, tmem_cols;
  size_t smem;
};

// Tile width, K block and stages.  First choice: two CTAs of 8 warps per
// SM (each with at most 256 tensor-memory columns and half the shared
// memory), so that one CTA's epilogue -- the FP64 read-modify-write of its C
// tile -- overlaps the other's loads and MMAs; tiles at least 64 wide.
// Otherwise one CTA per SM: the widest tile whose accumulators fit in the
// 512 columns.  Then the deepest K-block pipeline that fits in shared memory
// (two stages overlap the loads of one K block with the MMAs of the
// previous one).
static bool tc_config(int S, int exact, int kpad, TcCfg &c) {
  const int nacc = tc_nacc(S, exact, kpad);
  {
    int bn2 = 128;
    while (bn2 > 64 && nacc * bn2 > 256) bn2 /= 2;
    if (nacc * bn2 <= 256) {
      const int opts2[3][2] = {{64, 2}, {32, 2}, {32, 1}};
      for (auto &o : opts2) {
        const int bk = o[0];
        int ns = o[1];
        const int kblocks = kpad / bk;
        if (ns > kblocks) ns = kblocks;
        const size_t smem = ns * tc_stage_bytes(S, bn2, bk) + 1024 + 256;
        if (smem <= kTcSmemHalf) {
          c = {bn2, bk, bk == 64 ? 2 : 4, ns, pow2_at_least(nacc * bn2), smem};
          return true;
        }
      }
    }
  }
  int bn = 128;
  while (bn > 32 && nacc * bn > 512) bn /= 2;
  if (nacc * bn > 512) return false;
  const int opts[4][2] = {{64, 2}, {32, 2}, {64, 1}, {32, 1}};
  for (auto &o : opts) {
    const int bk = o[0];
    int ns = o[1];
    const int kblocks = kpad / bk;
    if (ns > kblocks) ns = kblocks;
    const size_t smem = ns * tc_stage_bytes(S, bn, bk) + 1024 + 256;
    if (smem <= kTcSmemBudget) {
      c = {bn, bk, bk == 64 ? 2 : 4, ns, pow2_at_least(nacc * bn), smem};
      return true;
    }
  }
  return false;
}

size_t tc_gemm_ws_bytes_batched(int m, int n, int k, int S, int nbatch) {
  const size_t mp = rup(m > 0 ? m : 1, kTcBM), np = rup(n > 0 ? n : 1, 128), kp = rup(k > 0 ? k : 1, kTcKpad);
  const size_t nb = nbatch > 0 ? nbatch : 1;
  return align256(nb * S * mp * kp * 2) + align256(nb * S * np * kp * 2) + align256(nb * mp * 4) +
         align256(nb * np * 4) + 256;
}

size_t tc_gemm_ws_bytes(int m, int n, int k, int S) { return tc_gemm_ws_bytes_batched(m, n, k, S, 1); }

bool tc_gemm_supported(int k, int S, int exact) {
  if (k < 1 || k > 256 || S < 1 || S > 8) return false;
  if (exact && (S > 7 || k > 128)) return false;
  TcCfg c;
  return tc_config(S, exact, rup(k, kTcKpad), c);
}

cudaError_t gemm_tc(const TcGemm &g, void *ws, int *status, cudaStream_t st) {
  const int m = g.A.nv, n = g.B.nv, k = g.A.K > g.A.K_last ? g.A.K : g.A.K_last;
  if (m <= 0 || n <= 0 || k <= 0 || g.nbatch <= 0) return cudaSuccess;
  if (!tc_gemm_supported(k, g.S, g.exact)) return cudaErrorInvalidValue;
  const int S = g.S, exact = g.exact;
  const int mp = rup(m, kTcBM), np = rup(n, 128), kp = rup(k, kTcKpad);
  TcCfg cfg;
  if (!tc_config(S, exact, kp, cfg)) return cudaErrorInvalidValue;
  const int bn = cfg.bn;
  const size_t nb = g.nbatch;
  char *p = (char *)(((uintptr_t)ws + 255) & ~(uintptr_t)255);
  __nv_bfloat16 *sa = (__nv_bfloat16 *)p;
  p += align256(nb * S * mp * kp * 2);
  __nv_bfloat16 *sb = (__nv_bfloat16 *)p;
  p += align256(nb * S * np * kp * 2);
  int *ea = (int *)p;
  p += align256(nb * mp * 4);
  int *eb = (int *)p;
  {
    ProfScope ps(kClsSplit, st, 0.0);
    split_kernel<<<dim3((mp + 7) / 8, g.nbatch), 256, 0, st>>>(g.A, g.nbatch, S, mp, kp, exact, sa, ea,
                                                                g.skip);
  }
  {
    ProfScope ps(kClsSplit, st, 0.0);
    split_kernel<<<dim3((np + 7) / 8, g.nbatch), 256, 0, st>>>(g.B, g.nbatch, S, np, kp, exact, sb, eb,
                                                                g.skip);
  }
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  CUtensorMap ma, mb;
  if (!make_map(&ma, sa, kp, (int)(nb * S * mp), kTcBM, cfg.bk) ||
      !make_map(&mb, sb, kp, (int)(nb * S * np), bn, cfg.bk))
    return cudaErrorInvalidValue;
  TcArgs a;
  a.kblocks = kp / cfg.bk;
  a.S = S;
  a.mpad = mp;
  a.npad = np;
  a.bn = bn;
  a.bk = cfg.bk;
  a.swz = cfg.swz;
  a.exact = exact;
  a.nstages = cfg.nstages;
  a.nacc = tc_nacc(S, exact, kp);
  a.tmem_cols = cfg.tmem_cols;
  a.nbatch = g.nbatch;
  a.m = g.A.nv;
  a.m_last = g.A.nv_last;
  a.n = g.B.nv;
  a.n_last = g.B.nv_last;
  a.m_item = g.A.nv_item;
  a.n_item = g.B.nv_item;
  a.ea = ea;
  a.eb = eb;
  a.C = g.C;
  a.ldc = g.ldc;
  a.sbc = g.sbc;
  a.coff = g.coff;
  a.sign = g.sign > 0 ? 1 : -1;
  a.status = status;
  a.skip = g.skip;
  const size_t smem = cfg.smem;
  static std::atomic<unsigned long long> init{0};
  e = once_per_device(init, [] {
    cudaError_t r = cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)kTcSmemBudget);
    if (r != cudaSuccess) return r;
    return cudaFuncSetAttribute(tc_gemm_kernel, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  });
  if (e != cudaSuccess) return e;
  dim3 grid(mp / kTcBM, np / bn, g.nbatch);
  // bf16 tensor-core flops issued: S (S + 1) / 2 digit products
  ProfScope ps(kClsGemmTc, st, 2.0 * (double)mp * np * kp * (S * (S + 1) / 2) * nb);
  tc_gemm_kernel<<<grid, 256, smem, st>>>(ma, mb, a);
  return cudaGetLastError();
}

cudaError_t gemm_minus_tc(int m, int n, int k, const double *A, int lda, const double *B, int ldb, double *C,
                          int ldc, int S, int exact, void *ws, int *status, cudaStream_t st, const int *skip) {
  TcGemm g = {};
  g.skip = skip;
  g.A.X = A;  // rows of A: element (i, k) at A[i + k lda]
  g.A.sv = 1;
  g.A.sk = lda;
  g.A.nv = g.A.nv_last = m;
  g.A.K = g.A.K_last = k;
  g.B.X = B;  // columns of B: element (j, k) at B[k + j ldb]
  g.B.sv = ldb;
  g.B.sk = 1;
  g.B.nv = g.B.nv_last = n;
  g.B.K = g.B.K_last = k;
  g.nbatch = 1;
  g.C = C;
  g.ldc = ldc;
  g.sign = 1.0;
  g.S = S;
  g.exact = exact;
  return gemm_tc(g, ws, status, st);
}

}  // namespace cagb
