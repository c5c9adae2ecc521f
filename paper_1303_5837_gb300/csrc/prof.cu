// prof.cu -- launch counting and per-kernel-class device timing.
//
// Every kernel launch of the library goes through a ProfScope: it counts the
// launch and, while profiling is enabled, records a CUDA event before and
// after it on the launching stream, together with the launch's algorithmic
// flop count.  Events come from a pool created by ca_prof_enable, never in
// the middle of a factorization.
#include <mutex>
#include <vector>

#include "ca_internal.cuh"

namespace cagb {

namespace {
struct Rec {
  int cls;
  double flops;
  cudaEvent_t a, b;
};
struct Prof {
  std::mutex mu;
  bool on = false;
  std::vector<cudaEvent_t> pool;
  size_t next = 0;
  std::vector<Rec> recs;
  long long dropped = 0;
  long long launches = 0;
  long long cls_launches[kNumClasses] = {};
};
Prof &prof() {
  static Prof p;
  return p;
}
const char *kNames[kNumClasses] = {"tslu_node", "laswp",      "lu_finish", "trsm_u12",
                                   "gemm_fp64", "tsqr_node",  "tree_apply", "solve",
                                   "split_bf16", "gemm_tc",    "refine",   "batched",
                                   "tree_narrow"};
}  // namespace

ProfScope::ProfScope(int cls, cudaStream_t st, double flops) : cls_(cls), st_(st), flops_(flops) {
  Prof &p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.launches++;
  p.cls_launches[cls]++;
  if (p.on && p.next + 2 <= p.pool.size()) {
    a_ = p.pool[p.next++];
    b_ = p.pool[p.next++];
    cudaEventRecord(a_, st_);
  } else if (p.on) {
    p.dropped++;
  }
}

ProfScope::~ProfScope() {
  if (!a_) return;
  cudaEventRecord(b_, st_);
  Prof &p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  p.recs.push_back(Rec{cls_, flops_, a_, b_});
}

// Peak probe: every thread runs `iters` rounds of 8 independent fused
// multiply-adds (a = a x + y), so the FMA pipe of the type, not latency or
// memory, bounds the kernel; the sums are stored so nothing is eliminated.
// x and y are held in registers (an operand read from the constant bank
// slows the FP64 pipe on this part: 1011 against 1201 GFLOP/s measured).
template <typename T>
__global__ void __launch_bounds__(256) fma_peak_kernel(int iters, T x0, T y0, T *out) {
  const T z = (T)(blockIdx.x >> 30) * (T)1e-30;  // zero, but not a compile-time constant
  const T x = x0 + z, y = y0 + z;
  T a[8];
#pragma unroll
  for (int i = 0; i < 8; ++i) a[i] = (T)(threadIdx.x + 1) * (T)1e-3 + (T)i;
  for (int it = 0; it < iters; ++it) {
#pragma unroll
    for (int i = 0; i < 8; ++i) a[i] = fma(a[i], x, y);
  }
  T s = 0;
#pragma unroll
  for (int i = 0; i < 8; ++i) s += a[i];
  out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

}  // namespace cagb

using namespace cagb;

extern "C" {

int ca_prof_enable(int on, int max_launches) {
  Prof &p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (on) {
    if (max_launches < 1) return -2;
    size_t want = 2 * (size_t)max_launches;
    while (p.pool.size() < want) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return CA_ERR_LAUNCH;
      p.pool.push_back(e);
    }
  }
  p.on = on != 0;
  p.next = 0;
  p.recs.clear();
  p.dropped = 0;
  return CA_OK;
}

int ca_prof_read(int cls, long long *launches, double *ms, double *flops) {
  if (cls < 0 || cls >= kNumClasses) return -1;
  Prof &p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  long long n = 0;
  double t = 0.0, f = 0.0;
  for (const Rec &r : p.recs) {
    if (r.cls != cls) continue;
    if (cudaEventSynchronize(r.b) != cudaSuccess) return CA_ERR_LAUNCH;
    float x = 0.f;
    if (cudaEventElapsedTime(&x, r.a, r.b) != cudaSuccess) return CA_ERR_LAUNCH;
    ++n;
    t += x;
    f += r.flops;
  }
  if (launches) *launches = n;
  if (ms) *ms = t;
  if (flops) *flops = f;
  return p.dropped ? 1 : CA_OK;
}

long long ca_launch_count(int cls) {
  Prof &p = prof();
  std::lock_guard<std::mutex> g(p.mu);
  if (cls < 0) return p.launches;
  if (cls >= kNumClasses) return -1;
  return p.cls_launches[cls];
}

int ca_peak_probe(int dtype, int blocks, int iters, void *dev_out, cudaStream_t stream) {
  if (dtype != CA_DTYPE_F64 && dtype != CA_DTYPE_F32) return -1;
  if (blocks < 1) return -2;
  if (iters < 1) return -3;
  if (!dev_out) return -4;
  if (dtype == CA_DTYPE_F64)
    fma_peak_kernel<double><<<blocks, 256, 0, stream>>>(iters, 0.999999, 1e-6, (double *)dev_out);
  else
    fma_peak_kernel<float><<<blocks, 256, 0, stream>>>(iters, 0.9999f, 1e-4f, (float *)dev_out);
  return cudaGetLastError() == cudaSuccess ? CA_OK : CA_ERR_LAUNCH;
}

const char *ca_kernel_class_name(int cls) {
  if (cls < 0 || cls >= kNumClasses) return "";
  return kNames[cls];
}

}  // extern "C"
