// noalloc.cu -- tslu_noalloc: the TSLU panel factorization with its scratch
// in a fixed device array compiled into the library, for callers that cannot
// allocate device memory.
//
// Who needs it: a caller whose device memory belongs to someone else (a
// plug-in inside a framework whose caching allocator owns the GPU, a serving
// process that reserved its whole HBM budget up front) or that cannot afford
// cudaMalloc on its path (cudaMalloc may synchronize the device and has no
// latency bound).  Such a caller can still pass its inputs and outputs but
// has no way to provide the tournament's scratch workspace.
//
// The scratch is one static __device__ array of CA_TSLU_NOALLOC_SCRATCH_BYTES
// per GPU that loads the library (held until the process exits).  Host code
// must not use the array's name as a device address: the first call on each
// device looks up the array's device address with cudaGetSymbolAddress while
// that device is current and keeps it for later calls.
#include <mutex>

#include "ca_internal.cuh"

namespace {

constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_tslu_scratch[CA_TSLU_NOALLOC_SCRATCH_BYTES];

std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

// Device address of g_tslu_scratch on the current device (set-up on first use).
int scratch_address(void **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return CA_ERR_LAUNCH;
  std::lock_guard<std::mutex> g(g_mu);
  if (!g_scratch_addr[dev]) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_tslu_scratch) != cudaSuccess || !p) return CA_ERR_LAUNCH;
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CA_OK;
}

}  // namespace

extern "C" int tslu_noalloc(int m, int n, double *A, int lda, const ca_tree_t *tree, int *ipiv,
                            int *dev_info, cudaStream_t stream) {
  if (m < 0) return -1;
  if (n < 0) return -2;
  size_t need = 0;
  int rc = ca_calu_workspace(m, n, n > 0 ? n : 1, tree, &need);
  if (rc == -4) return -5;  // the tree is argument 5 here
  if (rc != CA_OK) return rc;
  if (need > (size_t)CA_TSLU_NOALLOC_SCRATCH_BYTES) return CA_ERR_WORKSPACE;
  void *scratch = nullptr;
  rc = scratch_address(&scratch);
  if (rc != CA_OK) return rc;
  rc = tslu(m, n, A, lda, tree, ipiv, scratch, (size_t)CA_TSLU_NOALLOC_SCRATCH_BYTES, dev_info,
            stream);
  // tslu numbers work and lwork as arguments 7 and 8; this call has neither
  if (rc == -6) return -6;
  if (rc == -9) return -7;
  return rc;
}
