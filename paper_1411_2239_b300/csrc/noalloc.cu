// rv_verify_trace_noalloc: offline verification that allocates nothing.
//
// Some callers cannot allocate device memory when they verify: code that runs
// while a CUDA graph is being captured (cudaMalloc is not allowed there), a
// host that hands all free device memory to another allocator, or a
// monitoring loop that must never block or fail on an allocation.  This entry
// point runs the same kernels as rv_verify_trace_async, but its workspace is a
// fixed array compiled into the library instead of caller or library
// allocations.
#include <mutex>

#include "rv_internal.h"

// Fixed workspace of the no-allocation entry point.  Every GPU that loads
// librv holds these bytes until the process exits.
#define RV_NOALLOC_SCRATCH_BYTES (64ull << 20)
#define RV_NOALLOC_MAX_EVENTS 1000000ull

static __device__ __align__(256) unsigned char g_noalloc_scratch[RV_NOALLOC_SCRATCH_BYTES];

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_setup_mu;
void* g_scratch_ptr[kMaxDevices];   // device address of g_noalloc_scratch, per device
}  // namespace

extern "C" rv_status rv_verify_trace_noalloc(const rv_formula* f, const rv_trace* t, rv_result* dev_out,
                                             cudaStream_t s) {
  if (!f || !t || !dev_out) return rv_fail(RV_EINVAL, "null argument");
  if (t->n > RV_NOALLOC_MAX_EVENTS)
    return rv_fail(RV_EINVAL, "trace of %llu events is longer than the %llu events the no-allocation entry point "
                              "supports; use rv_verify_trace with a workspace",
                   (unsigned long long)t->n, RV_NOALLOC_MAX_EVENTS);
  const size_t need = rv_verify_workspace_size(f, t->n, 0, nullptr);
  if (need > RV_NOALLOC_SCRATCH_BYTES)
    return rv_fail(RV_EINVAL, "trace needs %zu bytes of scratch, the no-allocation entry point has %llu",
                   need, RV_NOALLOC_SCRATCH_BYTES);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return rv_fail(RV_ECUDA, "cudaGetDevice: %s", cudaGetErrorString(e));
  if (dev < 0 || dev >= kMaxDevices) return rv_fail(RV_EINVAL, "device %d out of range", dev);
  void* scratch = nullptr;
  {
    // set-up, once per device and with that device current: in host code the
    // array's name is only a stand-in, so look up its device address
    std::lock_guard<std::mutex> lk(g_setup_mu);
    if (!g_scratch_ptr[dev]) {
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
      if (e != cudaSuccess) return rv_fail(RV_ECUDA, "cudaGetSymbolAddress: %s", cudaGetErrorString(e));
      g_scratch_ptr[dev] = p;
    }
    scratch = g_scratch_ptr[dev];
  }
  return rv_verify_trace_async(f, t, scratch, RV_NOALLOC_SCRATCH_BYTES, dev_out, nullptr, nullptr, s);
}
