// qp_noalloc.cu -- qp_forward_noalloc: the batched forward solve for callers that cannot
// allocate device memory.
//
// Who needs it: code that must not call cudaMalloc (or any allocating library routine) on
// its hot path.  Examples are a control loop with a hard latency budget, a process
// whose device memory is fixed by a budget set when it starts, and a plugin living inside a
// host framework that owns all allocation.  Those callers still pass their own inputs and
// outputs, but cannot provide the workspace that qp_forward needs.
//
// The workspace here is a file-scope device array of QP_NOALLOC_SCRATCH_BYTES bytes, created
// when the library's module is loaded on a device and held by every device that loads it
// until the process exits.  Its device address is looked up once per device, with that device
// current, the first time the entry point runs there; do that first call before any stream
// capture.  The address is then cached for the life of the process: a cudaDeviceReset (or any
// other teardown of the device's primary context) reloads the module at a new address and
// leaves the cached one dangling, so callers that reset a device must not call this entry
// point on it afterwards.  Every call shares the array and leaves its contents behind: the forward kernel
// writes everything it later reads, so nothing has to be cleared between calls, but calls
// that overlap on the GPU (different streams, or a second call before the first finished)
// race on it.
#include <cuda_runtime.h>

#include <mutex>

#include "qp_gb300.h"

namespace {

static __device__ __align__(256) unsigned char g_qp_scratch[QP_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
void* g_addr[kMaxDevices] = {nullptr};

// Device address of g_qp_scratch on the current device (nullptr on failure).
void* scratch_address() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(g_mu);
  if (!g_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_qp_scratch) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    g_addr[dev] = p;
  }
  return g_addr[dev];
}

}  // namespace

extern "C" int qp_forward_noalloc(const qp_options* opt, int dtype, int B, int n, int nineq,
                                  int neq, const void* Q, const void* q, const void* G,
                                  const void* h, const void* A, const void* b, void* z,
                                  void* lam, void* nu, int32_t* status, int32_t* iters,
                                  double* resid, void* stream) {
  const size_t need = qp_workspace_bytes_opt(opt, dtype, B, n, nineq, neq);
  if (B > 0 && need == 0) return QP_EINVAL;
  if (need > (size_t)QP_NOALLOC_SCRATCH_BYTES) return QP_ENOSPACE;
  void* ws = scratch_address();
  if (!ws) return QP_ECUDA;
  return qp_forward(opt, dtype, B, n, nineq, neq, Q, q, G, h, A, b, z, lam, nu, status, iters,
                    resid, ws, (size_t)QP_NOALLOC_SCRATCH_BYTES, stream);
}
