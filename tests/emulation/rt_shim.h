// Host stand-ins for the CUDA runtime calls the library's host code makes, and the launch of
// a kernel as blocks of host threads (one block after another).
#pragma once
#include "shim.h"
typedef int cudaError_t;
enum : int { cudaSuccess = 0, cudaErrorInvalidValue = 1, cudaErrorMemoryAllocation = 2 };
typedef void* cudaStream_t;
typedef void* cudaEvent_t;
enum cudaDeviceAttr { cudaDevAttrMultiProcessorCount = 16, cudaDevAttrMaxSharedMemoryPerBlockOptin = 97 };
enum cudaFuncAttribute { cudaFuncAttributeMaxDynamicSharedMemorySize = 8 };
#define cudaStreamNonBlocking 1u
#define cudaEventDisableTiming 2u
inline cudaError_t cudaGetDevice(int* d) { *d = 0; return cudaSuccess; }
inline cudaError_t cudaDeviceGetAttribute(int* v, cudaDeviceAttr a, int) {
  *v = a == cudaDevAttrMultiProcessorCount ? 152 : 232448;   // GB300
  return cudaSuccess;
}
inline cudaError_t cudaFuncSetAttribute(const void*, cudaFuncAttribute, int) { return cudaSuccess; }
inline cudaError_t cudaGetLastError() { return cudaSuccess; }
inline cudaError_t cudaMemsetAsync(void* p, int v, size_t n, cudaStream_t = nullptr) {
  std::memset(p, v, n);
  return cudaSuccess;
}
inline cudaError_t cudaEventRecord(cudaEvent_t, cudaStream_t = nullptr) { return cudaSuccess; }
inline cudaError_t cudaStreamWaitEvent(cudaStream_t, cudaEvent_t, unsigned = 0) { return cudaSuccess; }
inline cudaError_t cudaStreamCreateWithFlags(cudaStream_t* s, unsigned) { *s = (void*)1; return cudaSuccess; }
inline cudaError_t cudaEventCreateWithFlags(cudaEvent_t* e, unsigned) { *e = (void*)1; return cudaSuccess; }

// Shared memory is filled with 0xff bytes (NaN in either float type), so a read before the
// kernel writes shows up in the results.
template <class P>
void emu_launch(void (*kernel)(const P), int grid, size_t smem, const P& params) {
  constexpr int kThreads = 512;
  for (int b = 0; b < grid; ++b) {
    EmuBlock blk;
    blk.block = std::make_unique<std::barrier<>>(kThreads);
    for (int w = 0; w < 32; ++w) blk.warp[w] = std::make_unique<std::barrier<>>(32);
    emu_blk = &blk;
    void* s = nullptr;
    if (posix_memalign(&s, 128, smem ? smem : 16) != 0) abort();
    std::memset(s, 0xff, smem ? smem : 16);
    emu_dyn_smem = (unsigned char*)s;
    std::vector<std::thread> th;
    for (int t = 0; t < kThreads; ++t)
      th.emplace_back([&, t, b] {
        threadIdx.x = t;
        blockIdx.x = b;
        kernel(params);
        emu_blk->warp[t >> 5]->arrive_and_drop();
        emu_blk->block->arrive_and_drop();
      });
    for (auto& x : th) x.join();
    free(s);
  }
}
