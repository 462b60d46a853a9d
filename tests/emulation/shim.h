// Host emulation of the CUDA device features the library's kernels use, for CPU checks of
// the kernel source: one thread block runs as NTHREADS std::threads, __syncthreads and
// __syncwarp are std::barrier waits, and warp shuffles go through a per-warp exchange
// buffer between two warp barriers (so a shuffle that not every lane of a warp reaches
// deadlocks here, as it may hang a GPU).  Shared memory is a heap buffer of the launch's
// exact size, so AddressSanitizer sees any access past it.
#pragma once
#include <algorithm>
#include <atomic>
#include <barrier>
#include <chrono>
#include <cmath>
#include <cstddef>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <memory>
#include <stdint.h>
#include <thread>
#include <vector>

#define __device__
#define __host__
#define __global__
#define __forceinline__ inline
#define __noinline__ __attribute__((noinline))
#define __launch_bounds__(a, b)
#define __restrict__ __restrict
#define __align__(n) alignas(n)

struct alignas(8) float2 { float x, y; };
struct alignas(16) float4 { float x, y, z, w; };
struct alignas(16) double2 { double x, y; };
inline float2 make_float2(float a, float b) { return {a, b}; }
inline float4 make_float4(float a, float b, float c, float d) { return {a, b, c, d}; }
inline double2 make_double2(double a, double b) { return {a, b}; }

struct EmuDim3 { unsigned x = 0, y = 0, z = 0; };
extern thread_local EmuDim3 threadIdx, blockIdx;
extern unsigned char* emu_dyn_smem;

struct EmuBlock {
  std::unique_ptr<std::barrier<>> block;
  std::unique_ptr<std::barrier<>> warp[32];
  alignas(16) unsigned char xbuf[32][32][8];
};
extern EmuBlock* emu_blk;

inline void __syncthreads() { emu_blk->block->arrive_and_wait(); }
inline void __syncwarp(unsigned = 0xffffffffu) { emu_blk->warp[threadIdx.x >> 5]->arrive_and_wait(); }

template <class T>
inline T emu_shfl(T v, int src) {
  static_assert(sizeof(T) <= 8, "shuffle width");
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  std::memcpy(emu_blk->xbuf[w][lane], &v, sizeof(T));
  emu_blk->warp[w]->arrive_and_wait();
  T r;
  std::memcpy(&r, emu_blk->xbuf[w][src & 31], sizeof(T));
  emu_blk->warp[w]->arrive_and_wait();
  return r;
}
template <class T> inline T __shfl_sync(unsigned, T v, int src) { return emu_shfl(v, src); }
template <class T> inline T __shfl_xor_sync(unsigned, T v, int m) {
  return emu_shfl(v, (int)(threadIdx.x & 31) ^ m);
}
template <class T> inline T __shfl_down_sync(unsigned, T v, unsigned d) {
  const int lane = threadIdx.x & 31;
  return emu_shfl(v, lane + (int)d < 32 ? lane + (int)d : lane);
}

template <class T> inline T __ldg(const T* p) { return *p; }
template <class V> inline void emu_stcs(V* p, V v) { *p = v; }
inline float __fadd_rn(float a, float b) { return a + b; }
inline float __fsub_rn(float a, float b) { return a - b; }
inline float __fmul_rn(float a, float b) { return a * b; }
inline float __double2float_rn(double x) { return (float)x; }
inline double __longlong_as_double(long long x) { double d; std::memcpy(&d, &x, 8); return d; }
inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }
inline float rsqrt(float x) { return 1.0f / std::sqrt(x); }
using std::fma; using std::fmax; using std::fmin; using std::fabs; using std::isfinite;
inline int max(int a, int b) { return a > b ? a : b; }
inline int min(int a, int b) { return a < b ? a : b; }
inline long long max(long long a, long long b) { return a > b ? a : b; }
inline long long min(long long a, long long b) { return a < b ? a : b; }
inline size_t max(size_t a, size_t b) { return a > b ? a : b; }
inline size_t min(size_t a, size_t b) { return a < b ? a : b; }
inline int atomicAdd(int* p, int v) { return __atomic_fetch_add(p, v, __ATOMIC_SEQ_CST); }
inline int atomicExch(int* p, int v) { return __atomic_exchange_n(p, v, __ATOMIC_SEQ_CST); }
inline size_t __cvta_generic_to_shared(const void* p) { return (size_t)p; }
inline unsigned long long emu_time_ns() {
  return (unsigned long long)std::chrono::duration_cast<std::chrono::nanoseconds>(
      std::chrono::steady_clock::now().time_since_epoch()).count();
}
