// Host emulation of the tensor-core, bulk-copy and mbarrier wrappers of qp_tc.cuh, for the
// CPU check of the kernel source.  Blocks run one at a time, so one tensor-memory array
// serves every block.  MMAs complete when issued; an mbarrier word holds the number of
// completed phases.
// The operand layouts are read exactly as the descriptors describe them (start address,
// leading- and stride-dimension byte offsets of the canonical K-major layout), so a layout
// or descriptor that disagrees with the panels' writer gives wrong results here, and any
// access outside shared memory or the workspace is an AddressSanitizer error.
#pragma once
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <atomic>
#include <thread>

namespace qpk {

struct EmuTmem {
  float v[128][512];
  int cols = 0;
};
inline EmuTmem& emu_tmem() {
  static EmuTmem* t = new EmuTmem();
  return *t;
}
[[noreturn]] inline void emu_tc_fail(const char* what) {
  fprintf(stderr, "tensor-core emulation: %s\n", what);
  abort();
}
inline void emu_bar_complete(uint64_t* bar) { __atomic_fetch_add(bar, 1ull, __ATOMIC_SEQ_CST); }

inline void tc_mbar_init(uint64_t* bar) {
  if ((uintptr_t)bar % 8) emu_tc_fail("mbarrier not 8-byte aligned");
  __atomic_store_n(bar, 0ull, __ATOMIC_SEQ_CST);
}
inline void tc_mbar_inval(uint64_t*) {}
inline bool tc_try_wait(uint64_t* bar, uint32_t parity) {
  const bool done = ((uint32_t)__atomic_load_n(bar, __ATOMIC_SEQ_CST) & 1u) != parity;
  if (!done) std::this_thread::yield();   // let the issuing thread run
  return done;
}
// alloc and dealloc are warp-collective: lane 0 of the calling warp acts for it
inline void tc_alloc256(uint32_t* slot) {
  const uint32_t ncols = 256;
  if (threadIdx.x & 31) return;
  EmuTmem& t = emu_tmem();
  if (ncols < 32 || ncols > 512 || (ncols & (ncols - 1))) emu_tc_fail("bad column count");
  if (t.cols) emu_tc_fail("tensor memory allocated twice");
  t.cols = (int)ncols;
  for (auto& row : t.v)
    for (float& x : row) x = std::nanf("");
  *slot = 0;
}
inline void tc_dealloc256(uint32_t tmem) {
  const uint32_t ncols = 256;
  if (threadIdx.x & 31) return;
  EmuTmem& t = emu_tmem();
  if (tmem != 0 || (int)ncols != t.cols) emu_tc_fail("dealloc does not match alloc");
  t.cols = 0;
}
inline float emu_tf32(float x) {
  uint32_t u;
  std::memcpy(&u, &x, 4);
  u &= 0xFFFFE000u;
  std::memcpy(&x, &u, 4);
  return x;
}
inline void tc_mma_tf32(uint32_t tmem, const void* a, const void* b, uint32_t lbo, uint32_t sbo,
                        uint32_t idesc, bool accumulate) {
  EmuTmem& t = emu_tmem();
  const int M = (int)((idesc >> 24) & 0x1F) << 4, N = (int)((idesc >> 17) & 0x3F) << 3;
  if (((idesc >> 4) & 3) != 1 || ((idesc >> 7) & 7) != 2 || ((idesc >> 10) & 7) != 2 ||
      ((idesc >> 15) & 3) != 0 || M != 128 || N < 8 || N > 256)
    emu_tc_fail("unexpected instruction descriptor");
  const int lane0 = (int)(tmem >> 16), col0 = (int)(tmem & 0xFFFF);
  if (lane0 != 0 || col0 + N > t.cols) emu_tc_fail("accumulator outside the allocation");
  if ((uintptr_t)a % 16 || (uintptr_t)b % 16) emu_tc_fail("operand not 16-byte aligned");
  // gather the operands as the descriptors lay them out, then multiply
  static thread_local float A[128][8], Bm[256][8];
  auto at = [&](const void* base, int r, int k) {
    float x;
    std::memcpy(&x, (const unsigned char*)base + (r >> 3) * sbo + (k >> 2) * lbo + (r & 7) * 16 +
                        (k & 3) * 4, 4);
    return emu_tf32(x);
  };
  for (int i = 0; i < M; ++i)
    for (int k = 0; k < 8; ++k) A[i][k] = at(a, i, k);
  for (int j = 0; j < N; ++j)
    for (int k = 0; k < 8; ++k) Bm[j][k] = at(b, j, k);
  for (int i = 0; i < M; ++i)
    for (int j = 0; j < N; ++j) {
      float s = accumulate ? t.v[i][col0 + j] : 0.f;
      for (int k = 0; k < 8; ++k) s += A[i][k] * Bm[j][k];
      t.v[i][col0 + j] = s;
    }
}
inline void tc_commit(uint64_t* bar) { emu_bar_complete(bar); }
inline void tc_ld32(uint32_t taddr, float (&v)[32]) {
  EmuTmem& t = emu_tmem();
  const int lane0 = (int)(taddr >> 16), col = (int)(taddr & 0xFFFF);
  const int warp = (int)(threadIdx.x >> 5), lane = (int)(threadIdx.x & 31);
  if (lane0 != 32 * (warp & 3)) emu_tc_fail("warp reads a lane quarter that is not its own");
  if (col + 32 > t.cols) emu_tc_fail("read outside the allocation");
  for (int j = 0; j < 32; ++j) v[j] = t.v[lane0 + lane][col + j];
}
inline void tc_fence_before() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void tc_fence_after() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
inline void tc_proxy_fence() { __atomic_thread_fence(__ATOMIC_SEQ_CST); }
// A virtual clock for the bounded waits: 1 µs per reading, so a wait gives up after about
// 32 million polls whatever the host's load (a barrier that never completes still ends the
// wait, as on the GPU).
inline unsigned long long tc_now() {
  static std::atomic<unsigned long long> t{0};
  return t.fetch_add(1000, std::memory_order_relaxed);
}

}  // namespace qpk
