// qp_tc.cuh -- tensor-core (tcgen05) rank-64 updates of the global-memory setup sweep (FP32).
//
// The setup sweep (§3.1: S = [Q Aᵀ; A 0]⁻¹, RE and M = G P Gᵀ are computed once, before the
// iterations) is a symmetric Gauss-Jordan sweep over the first m1 pivots of the N × N KKT
// block matrix.  Taking the pivots 64 at a time, the sweep of one superblock K of 64 pivots
// changes every entry outside K's rows and columns by a rank-64 product,
//     a_ij −= Σ_{q∈K} p_iq c_jq,   p_iq = ĉ_iq / d_q, c_jq = ĉ_jq,
// where ĉ_iq is row i's entry in pivot column q just before pivot q is swept and d_q that
// pivot (the same sum the 16-pivot blocks of gsweep_setup apply on CUDA cores).  That
// product is the dense contraction of the setup, and here it runs on the tensor cores:
//
//  * phase A: the 64 × 64 pivot block is swept pivot after pivot, in registers (eight
//    entries per thread; each pivot's row and column go through shared memory), recording
//    each pivot's row of multipliers r_k (r_kk = 1/d_k, r_kq = a_kq/d_k);
//  * phase B (all threads, one row each): every row outside K replays the 64 scalar sweeps
//    on its 64 entries of K's columns (so the result equals the pivot-by-pivot sweep), and
//    writes p_iq and c_iq, split into TF32 high and low parts, to the panel tiles in the
//    workspace;
//  * phase C: for each 128 × 128 output tile, all threads stage the four 32 KB operand tiles
//    in shared memory (16-byte loads of the contiguous panel tiles, then a proxy fence), one
//    thread issues 8 K-steps × 3 tcgen05.mma (kind::tf32:
//    hi·hi + hi·lo + lo·hi, the 3×TF32 split that keeps FP32 accuracy) into one of two TMEM
//    accumulators, and, while the tensor core computes that tile, all 16 warps read the
//    previous tile's accumulator back (tcgen05.ld) and subtract it from the matrix in global
//    memory, skipping K's rows and columns and, in the λ-by-λ block, the strict lower
//    triangle.  The product is formed transposed (c tile as the MMA's A operand), so a TMEM
//    lane is an output column and each warp's accesses cover consecutive columns of a row.
//
// Panel tiles (workspace): four parts (p-hi, p-lo, c-hi, c-lo), each NT = T1 + T2 tiles of
// 128 rows × 64 columns (T1 = ⌈m1/128⌉ tiles for rows 0..m1−1, T2 = ⌈p/128⌉ for the λ rows
// m1..N−1), each tile 32 KB in the canonical K-major layout of the tensor core's shared-memory
// operands without swizzle: 8-row × 16-byte core matrices stored contiguously, K-adjacent
// core matrices 128 bytes apart, row groups 2048 bytes apart.  A tile moves to shared memory
// as one contiguous 32 KB block.
//
// The wait for MMA completion polls an mbarrier for at most TC_WAIT_NS of the GPU's global
// timer; on expiry the routine reports failure, waits (again bounded) for what it issued,
// frees its tensor memory and returns.
#pragma once

#include <stdint.h>
#include <string.h>

namespace qpk {

constexpr int TC_KB = 64;                       // pivots per superblock (the MMA's K)
constexpr int TC_TM = 128;                      // rows of an output tile (MMA M) and of a panel tile
constexpr int TC_TN = 128;                      // columns of an output tile (MMA N)
constexpr size_t TC_TILE_BYTES = (size_t)TC_TM * TC_KB * 4;   // 32 KB
// A hi/lo, B hi/lo at a 1024-byte boundary of the work region, then the mbarrier, the TMEM
// address and a flag
constexpr size_t TC_SMEM_BYTES = 4 * TC_TILE_BYTES + 128 + 1024;
constexpr int TC_MIN_M1 = 128;                  // at least two superblocks
constexpr unsigned long long TC_WAIT_NS = 500000000ull;   // 0.5 s per wait
// Dynamic shared memory the global-memory kernel may use with the tensor-core sweep: the
// opt-in limit per block of the target (227 KB) less 1 KB for static shared memory.
constexpr size_t TC_SMEM_CAP = 227 * 1024 - 1024;

// Byte offset of element (row r, column k) in a 128 × 64 operand tile (canonical K-major
// layout without swizzle, see above).
__host__ __device__ inline uint32_t tc_off(int r, int k) {
  return (uint32_t)((r >> 3) * 2048 + (k >> 2) * 128 + (r & 7) * 16 + (k & 3) * 4);
}

// Panel tiles of a size: T1 = ⌈m1/128⌉ + T2 = ⌈p/128⌉.
__host__ __device__ inline int tc_tiles(int m1, int p) {
  return (m1 + TC_TM - 1) / TC_TM + (p + TC_TM - 1) / TC_TM;
}
__host__ __device__ inline size_t tc_panel_bytes(int m1, int p) {
  return 4 * (size_t)tc_tiles(m1, p) * TC_TILE_BYTES;
}

// ---- the tensor-core and mbarrier operations used below, one wrapper each.  They
// are defined with inline PTX for the device; a host emulation of the kernel source (the CPU
// check under AddressSanitizer) supplies its own definitions instead.
__device__ void tc_mbar_init(uint64_t* bar);
__device__ void tc_mbar_inval(uint64_t* bar);
__device__ bool tc_try_wait(uint64_t* bar, uint32_t parity);
__device__ void tc_alloc256(uint32_t* slot);
__device__ void tc_dealloc256(uint32_t tmem);
__device__ void tc_mma_tf32(uint32_t tmem, const void* a, const void* b, uint32_t lbo,
                            uint32_t sbo, uint32_t idesc, bool accumulate);
__device__ void tc_commit(uint64_t* bar);
__device__ void tc_ld32(uint32_t taddr, float (&v)[32]);
__device__ void tc_fence_before();
__device__ void tc_fence_after();
__device__ void tc_proxy_fence();
__device__ unsigned long long tc_now();

// Instruction descriptor of kind::tf32: D FP32 (bits 4-5 = 1), A and B TF32 (bits 7-9 and
// 10-12 = 2), both K-major (bits 15, 16 = 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28.
__host__ __device__ constexpr uint32_t tc_idesc(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}

#if defined(__CUDA_ARCH__)
__device__ __forceinline__ uint32_t tc_smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// Shared-memory matrix descriptor: start address, leading-dimension byte offset (between
// K-adjacent core matrices), stride-dimension byte offset (between 8-row groups), descriptor
// version 1 (bits 46-47), base offset 0, no swizzle.
__device__ __forceinline__ uint64_t tc_sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr >> 4) & 0x3FFF) | ((uint64_t)((lbo >> 4) & 0x3FFF) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}
__device__ __forceinline__ void tc_mbar_init(uint64_t* bar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(tc_smem_u32(bar)) : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void tc_mbar_inval(uint64_t* bar) {
  asm volatile("mbarrier.inval.shared::cta.b64 [%0];" :: "r"(tc_smem_u32(bar)) : "memory");
}
__device__ __forceinline__ bool tc_try_wait(uint64_t* bar, uint32_t parity) {
  uint32_t ok;
  asm volatile("{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
               "selp.u32 %0, 1, 0, p;\n\t}" : "=r"(ok) : "r"(tc_smem_u32(bar)), "r"(parity) : "memory");
  return ok != 0;
}
// TMEM allocation of the 256 columns of two FP32 128 × 128 accumulators (warp-collective).
__device__ __forceinline__ void tc_alloc256(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 256;"
               :: "r"(tc_smem_u32(slot)) : "memory");
}
__device__ __forceinline__ void tc_dealloc256(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 256;" :: "r"(tmem) : "memory");
}
__device__ __forceinline__ void tc_mma_tf32(uint32_t tmem, const void* a, const void* b,
                                            uint32_t lbo, uint32_t sbo, uint32_t idesc,
                                            bool accumulate) {
  const uint64_t da = tc_sdesc(tc_smem_u32(a), lbo, sbo), db = tc_sdesc(tc_smem_u32(b), lbo, sbo);
  asm volatile("{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
               "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}"
               :: "r"(tmem), "l"(da), "l"(db), "r"(idesc), "r"((uint32_t)accumulate));
}
__device__ __forceinline__ void tc_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
               :: "r"(tc_smem_u32(bar)) : "memory");
}
// 32 consecutive FP32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tc_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int j = 0; j < 32; ++j) v[j] = __uint_as_float(r[j]);
}
__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
// Orders this thread's ordinary shared-memory stores before the tensor core's reads of them.
__device__ __forceinline__ void tc_proxy_fence() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ unsigned long long tc_now() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
#endif  // __CUDA_ARCH__

// Bounded wait for the completion of phase `parity`; false when TC_WAIT_NS ran out.
__device__ __forceinline__ bool tc_wait(uint64_t* bar, uint32_t parity) {
  if (tc_try_wait(bar, parity)) return true;
  const unsigned long long t0 = tc_now();
  for (;;) {
#pragma unroll 1
    for (int it = 0; it < 64; ++it)
      if (tc_try_wait(bar, parity)) return true;
    if (tc_now() - t0 > TC_WAIT_NS) return false;
  }
}
// TF32 high part (low 13 mantissa bits cleared, exact in TF32); x − tc_hi(x) is exact.
__device__ __forceinline__ float tc_hi(float x) {
  uint32_t u;
  memcpy(&u, &x, 4);
  u &= 0xFFFFE000u;
  float r;
  memcpy(&r, &u, 4);
  return r;
}

// Superblock sweeps of pivots [0, m1) in nsb = ⌈m1/64⌉ superblocks (the last one 16, 32, 48
// or 64 pivots) of the matrix gsweep_setup holds (SR: rows 0..N−1
// × columns 0..m1−1, row stride m1; the λ-by-λ block: strict upper triangle of Mb (row stride
// ldM) plus dM).  `tcp` is the panel-tile region of the workspace, `cb0` the shared work
// region (≥ TC_SMEM_BYTES, 16-byte aligned).  Pivot sign tests as in gsweep_setup.  Returns
// false on a pivot that fails its test or on an expired wait.
static __device__ __noinline__ bool tc_sweep_superblocks(int n, int nz, int p, int m, int nsb,
                                                         float* SR, float* Mb, int ldM, float* dM,
                                                         float* tcp, unsigned char* cb0,
                                                         float zthr) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m1 = nz + m, N = m1 + p, ldS = m1;
  const int T1 = (m1 + TC_TM - 1) / TC_TM, T2 = (p + TC_TM - 1) / TC_TM, NT = T1 + T2;
  unsigned char* part[4];
#pragma unroll
  for (int u = 0; u < 4; ++u)
    part[u] = reinterpret_cast<unsigned char*>(tcp) + (size_t)u * NT * TC_TILE_BYTES;
  // shared layout from the first 1024-byte boundary: phase C operand tiles p-hi, p-lo (sA),
  // c-hi, c-lo (sBt) at 0 / 32 / 64 / 96 KB, then the mbarrier, the TMEM address and a flag;
  // phases A/B reuse the operand space
  unsigned char* cb = cb0 + ((1024 - (reinterpret_cast<uintptr_t>(cb0) & 1023)) & 1023);
  unsigned char* sA[2] = {cb, cb + TC_TILE_BYTES};
  unsigned char* sBt[2] = {cb + 2 * TC_TILE_BYTES, cb + 3 * TC_TILE_BYTES};
  float* rowbuf = reinterpret_cast<float*>(cb);               // pivot row, two buffers
  float* colbuf = rowbuf + 2 * TC_KB;                          // pivot column, two buffers
  float* sR = reinterpret_cast<float*>(cb + 16384);            // 64 × 64 multipliers
  uint64_t* bar_mma = reinterpret_cast<uint64_t*>(cb + 4 * TC_TILE_BYTES);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(cb + 4 * TC_TILE_BYTES + 16);
  int* flag = reinterpret_cast<int*>(cb + 4 * TC_TILE_BYTES + 20);

  // Zero the panel rows past each segment's end (read by the MMA, never stored).
  {
    const int pad0 = T1 * TC_TM - m1, pad1 = T2 * TC_TM - p;
    const int rows = pad0 + pad1;
    for (int e = tid; e < rows * 4 * (TC_KB / 4); e += NTHREADS) {
      const int u = e / (rows * (TC_KB / 4)), rem = e - u * rows * (TC_KB / 4);
      const int rr = rem / (TC_KB / 4), g = rem - rr * (TC_KB / 4);
      const int ti = rr < pad0 ? T1 - 1 : NT - 1;
      const int r = rr < pad0 ? (m1 - (T1 - 1) * TC_TM) + rr : (p - (T2 - 1) * TC_TM) + (rr - pad0);
      *reinterpret_cast<float4*>(part[u] + (size_t)ti * TC_TILE_BYTES + tc_off(r, 4 * g)) =
          make_float4(0.f, 0.f, 0.f, 0.f);
    }
  }
  if (tid == 0) {
    tc_mbar_init(bar_mma);
    flag[0] = 0;
  }
  __syncwarp();
  if (warp == 0) tc_alloc256(tslot);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t ph_mma = 0;
  bool ok = true;

  for (int sb = 0; sb < nsb && ok; ++sb) {
    const int k0 = sb * TC_KB;
    const int kb = m1 - k0 < TC_KB ? m1 - k0 : TC_KB;   // the last superblock may be partial
    // (kb a multiple of 16: entries outside its kb × kb pivot block are held as zeros)
    // ---- phase A: sweep the pivot block, recording the multipliers.  Thread t holds the
    // eight entries of column t % 64 in rows t / 64 + 8u in registers; per pivot, the owners
    // of its row and column publish them (double-buffered by pivot parity, one barrier per
    // pivot) and every thread updates its entries.
    {
      const int pc = tid & (TC_KB - 1), pr0 = tid >> 6;
      float v[8];
#pragma unroll
      for (int u = 0; u < 8; ++u)
        v[u] = (pr0 + 8 * u < kb && pc < kb) ? SR[(size_t)(k0 + pr0 + 8 * u) * ldS + k0 + pc] : 0.f;
      bool good = true;
      for (int k = 0; k < kb; ++k) {
        float* rowb = rowbuf + (k & 1) * TC_KB;
        float* colb = colbuf + (k & 1) * TC_KB;
        const bool rowown = pr0 == (k & 7);
        float rk_own = 0.f;
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (rowown && u == (k >> 3)) rk_own = v[u];
        if (rowown) rowb[pc] = rk_own;
        if (pc == k) {
#pragma unroll
          for (int u = 0; u < 8; ++u) colb[pr0 + 8 * u] = v[u];
        }
        __syncthreads();
        const float d = rowb[k];
        const float dinv = 1.f / d;
        if (tid == 0) {
          const int kk = k0 + k;
          good = good && isfinite(d) && (kk < n ? d > zthr : (kk < nz ? d > 0.f : d < 0.f));
        }
        const float rk = rowb[pc];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int r = pr0 + 8 * u;
          if (r != k && pc != k) v[u] = fmaf(-(colb[r] * dinv), rk, v[u]);
          else if (r == k && pc == k) v[u] = -dinv;
          else v[u] = v[u] * dinv;
        }
        if (rowown) sR[k * TC_KB + pc] = (pc == k) ? dinv : rk * dinv;
      }
      if (tid == 0) flag[0] = good ? 0 : 1;
      __syncthreads();
      if (flag[0]) { ok = false; break; }
#pragma unroll
      for (int u = 0; u < 8; ++u)
        if (pr0 + 8 * u < kb && pc < kb) SR[(size_t)(k0 + pr0 + 8 * u) * ldS + k0 + pc] = v[u];
    }
    // ---- phase B: replay the 64 sweeps on every row outside the superblock; write the
    // panels (p = ĉ/d and c = ĉ, TF32 hi and lo) and the row's superblock entries.
    for (int i = tid; i < N; i += NTHREADS) {
      if (i >= k0 && i < k0 + kb) continue;
      float* row = SR + (size_t)i * ldS + k0;
      float v[TC_KB];
#pragma unroll
      for (int q = 0; q < TC_KB; q += 4) {
        float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
        if (q < kb) t = *reinterpret_cast<const float4*>(row + q);
        v[q] = t.x; v[q + 1] = t.y; v[q + 2] = t.z; v[q + 3] = t.w;
      }
      const int seg1 = i >= m1;
      const int li = seg1 ? i - m1 : i;
      const int ti = seg1 ? T1 + li / TC_TM : li / TC_TM, r = li % TC_TM;
      const size_t tb = (size_t)ti * TC_TILE_BYTES;
#pragma unroll
      for (int g = 0; g < TC_KB / 4; ++g) {
        float cc[4], pp[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int k = 4 * g + u;
          cc[u] = pp[u] = 0.f;   // pivots past kb: zero panel columns
          if (k < kb) {
            const float c = v[k];
            const float4* rk = reinterpret_cast<const float4*>(sR + k * TC_KB);
            const float dk = sR[k * TC_KB + k];
#pragma unroll
            for (int q4 = 0; q4 < TC_KB / 4; ++q4) {
              const float4 w = rk[q4];
              v[4 * q4 + 0] = fmaf(-c, w.x, v[4 * q4 + 0]);
              v[4 * q4 + 1] = fmaf(-c, w.y, v[4 * q4 + 1]);
              v[4 * q4 + 2] = fmaf(-c, w.z, v[4 * q4 + 2]);
              v[4 * q4 + 3] = fmaf(-c, w.w, v[4 * q4 + 3]);
            }
            v[k] = c * dk;   // overwrite the pivot column's (meaningless) update
            cc[u] = c;
            pp[u] = c * dk;
          }
        }
        const uint32_t o = tc_off(r, 4 * g);
        float ph[4], pl[4], ch[4], cl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          ph[u] = tc_hi(pp[u]); pl[u] = pp[u] - ph[u];
          ch[u] = tc_hi(cc[u]); cl[u] = cc[u] - ch[u];
        }
        *reinterpret_cast<float4*>(part[0] + tb + o) = make_float4(ph[0], ph[1], ph[2], ph[3]);
        *reinterpret_cast<float4*>(part[1] + tb + o) = make_float4(pl[0], pl[1], pl[2], pl[3]);
        *reinterpret_cast<float4*>(part[2] + tb + o) = make_float4(ch[0], ch[1], ch[2], ch[3]);
        *reinterpret_cast<float4*>(part[3] + tb + o) = make_float4(cl[0], cl[1], cl[2], cl[3]);
      }
#pragma unroll
      for (int q = 0; q < TC_KB; q += 4)
        if (q < kb) *reinterpret_cast<float4*>(row + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      if (i < m1) {
#pragma unroll
        for (int q = 0; q < TC_KB; ++q)
          if (q < kb) SR[(size_t)(k0 + q) * ldS + i] = v[q];
      }
    }
    __syncthreads();
    // ---- phase C: the rank-64 update, one 128 × 128 output tile at a time.  SR tiles:
    // row tiles 0..NT−1 (both segments) × column tiles 0..T1−1; λ-by-λ tiles: row tile I ≤
    // column tile J among the T2 λ tiles.  Tile t accumulates in TMEM columns 128·(t & 1);
    // its epilogue runs while the tensor core computes tile t + 1.
    const int nsr = NT * T1, nll = T2 * (T2 + 1) / 2, ntiles = nsr + nll;
    auto tile_of = [&](int t, int& ta, int& tbi) {
      if (t < nsr) {
        ta = t / T1; tbi = t - ta * T1;
      } else {
        int u = t - nsr, I = 0;
        while (u >= T2 - I) { u -= T2 - I; ++I; }
        ta = T1 + I; tbi = T1 + I + u;
      }
    };
    int prevA = -1, pta = 0, ptb = 0;
    for (int t = 0; t <= ntiles && ok; ++t) {
      int ta = 0, tbi = 0;
      if (t < ntiles) {
        tile_of(t, ta, tbi);
        // stage the operand tiles (A only when the row tile changes); the MMA of tile t − 1
        // has completed, so its operands may be overwritten.  All loads first, then stores.
        constexpr int PER = (int)(TC_TILE_BYTES / 16) / NTHREADS;   // float4 per thread, part
        // h = 0: the row tile's p panel (kept while the row tile stays), h = 1: the column
        // tile's c panel (every tile); hi and lo parts each
        for (int h = (ta != prevA) ? 0 : 1; h < 2; ++h) {
          const int tt = h ? tbi : ta;
          const float4* __restrict__ s0 =
              reinterpret_cast<const float4*>(part[2 * h] + (size_t)tt * TC_TILE_BYTES);
          const float4* __restrict__ s1 =
              reinterpret_cast<const float4*>(part[2 * h + 1] + (size_t)tt * TC_TILE_BYTES);
          float4 r[2 * PER];
#pragma unroll
          for (int j = 0; j < PER; ++j) {
            r[j] = s0[tid + j * NTHREADS];
            r[PER + j] = s1[tid + j * NTHREADS];
          }
          float4* d0 = reinterpret_cast<float4*>(h ? sBt[0] : sA[0]);
          float4* d1 = reinterpret_cast<float4*>(h ? sBt[1] : sA[1]);
#pragma unroll
          for (int j = 0; j < PER; ++j) {
            d0[tid + j * NTHREADS] = r[j];
            d1[tid + j * NTHREADS] = r[PER + j];
          }
        }
        prevA = ta;
        tc_proxy_fence();
        __syncthreads();
        if (tid == 0) {
          // D = C_tile · P_tileᵀ: TMEM lane l is the output column of c-panel row l and TMEM
          // column c the output row of p-panel row c, so the epilogue's warps touch
          // consecutive columns of one row per access
          tc_fence_after();
          constexpr uint32_t id = tc_idesc(TC_TM, TC_TN);
          const uint32_t acc = tmem + (uint32_t)(TC_TN * (t & 1));
#pragma unroll
          for (int s = 0; s < TC_KB / 8; ++s) {
            const uint32_t ko = (uint32_t)s * 256;   // two K-adjacent core matrices per step
            tc_mma_tf32(acc, sBt[0] + ko, sA[0] + ko, 128, 2048, id, s > 0);   // hi · hi
            tc_mma_tf32(acc, sBt[0] + ko, sA[1] + ko, 128, 2048, id, true);    // hi · lo
            tc_mma_tf32(acc, sBt[1] + ko, sA[0] + ko, 128, 2048, id, true);    // lo · hi
          }
          // arrives on bar_mma once every MMA issued so far has completed
          tc_commit(bar_mma);
        }
      }
      if (t > 0) {
        // epilogue of tile t − 1 (its MMA completed before the last barrier): warp w reads
        // TMEM lanes 32·(w%4)… (tile columns) and TMEM columns 32·(w/4)… (tile rows); lane
        // l holds column 32·(w%4) + l of 32 consecutive rows
        __syncwarp();
        tc_fence_after();
        const int qd = warp & 3, cg = warp >> 2;
        float d[32];
        tc_ld32(tmem + (uint32_t)(TC_TN * ((t - 1) & 1)) + ((uint32_t)(32 * qd) << 16) +
                    (uint32_t)(32 * cg), d);
        const int lc = 32 * qd + lane;                   // column within the tile
        const int lr = 32 * cg;                          // first row within the tile
        if (t - 1 < nsr) {
          const int j = ptb * TC_TM + lc;
          const bool colok = j < m1 && !(j >= k0 && j < k0 + kb);
          const int ib = pta < T1 ? pta * TC_TM + lr : m1 + (pta - T1) * TC_TM + lr;
          const int iend = pta < T1 ? m1 : N;
          float* __restrict__ c = SR + (size_t)ib * ldS + j;
          // all 32 loads in flight before the first store
          uint32_t live = 0;
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int i = ib + r;
            if (colok && i < iend && !(i >= k0 && i < k0 + kb)) live |= 1u << r;
          }
#pragma unroll
          for (int hh = 0; hh < 32; hh += 16) {   // 16 loads in flight, then 16 stores
            float x[16];
#pragma unroll
            for (int r = 0; r < 16; ++r)
              if (live >> (hh + r) & 1) x[r] = c[(size_t)(hh + r) * ldS];
#pragma unroll
            for (int r = 0; r < 16; ++r)
              if (live >> (hh + r) & 1) c[(size_t)(hh + r) * ldS] = x[r] - d[hh + r];
          }
        } else {
          // λ-by-λ block: the strict upper triangle in Mb, the diagonal in dM; loads first
          const int b = (ptb - T1) * TC_TM + lc;
          const int ab = (pta - T1) * TC_TM + lr;
          float* __restrict__ mrow = Mb + (size_t)ab * ldM + b;
          uint32_t live = 0;
#pragma unroll
          for (int r = 0; r < 32; ++r) {
            const int a = ab + r;
            if (a < p && b < p && b >= a) live |= 1u << r;
          }
          const int rdiag = b - ab;   // the row whose entry is the diagonal (if 0 ≤ rdiag < 32)
#pragma unroll
          for (int hh = 0; hh < 32; hh += 16) {
            float x[16];
#pragma unroll
            for (int r = 0; r < 16; ++r)
              if (live >> (hh + r) & 1)
                x[r] = (hh + r == rdiag) ? dM[ab + hh + r] : mrow[(size_t)(hh + r) * ldM];
#pragma unroll
            for (int r = 0; r < 16; ++r)
              if (live >> (hh + r) & 1) {
                if (hh + r == rdiag) dM[ab + hh + r] = x[r] - d[hh + r];
                else mrow[(size_t)(hh + r) * ldM] = x[r] - d[hh + r];
              }
          }
        }
      }
      if (t < ntiles) {
        if (!tc_wait(bar_mma, ph_mma)) atomicExch(flag, 2);
        ph_mma ^= 1;
        pta = ta; ptb = tbi;
      }
      // the epilogue's TMEM reads finish before the next MMA reuses its accumulator
      tc_fence_before();
      __syncthreads();
      if (flag[0]) ok = false;
    }
    __syncthreads();
  }
  // Leave nothing in flight: a failed wait is retried (bounded) before the memory goes.
  if (tid == 0 && flag[0] == 2) tc_wait(bar_mma, ph_mma ^ 1);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    __syncwarp();
    tc_fence_after();
    tc_dealloc256(tmem);
  }
  if (tid == 0) {
    tc_mbar_inval(bar_mma);
  }
  __syncthreads();
  return ok;
}

}  // namespace qpk
