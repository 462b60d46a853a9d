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
//  * phase A (warp 0): the 64 × 64 pivot block is swept in shared memory, pivot after
//    pivot, recording each pivot's row of multipliers r_k (r_kk = 1/d_k, r_kq = a_kq/d_k);
//  * phase B (all threads, one row each): every row outside K replays the 64 scalar sweeps
//    on its 64 entries of K's columns (so the result equals the pivot-by-pivot sweep), and
//    writes p_iq and c_iq, split into TF32 high and low parts, to the panel tiles in the
//    workspace;
//  * phase C: for each 128 × 128 output tile, all threads stage the four 32 KB operand tiles
//    in shared memory (16-byte loads of the contiguous panel tiles, then a proxy fence), one
//    thread issues 8 K-steps × 3 tcgen05.mma (kind::tf32:
//    hi·hi + hi·lo + lo·hi, the 3×TF32 split that keeps FP32 accuracy) into a TMEM
//    accumulator, and all 16 warps read it back (tcgen05.ld) and subtract it from the
//    matrix in global memory, skipping K's rows and columns and, in the λ-by-λ block, the
//    strict lower triangle.
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
__device__ void tc_alloc128(uint32_t* slot);
__device__ void tc_dealloc128(uint32_t tmem);
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
// TMEM allocation of the 128 columns of one FP32 128 × 128 accumulator (warp-collective).
__device__ __forceinline__ void tc_alloc128(uint32_t* slot) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], 128;"
               :: "r"(tc_smem_u32(slot)) : "memory");
}
__device__ __forceinline__ void tc_dealloc128(uint32_t tmem) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, 128;" :: "r"(tmem) : "memory");
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

// Superblock sweeps of pivots [0, 64·nsb) of the matrix gsweep_setup holds (SR: rows 0..N−1
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
  // shared layout from the first 1024-byte boundary: phase C operands A-hi, A-lo, B-hi, B-lo
  // at 0 / 32 / 64 / 96 KB, then the mbarrier, the TMEM address and a flag; phases A/B reuse
  // the operand space
  unsigned char* cb = cb0 + ((1024 - (reinterpret_cast<uintptr_t>(cb0) & 1023)) & 1023);
  unsigned char* sA[2] = {cb, cb + TC_TILE_BYTES};
  unsigned char* sBt[2] = {cb + 2 * TC_TILE_BYTES, cb + 3 * TC_TILE_BYTES};
  float* sB = reinterpret_cast<float*>(cb);                    // 64 × 64 pivot block
  float* sR = reinterpret_cast<float*>(cb + 16384);            // 64 × 64 multipliers
  float* colk = reinterpret_cast<float*>(cb + 4 * TC_TILE_BYTES - 512);   // inside B-lo
  float* rowk = colk + 64;
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
  if (warp == 0) tc_alloc128(tslot);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tslot;
  uint32_t ph_mma = 0;
  bool ok = true;

  for (int sb = 0; sb < nsb && ok; ++sb) {
    const int k0 = sb * TC_KB;
    // ---- phase A (warp 0): sweep the pivot block, recording the multipliers.
    if (warp == 0) {
      for (int e = lane; e < TC_KB * TC_KB; e += 32)
        sB[e] = SR[(size_t)(k0 + e / TC_KB) * ldS + k0 + e % TC_KB];
      __syncwarp();
      bool good = true;
      for (int k = 0; k < TC_KB; ++k) {
        const float d = sB[k * TC_KB + k];
        const int kk = k0 + k;
        good = good && isfinite(d) && (kk < n ? d > zthr : (kk < nz ? d > 0.f : d < 0.f));
        const float dinv = 1.f / d;
        colk[lane] = sB[lane * TC_KB + k];
        colk[lane + 32] = sB[(lane + 32) * TC_KB + k];
        rowk[lane] = sB[k * TC_KB + lane];
        rowk[lane + 32] = sB[k * TC_KB + lane + 32];
        sR[k * TC_KB + lane] = (lane == k) ? dinv : sB[k * TC_KB + lane] * dinv;
        sR[k * TC_KB + lane + 32] = (lane + 32 == k) ? dinv : sB[k * TC_KB + lane + 32] * dinv;
        __syncwarp();
#pragma unroll 4
        for (int r = 0; r < TC_KB; ++r) {
          const float f = colk[r] * dinv;
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const int c = lane + 32 * h;
            float v = sB[r * TC_KB + c];
            if (r != k && c != k) v = fmaf(-f, rowk[c], v);
            else if (r == k && c == k) v = -dinv;
            else v = v * dinv;
            sB[r * TC_KB + c] = v;
          }
        }
        __syncwarp();
      }
      for (int e = lane; e < TC_KB * TC_KB; e += 32)
        SR[(size_t)(k0 + e / TC_KB) * ldS + k0 + e % TC_KB] = sB[e];
      if (lane == 0) flag[0] = good ? 0 : 1;
    }
    __syncthreads();
    if (flag[0]) { ok = false; break; }
    // ---- phase B: replay the 64 sweeps on every row outside the superblock; write the
    // panels (p = ĉ/d and c = ĉ, TF32 hi and lo) and the row's superblock entries.
    for (int i = tid; i < N; i += NTHREADS) {
      if (i >= k0 && i < k0 + TC_KB) continue;
      float* row = SR + (size_t)i * ldS + k0;
      float v[TC_KB];
#pragma unroll
      for (int q = 0; q < TC_KB; q += 4) {
        const float4 t = *reinterpret_cast<const float4*>(row + q);
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
        *reinterpret_cast<float4*>(row + q) = make_float4(v[q], v[q + 1], v[q + 2], v[q + 3]);
      if (i < m1) {
#pragma unroll
        for (int q = 0; q < TC_KB; ++q) SR[(size_t)(k0 + q) * ldS + i] = v[q];
      }
    }
    __syncthreads();
    // ---- phase C: the rank-64 update, one 128 × 128 output tile at a time.  SR tiles:
    // row tiles 0..NT−1 (both segments) × column tiles 0..T1−1; λ-by-λ tiles: row tile I ≤
    // column tile J among the T2 λ tiles.
    const int nsr = NT * T1, nll = T2 * (T2 + 1) / 2;
    int prevA = -1;
    for (int t = 0; t < nsr + nll && ok; ++t) {
      int ta, tbi;
      if (t < nsr) {
        ta = t / T1; tbi = t - ta * T1;
      } else {
        int u = t - nsr, I = 0;
        while (u >= T2 - I) { u -= T2 - I; ++I; }
        ta = T1 + I; tbi = T1 + I + u;
      }
      // stage the operand tiles (A only when the row tile changes); the MMA of the previous
      // tile has completed, so its operands may be overwritten
      {
        const bool newA = ta != prevA;
        const float4* src[4] = {
            reinterpret_cast<const float4*>(part[0] + (size_t)ta * TC_TILE_BYTES),
            reinterpret_cast<const float4*>(part[1] + (size_t)ta * TC_TILE_BYTES),
            reinterpret_cast<const float4*>(part[2] + (size_t)tbi * TC_TILE_BYTES),
            reinterpret_cast<const float4*>(part[3] + (size_t)tbi * TC_TILE_BYTES)};
        float4* dst[4] = {reinterpret_cast<float4*>(sA[0]), reinterpret_cast<float4*>(sA[1]),
                          reinterpret_cast<float4*>(sBt[0]), reinterpret_cast<float4*>(sBt[1])};
        constexpr int NV = (int)(TC_TILE_BYTES / 16);
        for (int u = newA ? 0 : 2; u < 4; ++u)
          for (int e = tid; e < NV; e += NTHREADS) dst[u][e] = src[u][e];
        prevA = ta;
      }
      tc_proxy_fence();
      __syncthreads();
      if (tid == 0) {
        tc_fence_after();
        constexpr uint32_t id = tc_idesc(TC_TM, TC_TN);
#pragma unroll
        for (int s = 0; s < TC_KB / 8; ++s) {
          const uint32_t ko = (uint32_t)s * 256;   // two K-adjacent core matrices per step
          tc_mma_tf32(tmem, sA[0] + ko, sBt[0] + ko, 128, 2048, id, s > 0);   // hi · hi
          tc_mma_tf32(tmem, sA[0] + ko, sBt[1] + ko, 128, 2048, id, true);    // hi · lo
          tc_mma_tf32(tmem, sA[1] + ko, sBt[0] + ko, 128, 2048, id, true);    // lo · hi
        }
        // arrives on bar_mma once every MMA issued so far has completed
        tc_commit(bar_mma);
      }
      const bool done = tc_wait(bar_mma, ph_mma);
      ph_mma ^= 1;
      if (!done) atomicExch(flag, 2);
      __syncwarp();
      tc_fence_after();
      // epilogue: warp w reads TMEM lanes 32·(w%4)… (tile rows) and columns 32·(w/4)…
      {
        const int qd = warp & 3, cg = warp >> 2;
        float d[32];
        tc_ld32(tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(32 * cg), d);
        const int lr = 32 * qd + lane;                   // row within the tile
        const int lc = 32 * cg;                          // first column within the tile
        if (done) {
          if (t < nsr) {
            const int gi = ta < T1 ? ta * TC_TM + lr : m1 + (ta - T1) * TC_TM + lr;
            const int gj = tbi * TC_TM + lc;
            const bool rowok = (ta < T1 ? gi < m1 : gi < N) && !(gi >= k0 && gi < k0 + TC_KB);
            const bool colok = gj < m1 && !(gj >= k0 && gj < k0 + TC_KB);
            if (rowok && colok) {
              float* c = SR + (size_t)gi * ldS + gj;
#pragma unroll
              for (int q = 0; q < 32; q += 4) {
                if (gj + q < m1) {
                  float4 x = *reinterpret_cast<float4*>(c + q);
                  x.x -= d[q]; x.y -= d[q + 1]; x.z -= d[q + 2]; x.w -= d[q + 3];
                  *reinterpret_cast<float4*>(c + q) = x;
                }
              }
            }
          } else {
            const int a = (ta - T1) * TC_TM + lr;
            const int b0 = (tbi - T1) * TC_TM + lc;
            if (a < p) {
#pragma unroll 4
              for (int q = 0; q < 32; ++q) {
                const int b = b0 + q;
                if (b < p && b >= a) {
                  if (b == a) dM[a] -= d[q];
                  else Mb[(size_t)a * ldM + b] -= d[q];
                }
              }
            }
          }
        }
      }
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
    tc_dealloc128(tmem);
  }
  if (tid == 0) {
    tc_mbar_inval(bar_mma);
  }
  __syncthreads();
  return ok;
}

}  // namespace qpk
