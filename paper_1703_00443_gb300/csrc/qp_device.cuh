// qp_device.cuh -- device code of the batched differentiable QP solver for sm_103a.
//
// One thread block (512 threads) owns one QP instance for the whole solve, so the
// interior point loop runs without a host round trip and each instance stops on its own
// convergence test.  Method: Amos & Kolter 2017, §3.1 (Mehrotra predictor-corrector
// primal-dual interior point method in slack form, Eq. 9 and Eq. 10, with the KKT system
// symmetrised and block-eliminated so that only an nineq×nineq matrix is factored per
// iteration) and §3.1.1 (backward pass with the factorisation at the solution, Eq. 11).
//
// Block elimination used here.  With K11 = [Q Aᵀ; A 0] (the part of the symmetrised KKT
// matrix that never changes) and S = K11⁻¹ = [P T; Tᵀ −S_A⁻¹], the Newton system
//     [Q Gᵀ Aᵀ; G −D(s/λ) 0; A 0 0] [Δz; Δλ; Δν] = [r1; r̃3; r4]
// reduces to
//     (M + D(s/λ)) Δλ = RE·[r1; r4] − r̃3,   [Δz; Δν] = S·[r1; r4] − REᵀ Δλ,
// where RE = [G 0]·S = [GP, GT] (nineq × (n+neq)) and M = G P Gᵀ.  S, RE and M are
// produced together, once per solve, by a symmetric Gauss-Jordan sweep over the first
// n+neq pivots of [[K11, [G 0]ᵀ], [[G 0], 0]] held in registers (4×4 tiles per thread).
// Each iteration factors M + D(s/λ) = L Lᵀ by a right-looking Cholesky in 4×4 register
// tiles that forms X = L⁻¹ in the same loop (chol_blk with FULLX), so every triangular solve
// is a product with X or Xᵀ (chol_solve).
//
// Precision.  T is the matrix/factor type (float or double).  The iterate (z, s, λ, ν)
// is kept in FP64, and the KKT residual vectors and the backward refinement residual are
// FP64-accurate; the norms of the stopping test, μ and the step-length reductions are FP32
// reductions in both dtypes (enough for them).  For T = float the residual products
// use error-free FP32 transformations (Dekker's product by FMA and Knuth's two-sum), a
// double-float accumulation whose error is about 2⁻⁴⁸ of Σ|terms|, because the FP64 pipe
// of this part is a small fraction of the FP32 rate.  The Newton directions themselves
// are FP32; with an exact residual each iteration acts as a refinement step, so the
// returned iterate is accurate well past FP32 precision.
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

namespace qpk {

constexpr int NTHREADS = 512;
constexpr int NWARPS = NTHREADS / 32;
// Scratch elements blk_solve needs: the block's right-hand side, per-warp partial sums and
// the staged inverse diagonal block (32 × 33).
constexpr int BLK_SOLVE_SCR = 32 + 32 * NWARPS + 32 * 33;
// Shared-memory budget (bytes) under which the global-memory path keeps its Cholesky panels
// in shared memory; below every supported device's opt-in limit of the target (227 KB).
constexpr size_t LARGE_PANEL_SMEM_CAP = 200 * 1024;
// Column block of the global-memory Cholesky: 32 for FP32, 16 for FP64 (one warp holds the
// pivot block's row and its inverse's row in registers).
__host__ __device__ constexpr int chol_nb(int esz) { return esz == 4 ? 32 : 16; }
// Largest p for which the global-memory path factors with the register-tile Cholesky
// (4×4 tiles of the lower triangle in at most two register slots per thread).
constexpr int REG_CHOL_MAX_P = 176;
// Whether the global-memory path factors a p×p Schur complement with the register-tile
// Cholesky (chol_blk with FULLX: X = L⁻¹ in Mb, solves by two products) rather than the
// blocked routine (gchol_factor: L with inverted 32×32 (16×16 in FP64) diagonal blocks in
// Mb, solved by block substitution, blk_solve).
__host__ __device__ inline bool reg_chol_ok(int p, int esz) {
  const int NT = (p + 3) >> 2, nt = NT * (NT + 1) / 2;
  return nt <= NTHREADS || (esz == 4 && nt <= 2 * NTHREADS && p <= REG_CHOL_MAX_P);
}

enum : int { ST_CONV = 0, ST_MAXIT = 1, ST_NOTPD = 2, ST_NUM = 3, ST_NOFWD = 4, ST_INFEAS = 5,
             ST_TIMEOUT = 6 };
// Flag bit of the status word kept in the workspace (reported by the backward pass): a nearly
// degenerate complementarity pair at the returned iterate.
constexpr int FLAG_NEARDEG = 0x100;
// Flag bit: Q was only positive semidefinite and the factorisations used Q + δI (the
// residual and the backward refinement use Q itself).
constexpr int FLAG_REGQ = 0x200;
// Magic word of the workspace stamp the forward pass leaves for the backward pass.
constexpr int32_t STAMP_MAGIC = 0x51504657;

// 32-bit mix of an instance's Q, G and A addresses (part of the workspace stamp), so that a
// backward pass given other buffers than its forward pass is detected.
__host__ __device__ inline int32_t stamp_hash(const void* Q, const void* G, const void* A) {
  unsigned long long h = (unsigned long long)(uintptr_t)Q * 0x9E3779B97F4A7C15ull;
  h ^= (unsigned long long)(uintptr_t)G * 0xC2B2AE3D27D4EB4Full;
  h ^= (unsigned long long)(uintptr_t)A * 0x165667B19E3779F9ull;
  h ^= h >> 29;
  return (int32_t)(uint32_t)(h ^ (h >> 32));
}

__host__ __device__ inline size_t align_up(size_t x, size_t a) { return (x + a - 1) / a * a; }
}  // namespace qpk

#include "qp_tc.cuh"

namespace qpk {

// Shared memory of the global-memory forward kernel after its work region: the FP64 and
// split vectors, the FP32 vectors and the reduction scratch (FwdSmem: odbl .. total).
__host__ __device__ inline size_t large_tail_bytes(int n, int p, int m, int m1, size_t es) {
  const size_t p4 = (size_t)(p + 3) / 4 * 4;
  return align_up(8 * (3 * (size_t)n + 4 * (size_t)p + 3 * (size_t)m), 16) +
         align_up(8 * ((size_t)n + p + m), 16) + align_up(es * (3 * (size_t)m1 + 12 * p4), 16) +
         align_up(8 * 4 * NWARPS, 16);
}

// Whether the global-memory path runs the setup sweep's rank-64 updates on the tensor cores
// (qp_tc.cuh): FP32, at least two 64-pivot superblocks, and the operand tiles fit in the
// shared work region next to the vectors.  A pure function of the sizes, so the workspace
// layout, the shared-memory size and the kernel agree.
__host__ __device__ inline bool tc_sweep_ok(int n, int nz, int p, int m, int esz) {
  const int m1 = nz + m;
  return esz == 4 && m1 >= TC_MIN_M1 &&
         TC_SMEM_BYTES + large_tail_bytes(n, p, m, m1, 4) <= TC_SMEM_CAP;
}

// Number of primal variables after padding: 0-3 decoupled dummy variables (Q = 1 on the
// diagonal, no constraint coupling) make n + neq a multiple of 4, so the pivot blocks of
// the setup sweep are whole 4×4 tiles.  Dummies sit after the real z entries and stay 0.
__host__ __device__ inline int padded_nz(int n, int m) { return n + ((4 - (n + m) % 4) % 4); }

// ------------------------------------------------------------------ layouts
// Per-instance workspace (global memory) kept from forward to backward.
// Layout shared by both kernel paths (the backward pass reads only this prefix):
// SR = [S; RE] ((m1+p) × m1, m1 = nz + neq), the p×p block with the factor of M + D(s/λ)
// (lower triangle: X = L⁻¹, or for large p on the global path L with inverted diagonal
// blocks) and M (strict upper), the FP64 iterate (z, s, λ, ν) and the stamp: eight int32 words
// {status code | flags, STAMP_MAGIC, n, nineq, neq, element size | path << 8, nz,
// stamp_hash(Q, G, A)} that the backward pass checks before it trusts the rest.  The global-memory
// path appends diag(M), its Cholesky work matrix (row stride round4(p)) and its panel
// scratch (the sweep's two 16-row panels, or the Cholesky's panel and staging buffer).
struct WsLayout {
  size_t oSR, oX, oIt, oSt, odM, oAw, oPan, oTc, inst;
  // tc_region: room for the tensor-core sweep's panel tiles where the size takes that sweep
  // (the fixed-size global-memory kernel; the packed kernels use the CUDA-core sweep).
  __host__ __device__ void init(int n, int nz, int p, int m, int esz, bool large,
                                bool tc_region = true) {
    const size_t m1 = (size_t)nz + m;
    oSR = 0;
    oX = align_up(oSR + (m1 + p) * m1 * esz, 256);
    oIt = align_up(oX + (size_t)p * p * esz, 256);
    oSt = align_up(oIt + 8 * ((size_t)n + 2 * (size_t)p + m), 256);
    size_t o = align_up(oSt + 32, 256);
    odM = oAw = oPan = oTc = o;
    if (large) {
      const size_t N = m1 + p, ldp = (N + 7) / 8 * 8;
      odM = o;  o = align_up(o + (size_t)p * esz, 256);
      const size_t cpan = 2 * (size_t)chol_nb(esz) * (size_t)((p + 7) & ~7);
      const size_t span = 2 * 16 * ldp;
      oAw = o;  o = align_up(o + (size_t)p * ((p + 3) & ~3) * esz, 256);
      oPan = o; o = align_up(o + (span > cpan ? span : cpan) * esz, 256);
      oTc = o;
      if (tc_region && tc_sweep_ok(n, nz, p, m, esz))
        o = align_up(o + tc_panel_bytes((int)m1, p), 256);
    }
    inst = o;
  }
};

// Dynamic shared memory of the forward kernel.
template <typename T>
struct FwdSmem {
  int nz, m1, N3, ldS, ldM, NT3, NTp, pan_smem, span_smem, tc_sweep;
  size_t oSR, oMb, odM, ocb, cbytes, odbl, osplit, ovec, ored, total;
  // large: S/RE, M/X and diag(M) live in the global workspace, only vectors and a work
  // region stay in shared memory.
  __host__ __device__ void init(int n, int nzp, int p, int m, bool large) {
    nz = nzp;
    m1 = nz + m;
    N3 = m1 + p;
    ldS = m1;
    ldM = p > 0 ? (p + 3) / 4 * 4 : 1;   // rows of M/X on 16-byte boundaries
    NT3 = (N3 + 3) / 4;
    NTp = (p + 3) / 4;
    const size_t es = sizeof(T);
    size_t o = 0;
    oSR = oMb = odM = 0;
    if (!large) {
      oSR = o;   o = align_up(o + (size_t)(m1 + p) * ldS * es, 16);
      oMb = o;   o = align_up(o + (size_t)p * ldM * es, 16);
      odM = o;   o = align_up(o + (size_t)p * es, 16);
    }
    // Work region: panel buffers of the blocked factorisations, reused as partial-sum
    // scratch by kkt_apply and mv_cols (never live at the same time).
    ocb = o;
    {
      size_t c;
      if (!large) {
        size_t a = 2 * (32 * (size_t)NT3 + 16), b = 2 * (32 * (size_t)NTp + 16);
        c = (a > b ? a : b) * es + 64;
        if (c < 8 * (size_t)NTHREADS) c = 8 * (size_t)NTHREADS;
        if (c < BLK_SOLVE_SCR * es) c = BLK_SOLVE_SCR * es;
      } else {
        // ≥ the pivot scratch of the large routines, and ≥ the panels of the register-tile
        // Cholesky, which the global-memory path uses while p ≤ REG_CHOL_MAX_P.
        c = 8 * (size_t)4 * NTHREADS;
        const size_t nt = (size_t)((p < REG_CHOL_MAX_P ? p : REG_CHOL_MAX_P) + 3) / 4;
        const size_t rc = (2 * (32 * nt + 16) + 16) * es;
        if (rc > c) c = rc;
      }
      cbytes = align_up(c, 16);
    }
    pan_smem = span_smem = tc_sweep = 0;
    const size_t p4 = (size_t)(p + 3) / 4 * 4;
    const size_t tail = large_tail_bytes(n, p, m, m1, es);
    if (large) {
      // The Cholesky panel and staging buffer (pivot scratch plus 2·chol_nb rows of ld
      // round8(p)) go to the work region when the whole layout stays within
      // LARGE_PANEL_SMEM_CAP bytes.
      // The setup sweep's two 16-row panels (ld round8(m1 + p)) likewise, after its pivot
      // scratch, if they fit too.
      const size_t nb = (size_t)chol_nb((int)es);
      const size_t pc = align_up(((2 * nb * nb + 2 * nb + 16) + 2 * nb * (size_t)((p + 7) & ~7)) * es, 16);
      const size_t sc = align_up((2 * 16 * 16 + 16 + 2 * 16 * (size_t)((N3 + 7) & ~7)) * es, 16);
      if (o + (pc > cbytes ? pc : cbytes) + tail <= LARGE_PANEL_SMEM_CAP) {
        pan_smem = 1;
        if (pc > cbytes) cbytes = pc;
      }
      if (o + (sc > cbytes ? sc : cbytes) + tail <= LARGE_PANEL_SMEM_CAP) {
        span_smem = 1;
        if (sc > cbytes) cbytes = sc;
      }
      // The tensor-core sweep stages its operand tiles in the work region.
      if (tc_sweep_ok(n, nz, p, m, (int)es)) {
        tc_sweep = 1;
        if (TC_SMEM_BYTES > cbytes) cbytes = align_up(TC_SMEM_BYTES, 16);
      }
    }
    o += cbytes;
    odbl = o;  o = align_up(o + 8 * (3 * (size_t)n + 4 * (size_t)p + 3 * (size_t)m), 16);
    osplit = o; o = align_up(o + 8 * ((size_t)n + p + m), 16);
    ovec = o;  o = align_up(o + es * (3 * (size_t)m1 + 12 * p4), 16);
    ored = o;  o = align_up(o + 8 * 4 * NWARPS, 16);
    total = o;
  }
};

// Dynamic shared memory of the backward kernel (vectors only).
template <typename T>
struct BwdSmem {
  size_t odbl, osplit, ovec, ored, oscr, oSR, oX, total;
  // staged: S/RE and X = L⁻¹ are copied from the workspace into shared memory first.
  __host__ __device__ void init(int n, int nz, int p, int m, bool staged = false) {
    const size_t m1 = (size_t)nz + m, es = sizeof(T);
    size_t o = 0;
    oSR = oX = 0;
    if (staged) {
      oSR = o; o = align_up(o + (m1 + p) * m1 * es, 16);
      oX = o;  o = align_up(o + (size_t)p * p * es, 16);
    }
    odbl = o;   o = align_up(o + 8 * (3 * ((size_t)n + p + m) + 2 * (size_t)p), 16);
    osplit = o; o = align_up(o + 8 * ((size_t)n + p + m), 16);
    ovec = o;   o = align_up(o + es * (3 * m1 + 4 * (size_t)(p + 3) / 4 * 4), 16);
    ored = o;   o = align_up(o + 8 * 4 * NWARPS, 16);
    oscr = o;   o = align_up(o + 8 * (size_t)4 * NTHREADS, 16);
    total = o;
  }
};

template <typename T>
struct FwdParams {
  int B, n, p, m, nz;
  const T *Q, *q, *G, *h, *A, *b;
  T *z, *lam, *nu;
  int32_t *status, *iters;
  double* resid;   // optional [B, 4]: final ‖r_z‖∞, ‖Gz+s−h‖∞, ‖Az−b‖∞, μ
  unsigned char* ws;
  size_t ws_inst;
  double tol, mu_tol;
  int max_iter;
  unsigned long long time_limit_ns;   // 0: none
};

// Per-instance views used by the kernel bodies (built from the fixed-size parameters or from
// a packed-batch descriptor).
template <typename T>
struct FwdInst {
  int n, p, m, nz;
  const T *Q, *q, *G, *h, *A, *b;
  T *z, *lam, *nu;
  int32_t *status, *iters;   // this instance's slots (or null)
  double* resid;             // this instance's four residual values (or null)
  unsigned char* ws;         // this instance's workspace
  double tol, mu_tol;
  int max_iter;
  unsigned long long time_limit_ns;   // 0: none
};

template <typename T>
struct BwdInst {
  int n, p, m, nz, large, staged;
  const T *Q, *G, *A, *dl_dz;
  T *dQ, *dq, *dG, *dh, *dA, *db;
  const unsigned char* ws;
  int refine;
  const T *dl_dlam, *dl_dnu;   // ∂ℓ/∂λ*, ∂ℓ/∂ν* of this instance (or null: zero)
  int32_t* status;             // this instance's backward status slot (or null)
};

// Descriptor of one instance of a packed (uneven) batch; the C ABI's qp_instance_desc has
// the same layout.
struct PackedDesc {
  int32_t n, nineq, neq, id, nz, flags;
  int64_t oQ, oq, oG, oh, oA, ob, oz, olam, onu, ows;
};

template <typename T>
struct PackedFwdParams {
  int B;
  const PackedDesc* desc;
  int* counter;
  const T *Q, *q, *G, *h, *A, *b;
  T *z, *lam, *nu;
  int32_t *status, *iters;
  double* resid;
  unsigned char* ws;
  double tol, mu_tol;
  int max_iter;
  unsigned long long time_limit_ns;
};

template <typename T>
struct PackedBwdParams {
  int B;
  const PackedDesc* desc;
  int* counter;
  const T *Q, *G, *A, *dl_dz;
  T *dQ, *dq, *dG, *dh, *dA, *db;
  const unsigned char* ws;
  int refine;
  int32_t* status;   // [B] by instance id, or null
};

template <typename T>
struct BwdParams {
  int B, n, p, m, nz;
  int large;
  int staged;   // S/RE and X staged in shared memory (BwdSmem with staged = true)
  const T *Q, *G, *A, *dl_dz;
  T *dQ, *dq, *dG, *dh, *dA, *db;
  const unsigned char* ws;
  size_t ws_inst;
  int refine;
  const T *dl_dlam, *dl_dnu;   // [B, nineq], [B, neq] or null (zero)
  int32_t* status;             // [B] or null
};

// ------------------------------------------------------------------ FP64-accurate dot products
template <typename T> struct Split;
template <> struct Split<float> {
  using V = float2;
  __device__ static __forceinline__ V make(double x) {
    const float hi = __double2float_rn(x);
    return make_float2(hi, __double2float_rn(x - (double)hi));
  }
};
template <> struct Split<double> {
  using V = double;
  __device__ static __forceinline__ V make(double x) { return x; }
};

template <typename T> struct Acc;
template <> struct Acc<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double a, double x) { s = fma(a, x, s); }
  __device__ __forceinline__ void merge(const Acc& o) { s += o.s; }
  __device__ __forceinline__ void shfl_merge(int off) {
    s += __shfl_xor_sync(0xffffffffu, s, off);
  }
  __device__ __forceinline__ double value() const { return s; }
};
// Double-float accumulator: a·x_hi is split exactly into p + e (FMA), p is added to hi
// with Knuth's two-sum, and all low-order parts go to lo.  __fadd_rn/__fmul_rn are never
// contracted into FMAs, which keeps the transformations error-free.
template <> struct Acc<float> {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float a, float2 x) {
    const float p = __fmul_rn(a, x.x);
    const float e = fmaf(a, x.x, -p);
    const float t = __fadd_rn(hi, p);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(p, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(err, fmaf(a, x.y, e)));
  }
  // (hi, lo) += (ohi, olo) with a two-sum on the high parts.
  __device__ __forceinline__ void merge2(float ohi, float olo) {
    const float t = __fadd_rn(hi, ohi);
    const float bp = __fsub_rn(t, hi);
    const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(t, bp)), __fsub_rn(ohi, bp));
    hi = t;
    lo = __fadd_rn(lo, __fadd_rn(olo, err));
  }
  __device__ __forceinline__ void merge(const Acc& o) { merge2(o.hi, o.lo); }
  __device__ __forceinline__ void shfl_merge(int off) {
    merge2(__shfl_xor_sync(0xffffffffu, hi, off), __shfl_xor_sync(0xffffffffu, lo, off));
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------------------ block reductions
enum : int { R_SUM = 0, R_MAX = 1, R_MIN = 2 };

template <int OP>
__device__ __forceinline__ double rop(double a, double b) {
  if (OP == R_SUM) return a + b;
  if (OP == R_MAX) return (a > b || a != a) ? a : b;   // propagates NaN
  return (a < b || a != a) ? a : b;
}

template <int OP>
__device__ __forceinline__ float ropf(float a, float b) {
  if (OP == R_SUM) return a + b;
  if (OP == R_MAX) return (a > b || a != a) ? a : b;   // propagates NaN
  return (a < b || a != a) ? a : b;
}

// Block-wide reduction of four floats (all threads get the results).  FP32 on purpose:
// the FP64 pipe of this part is a small fraction of the FP32 one, and the reduced
// quantities (norms for the stopping test, μ, step lengths) need no more than FP32.
template <int O0, int O1, int O2, int O3>
__device__ __forceinline__ void block_reduce4f(float (&v)[4], float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v[0] = ropf<O0>(v[0], __shfl_xor_sync(0xffffffffu, v[0], off));
    v[1] = ropf<O1>(v[1], __shfl_xor_sync(0xffffffffu, v[1], off));
    v[2] = ropf<O2>(v[2], __shfl_xor_sync(0xffffffffu, v[2], off));
    v[3] = ropf<O3>(v[3], __shfl_xor_sync(0xffffffffu, v[3], off));
  }
  if (lane == 0) {
    red[4 * w + 0] = v[0];
    red[4 * w + 1] = v[1];
    red[4 * w + 2] = v[2];
    red[4 * w + 3] = v[3];
  }
  __syncthreads();
  float r0 = red[0], r1 = red[1], r2 = red[2], r3 = red[3];
#pragma unroll
  for (int i = 1; i < NWARPS; ++i) {
    r0 = ropf<O0>(r0, red[4 * i + 0]);
    r1 = ropf<O1>(r1, red[4 * i + 1]);
    r2 = ropf<O2>(r2, red[4 * i + 2]);
    r3 = ropf<O3>(r3, red[4 * i + 3]);
  }
  v[0] = r0; v[1] = r1; v[2] = r2; v[3] = r3;
  __syncthreads();
}

// Block-wide maximum of eight floats (NaN-propagating; all threads get the results); `red`
// holds 8·NWARPS floats.
__device__ __forceinline__ void block_reduce8f_max(float (&v)[8], float* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1)
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ropf<R_MAX>(v[k], __shfl_xor_sync(0xffffffffu, v[k], off));
  if (lane == 0)
#pragma unroll
    for (int k = 0; k < 8; ++k) red[8 * w + k] = v[k];
  __syncthreads();
#pragma unroll
  for (int k = 0; k < 8; ++k) v[k] = red[k];
#pragma unroll
  for (int i = 1; i < NWARPS; ++i)
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = ropf<R_MAX>(v[k], red[8 * i + k]);
  __syncthreads();
}

template <int O0, int O1, int O2, int O3>
__device__ __forceinline__ void block_reduce4(double (&v)[4], double* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    v[0] = rop<O0>(v[0], __shfl_xor_sync(0xffffffffu, v[0], off));
    v[1] = rop<O1>(v[1], __shfl_xor_sync(0xffffffffu, v[1], off));
    v[2] = rop<O2>(v[2], __shfl_xor_sync(0xffffffffu, v[2], off));
    v[3] = rop<O3>(v[3], __shfl_xor_sync(0xffffffffu, v[3], off));
  }
  if (lane == 0) {
    red[4 * w + 0] = v[0];
    red[4 * w + 1] = v[1];
    red[4 * w + 2] = v[2];
    red[4 * w + 3] = v[3];
  }
  __syncthreads();
  double r0 = red[0], r1 = red[1], r2 = red[2], r3 = red[3];
#pragma unroll
  for (int i = 1; i < NWARPS; ++i) {
    r0 = rop<O0>(r0, red[4 * i + 0]);
    r1 = rop<O1>(r1, red[4 * i + 1]);
    r2 = rop<O2>(r2, red[4 * i + 2]);
    r3 = rop<O3>(r3, red[4 * i + 3]);
  }
  v[0] = r0; v[1] = r1; v[2] = r2; v[3] = r3;
  __syncthreads();
}

// ------------------------------------------------------------------ matrix-vector products
enum : int { TRI_ALL = 0, TRI_LOWER = 1, TRI_SUPPER = 2 };

// y_r = Σ_c M[r·ld + c]·x[c] for r < rows, over all c (TRI_ALL), c ≤ r (TRI_LOWER) or
// c > r (TRI_SUPPER); GL lanes per row.  Calls epi(r, y_r) once per row; the caller
// synchronises before reading the results.
template <int GL, typename T, typename F>
__device__ __forceinline__ void mv_rows(const T* M, int ld, int rows, int cols, int tri,
                                        const T* x, F epi) {
  const int tid = threadIdx.x;
  const int g = tid / GL, gl = tid % GL;
  constexpr int NG = NTHREADS / GL;
  for (int r0 = 0; r0 < rows; r0 += NG) {
    const int r = r0 + g;
    T acc0 = T(0), acc1 = T(0);
    if (r < rows) {
      const int cend = tri == TRI_LOWER ? min(cols, r + 1) : cols;
      const T* row = M + (size_t)r * ld;
      int c = (tri == TRI_SUPPER ? r + 1 : 0) + gl;
      for (; c + GL < cend; c += 2 * GL) {
        acc0 = fma(row[c], x[c], acc0);
        acc1 = fma(row[c + GL], x[c + GL], acc1);
      }
      if (c < cend) acc0 = fma(row[c], x[c], acc0);
    }
    T acc = acc0 + acc1;
#pragma unroll
    for (int off = GL / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
    if (r < rows && gl == 0) epi(r, acc);
  }
}

// y_r = Σ_c M[r·ld + c]·x[c] for r < rows and all c < cols, when M's rows and x start on
// 16-byte boundaries and cols is a whole number of 16-byte vectors (cols ≤ 8·GL vectors):
// lane gl of a row's GL lanes keeps x's vectors gl, gl+GL, ... in registers for every row, so
// each row is read once from shared memory and x once per call.  Returns false (doing
// nothing) when those conditions do not hold; the caller then uses mv_rows.
template <int GL, typename T, typename F>
__device__ __forceinline__ bool mv_rows_xreg(const T* M, int ld, int rows, int cols, const T* x,
                                             F epi) {
  constexpr int W = 16 / sizeof(T), XV = 8;
  const int nv = cols / W;
  if (cols % W != 0 || ld % W != 0 || nv > XV * GL ||
      ((((uintptr_t)M) | ((uintptr_t)x)) % 16) != 0)
    return false;
  const int tid = threadIdx.x;
  const int g = tid / GL, gl = tid % GL;
  constexpr int NG = NTHREADS / GL;
  T xr[XV][W];
#pragma unroll
  for (int k = 0; k < XV; ++k) {
    const int v = gl + k * GL;
    if (v < nv) {
      if constexpr (W == 4) {
        const float4 q = *reinterpret_cast<const float4*>(x + v * W);
        xr[k][0] = q.x; xr[k][1] = q.y; xr[k][2] = q.z; xr[k][3] = q.w;
      } else {
        const double2 q = *reinterpret_cast<const double2*>(x + v * W);
        xr[k][0] = q.x; xr[k][1] = q.y;
      }
    } else {
#pragma unroll
      for (int e = 0; e < W; ++e) xr[k][e] = T(0);
    }
  }
  for (int r0 = 0; r0 < rows; r0 += NG) {
    const int r = r0 + g;
    T acc[2] = {T(0), T(0)};
    if (r < rows) {
      const T* row = M + (size_t)r * ld;
#pragma unroll
      for (int k = 0; k < XV; ++k) {
        const int v = gl + k * GL;
        if (v < nv) {
          T a[W];
          if constexpr (W == 4) {
            const float4 q = *reinterpret_cast<const float4*>(row + v * W);
            a[0] = q.x; a[1] = q.y; a[2] = q.z; a[3] = q.w;
          } else {
            const double2 q = *reinterpret_cast<const double2*>(row + v * W);
            a[0] = q.x; a[1] = q.y;
          }
#pragma unroll
          for (int e = 0; e < W; ++e) acc[k & 1] = fma(a[e], xr[k][e], acc[k & 1]);
        }
      }
    }
    T s = acc[0] + acc[1];
#pragma unroll
    for (int off = GL / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
    if (r < rows && gl == 0) epi(r, s);
  }
  return true;
}

// y_c = Σ_r M[r·ld + c]·x[r] for c < cols, over all r (TRI_ALL), r ≥ c (TRI_LOWER) or
// r < c (TRI_SUPPER).  Row ranges are split over the threads that share a column; partial
// sums meet in `scr` (NTHREADS entries).  Ends with a barrier, so epi's writes are visible
// on return.
template <typename T, typename F>
__device__ __forceinline__ void mv_cols(const T* M, int ld, int rows, int cols, int tri,
                                        const T* x, T* scr, F epi, int cap = NTHREADS) {
  (void)cap;
  const int tid = threadIdx.x;
  if (cols <= 0) return;
  if (cols > NTHREADS / 2) {
    for (int c = tid; c < cols; c += NTHREADS) {
      T a0 = T(0), a1 = T(0);
      int r = tri == TRI_LOWER ? c : 0;
      const int rend = tri == TRI_SUPPER ? min(rows, c) : rows;
      for (; r + 1 < rend; r += 2) {
        a0 = fma(M[(size_t)r * ld + c], x[r], a0);
        a1 = fma(M[(size_t)(r + 1) * ld + c], x[r + 1], a1);
      }
      if (r < rend) a0 = fma(M[(size_t)r * ld + c], x[r], a0);
      epi(c, a0 + a1);
    }
    __syncthreads();
    return;
  }
  const int nparts = NTHREADS / cols;
  const int c = tid % cols, part = tid / cols;
  if (part < nparts) {
    const int chunk = (rows + nparts - 1) / nparts;
    int r = part * chunk;
    int r1 = min(rows, r + chunk);
    if (tri == TRI_LOWER && r < c) r = c;
    if (tri == TRI_SUPPER && r1 > c) r1 = c;
    T a0 = T(0), a1 = T(0);
    for (; r + 1 < r1; r += 2) {
      a0 = fma(M[(size_t)r * ld + c], x[r], a0);
      a1 = fma(M[(size_t)(r + 1) * ld + c], x[r + 1], a1);
    }
    if (r < r1) a0 = fma(M[(size_t)r * ld + c], x[r], a0);
    scr[part * cols + c] = a0 + a1;
  }
  __syncthreads();
  if (tid < cols) {
    T s = T(0);
    for (int q = 0; q < nparts; ++q) s += scr[q * cols + tid];
    epi(tid, s);
  }
  __syncthreads();
}

// Four consecutive elements from global memory, read-only path (16-byte aligned).
__device__ __forceinline__ void ldg4(float (&v)[4], const float* p) {
  const float4 t = __ldg(reinterpret_cast<const float4*>(p));
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ldg4(double (&v)[4], const double* p) {
  const double2 a = __ldg(reinterpret_cast<const double2*>(p));
  const double2 b = __ldg(reinterpret_cast<const double2*>(p) + 1);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// Four consecutive elements of a row, columns c0..c0+3 clipped to n: one 16-byte load when
// the address allows it, scalar loads otherwise.  The values (and so every result below) do
// not depend on which form is taken.
template <typename T>
__device__ __forceinline__ void ldg4_row(T (&v)[4], const T* row, int c0, int n, bool vec) {
  if (vec && c0 + 4 <= n) {
    ldg4(v, row + c0);
  } else {
#pragma unroll
    for (int c = 0; c < 4; ++c) v[c] = (c0 + c < n) ? __ldg(row + c0 + c) : T(0);
  }
}

// The leading part of a split value: the FP32 rounding for T = float, the value itself for
// T = double.
__device__ __forceinline__ float split_hi(float2 v) { return v.x; }
__device__ __forceinline__ double split_hi(double v) { return v; }

// Row pass of the KKT operator, G x_z and A x_z, with x_z held in registers: lane gl of a row's
// GL = 8 lanes keeps quads gl, gl+8, gl+16, gl+24 of x_z, so each element of a row costs one
// load and one accumulation.  For 8 < ⌈n/4⌉ ≤ 32 (9 ≤ n ≤ 128); returns false, doing
// nothing, otherwise.  FAST: plain T accumulation; else the double-float Acc.  The row loop
// is uniform over the block, as the shuffles need.
template <bool FAST, typename T, typename FL, typename FN>
__device__ __forceinline__ bool kkt_rows_xreg(int n, int p, int m, const T* __restrict__ G,
                                              const T* __restrict__ A,
                                              const typename Split<T>::V* xv, bool vec,
                                              FL add_l, FN add_n, double* out_l,
                                              double* out_n) {
  using V = typename Split<T>::V;
  constexpr int GL = 8, NG = NTHREADS / GL, XQ = 4;
  const int nq = (n + 3) / 4;
  if (nq <= 8 || nq > GL * XQ) return false;
  const int tid = threadIdx.x, g = tid / GL, gl = tid % GL;
  V xr[XQ][4];
#pragma unroll
  for (int u = 0; u < XQ; ++u)
#pragma unroll
    for (int c = 0; c < 4; ++c) {
      const int j = 4 * (gl + u * GL) + c;
      xr[u][c] = j < n ? xv[j] : V{};
    }
  for (int r0 = 0; r0 < p + m; r0 += NG) {
    const int r = r0 + g;
    const bool live = r < p + m;
    const T* rowv = !live ? G : (r < p) ? G + (size_t)r * n : A + (size_t)(r - p) * n;
    T av[XQ][4];
#pragma unroll
    for (int u = 0; u < XQ; ++u) {
      const int q = gl + u * GL;
      if (live && q < nq) {
        ldg4_row(av[u], rowv, 4 * q, n, vec);
      } else {
#pragma unroll
        for (int c = 0; c < 4; ++c) av[u][c] = T(0);
      }
    }
    double v;
    if constexpr (FAST) {
      T a0 = T(0), a1 = T(0);
#pragma unroll
      for (int u = 0; u < XQ; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          if (c & 1) a1 = fma(av[u][c], split_hi(xr[u][c]), a1);
          else a0 = fma(av[u][c], split_hi(xr[u][c]), a0);
        }
      T s = a0 + a1;
#pragma unroll
      for (int off = GL / 2; off > 0; off >>= 1) s += __shfl_xor_sync(0xffffffffu, s, off);
      v = (double)s;
    } else {
      Acc<T> acc;
#pragma unroll
      for (int u = 0; u < XQ; ++u)
#pragma unroll
        for (int c = 0; c < 4; ++c) acc.add(av[u][c], xr[u][c]);
#pragma unroll
      for (int off = GL / 2; off > 0; off >>= 1) acc.shfl_merge(off);
      v = acc.value();
    }
    if (live && gl == 0) {
      if (r < p) out_l[r] = v + add_l(r);
      else out_n[r - p] = v + add_n(r - p);
    }
  }
  return true;
}

// FP64-accurate application of the (unreduced, slack-eliminated) KKT operator:
//   out_z = Q x_z + Gᵀ x_λ + Aᵀ x_ν + add_z,  out_λ = G x_z + add_λ,  out_ν = A x_z + add_ν.
// x = [x_z; x_λ; x_ν] is given split (FP32 hi/lo pairs for T = float).  Q is symmetric, so
// Q x_z is formed column-wise together with Gᵀx_λ and Aᵀx_ν from one pass over the rows of
// [Q; G; A] (inputs read from global memory, where they stay L2-resident); G x_z and A x_z
// come from a row pass.  Work is split into quads of four columns; each thread reads a quad
// with one 16-byte load when n is a multiple of 4 and the rows are aligned, else with
// scalar loads, in the same order either way.  Partial sums stay double-float until one
// conversion per output element.  `scr` holds kscr ≥ NTHREADS accumulators.  Ends with a
// barrier.
template <typename T, typename FZ, typename FL, typename FN>
__device__ __forceinline__ void kkt_apply(int n, int p, int m, const T* __restrict__ Q,
                                          const T* __restrict__ G, const T* __restrict__ A,
                                          const typename Split<T>::V* xv, Acc<T>* scr, int kscr,
                                          FZ add_z, FL add_l, FN add_n,
                                          double* out_z, double* out_l, double* out_n) {
  using V = typename Split<T>::V;
  const int tid = threadIdx.x;
  const int R = n + p + m;
  auto rowp = [&](int r) -> const T* {
    return r < n ? Q + (size_t)r * n : (r < n + p ? G + (size_t)(r - n) * n : A + (size_t)(r - n - p) * n);
  };
  const bool vec = (n % 4 == 0) &&
      ((((uintptr_t)Q) | ((uintptr_t)G) | ((uintptr_t)A)) % (4 * sizeof(T)) == 0);
  const int nq = (n + 3) / 4;
  const int nparts = max(1, min(NTHREADS / nq, kscr / (4 * nq)));
  // Column pass: thread (jq, part) sums rows [r0, r1) of columns 4jq .. 4jq+3.
  for (int t = tid; t < nq * nparts; t += NTHREADS) {
    const int jq = t % nq, part = t / nq;
    const int chunk = (R + nparts - 1) / nparts;
    const int r0 = part * chunk, r1 = min(R, r0 + chunk);
    Acc<T> acc[4];
    int r = r0;
    for (; r + 4 <= r1; r += 4) {
      T av[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldg4_row(av[u], rowp(r + u), 4 * jq, n, vec);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const V x = xv[r + u];
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c].add(av[u][c], x);
      }
    }
    for (; r < r1; ++r) {
      T av[4];
      ldg4_row(av, rowp(r), 4 * jq, n, vec);
      const V x = xv[r];
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c].add(av[c], x);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) scr[part * 4 * nq + 4 * jq + c] = acc[c];
  }
  // Row pass: G x_z and A x_z.  For 9 ≤ n ≤ 128 with x_z in registers (kkt_rows_xreg); else
  // GL lanes per row (lane gl takes quads gl, gl+GL, ...), two rows per lane group at a time
  // so that both rows' loads are in flight together.
  if (!kkt_rows_xreg<false, T>(n, p, m, G, A, xv, vec, add_l, add_n, out_l, out_n)) {
    constexpr int GL = 8, NG = NTHREADS / GL, QB = 4;
    const int g = tid / GL, gl = tid % GL;
    for (int r0 = 0; r0 < p + m; r0 += 2 * NG) {
      const int rr[2] = {r0 + g, r0 + NG + g};
      const T* rowv[2];
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
        const int r = rr[h2];
        rowv[h2] = (r < p) ? G + (size_t)r * n : A + (size_t)(r - p) * n;
      }
      Acc<T> acc[2];
      for (int qb0 = 0; qb0 < nq; qb0 += GL * QB) {
        T av[2][QB][4];
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
          for (int u = 0; u < QB; ++u) {
            const int q = qb0 + gl + u * GL;
            if (rr[h2] < p + m && q < nq) {
              ldg4_row(av[h2][u], rowv[h2], 4 * q, n, vec);
            } else {
#pragma unroll
              for (int c = 0; c < 4; ++c) av[h2][u][c] = T(0);
            }
          }
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2)
#pragma unroll
          for (int u = 0; u < QB; ++u) {
            const int q = qb0 + gl + u * GL;
            if (rr[h2] < p + m && q < nq) {
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (4 * q + c < n) acc[h2].add(av[h2][u][c], xv[4 * q + c]);
            }
          }
      }
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
        for (int off = GL / 2; off > 0; off >>= 1) acc[h2].shfl_merge(off);
        const int r = rr[h2];
        if (r < p + m && gl == 0) {
          const double v = acc[h2].value();
          if (r < p) out_l[r] = v + add_l(r);
          else out_n[r - p] = v + add_n(r - p);
        }
      }
    }
  }
  __syncthreads();
  for (int j = tid; j < n; j += NTHREADS) {
    Acc<T> acc = scr[j];
    for (int q = 1; q < nparts; ++q) acc.merge(scr[q * 4 * nq + j]);
    out_z[j] = acc.value() + add_z(j);
  }
  __syncthreads();
}

// kkt_apply in plain T arithmetic (one FMA per matrix element, x rounded to T): the same
// operator and the same quad/partial-sum organisation, with an error of order
// n·2⁻²⁴·Σ|terms| for T = float instead of 2⁻⁴⁸.  The interior point loop uses it while μ
// is far above its tolerance, where that error is far below what the step needs.
template <typename T, typename FZ, typename FL, typename FN>
__device__ __forceinline__ void kkt_apply_fast(int n, int p, int m, const T* __restrict__ Q,
                                               const T* __restrict__ G, const T* __restrict__ A,
                                               const typename Split<T>::V* xv, T* scr, int kscr,
                                               FZ add_z, FL add_l, FN add_n,
                                               double* out_z, double* out_l, double* out_n) {
  const int tid = threadIdx.x;
  const int R = n + p + m;
  auto rowp = [&](int r) -> const T* {
    return r < n ? Q + (size_t)r * n : (r < n + p ? G + (size_t)(r - n) * n : A + (size_t)(r - n - p) * n);
  };
  const bool vec = (n % 4 == 0) &&
      ((((uintptr_t)Q) | ((uintptr_t)G) | ((uintptr_t)A)) % (4 * sizeof(T)) == 0);
  const int nq = (n + 3) / 4;
  const int nparts = max(1, min(NTHREADS / nq, kscr / (4 * nq)));
  for (int t = tid; t < nq * nparts; t += NTHREADS) {
    const int jq = t % nq, part = t / nq;
    const int chunk = (R + nparts - 1) / nparts;
    const int r0 = part * chunk, r1 = min(R, r0 + chunk);
    T acc[4] = {T(0), T(0), T(0), T(0)};
    int r = r0;
    for (; r + 4 <= r1; r += 4) {
      T av[4][4];
#pragma unroll
      for (int u = 0; u < 4; ++u) ldg4_row(av[u], rowp(r + u), 4 * jq, n, vec);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const T x = split_hi(xv[r + u]);
#pragma unroll
        for (int c = 0; c < 4; ++c) acc[c] = fma(av[u][c], x, acc[c]);
      }
    }
    for (; r < r1; ++r) {
      T av[4];
      ldg4_row(av, rowp(r), 4 * jq, n, vec);
      const T x = split_hi(xv[r]);
#pragma unroll
      for (int c = 0; c < 4; ++c) acc[c] = fma(av[c], x, acc[c]);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c) scr[part * 4 * nq + 4 * jq + c] = acc[c];
  }
  if (!kkt_rows_xreg<true, T>(n, p, m, G, A, xv, vec, add_l, add_n, out_l, out_n)) {
    constexpr int GL = 8, NG = NTHREADS / GL, QB = 4;
    const int g = tid / GL, gl = tid % GL;
    for (int r0 = 0; r0 < p + m; r0 += 2 * NG) {
      const int rr[2] = {r0 + g, r0 + NG + g};
      T acc[2] = {T(0), T(0)};
      for (int qb0 = 0; qb0 < nq; qb0 += GL * QB) {
#pragma unroll
        for (int h2 = 0; h2 < 2; ++h2) {
          const int rw = rr[h2];
          const T* rowv = (rw < p) ? G + (size_t)rw * n : A + (size_t)(rw - p) * n;
#pragma unroll
          for (int u = 0; u < QB; ++u) {
            const int q = qb0 + gl + u * GL;
            if (rw < p + m && q < nq) {
              T av[4];
              ldg4_row(av, rowv, 4 * q, n, vec);
#pragma unroll
              for (int c = 0; c < 4; ++c)
                if (4 * q + c < n) acc[h2] = fma(av[c], split_hi(xv[4 * q + c]), acc[h2]);
            }
          }
        }
      }
#pragma unroll
      for (int h2 = 0; h2 < 2; ++h2) {
#pragma unroll
        for (int off = GL / 2; off > 0; off >>= 1) acc[h2] += __shfl_xor_sync(0xffffffffu, acc[h2], off);
        const int rw = rr[h2];
        if (rw < p + m && gl == 0) {
          if (rw < p) out_l[rw] = (double)acc[h2] + add_l(rw);
          else out_n[rw - p] = (double)acc[h2] + add_n(rw - p);
        }
      }
    }
  }
  __syncthreads();
  for (int j = tid; j < n; j += NTHREADS) {
    T a = scr[j];
    for (int q = 1; q < nparts; ++q) a += scr[q * 4 * nq + j];
    out_z[j] = (double)a + add_z(j);
  }
  __syncthreads();
}

// ------------------------------------------------------------------ register tiles
// Lower-triangular tiling of an N×N symmetric matrix by 4×4 tiles; linear tile t maps to
// tile row I = ⌊(√(8t+1) − 1)/2⌋ and tile column J = t − I(I+1)/2.
__device__ __forceinline__ void tile_of(int t, int& I, int& J) {
  int i = (int)((sqrtf(8.0f * (float)t + 1.0f) - 1.0f) * 0.5f);
  while ((i + 1) * (i + 2) / 2 <= t) ++i;
  while (i * (i + 1) / 2 > t) --i;
  I = i;
  J = t - i * (i + 1) / 2;
}

// Column-major enumeration of the lower tiles of an NT×NT tile grid: tile column J holds
// tiles (J..NT−1, J) at consecutive indices starting at J·NT − J(J−1)/2.
__device__ __forceinline__ void tile_of_colmajor(int t, int NT, int& I, int& J) {
  int j = 0, off = 0;
  while (j < NT && off + (NT - j) <= t) { off += NT - j; ++j; }
  J = j;
  I = j + (t - off);
}

template <typename T>
__device__ __forceinline__ T sel4(T a0, T a1, T a2, T a3, int k) {
  return k == 0 ? a0 : (k == 1 ? a1 : (k == 2 ? a2 : a3));
}

// Element (i, j) of the symmetric matrix [[Q̃, Aᵀ, Gᵀ], [A, 0, 0], [G, 0, 0]] whose first
// m1 = nz + neq pivots are swept (rows ordered z, dummies, ν, λ; Q̃ = (Q + δI) ⊕ I on the
// dummy variables, δ = 0 unless Q is only positive semidefinite).  Zero outside N×N.
template <typename T>
__device__ __forceinline__ T k3_elem(int n, int nz, int m1, int N, const T* Q, const T* A,
                                     const T* G, int i, int j, T delta) {
  if (i >= N || j >= N) return T(0);
  if (i < j) { const int t = i; i = j; j = t; }
  if (i < n) return (i == j) ? Q[(size_t)i * n + j] + delta : Q[(size_t)i * n + j];
  if (i < nz) return (i == j) ? T(1) : T(0);
  if (j >= n) return T(0);
  if (i < m1) return A[(size_t)(i - nz) * n + j];
  return G[(size_t)(i - m1) * n + j];
}

// 4×4 tile helpers (row-major 16-element arrays, compile-time indices only).
template <typename T>
__device__ __forceinline__ void ld16(T (&d)[16], const T* src) {
#pragma unroll
  for (int e = 0; e < 16; ++e) d[e] = src[e];
}
template <typename T>
__device__ __forceinline__ void st16(T* dst, const T (&v)[16]) {
#pragma unroll
  for (int e = 0; e < 16; ++e) dst[e] = v[e];
}

// Four consecutive elements (16-byte aligned for float, 32-byte for double).
__device__ __forceinline__ void ld4(float (&v)[4], const float* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(double (&v)[4], const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}
__device__ __forceinline__ void st4(float* p, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double* p, double a, double b, double c, double d) {
  reinterpret_cast<double2*>(p)[0] = make_double2(a, b);
  reinterpret_cast<double2*>(p)[1] = make_double2(c, d);
}

// Panel buffers hold 4×4 blocks column-major by pivot: element (row r of block B, pivot
// column q) lives at q·ld + 4B + r with ld = 4·NT, so the four rows of a block for one
// pivot are one aligned vector and neighbouring blocks are neighbouring vectors (no shared
// memory bank conflicts when threads handle neighbouring blocks).
template <typename T>
__device__ __forceinline__ void ld_panel(T (&v)[16], const T* buf, int ld, int B) {
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    T t[4];
    ld4(t, buf + q * ld + 4 * B);
#pragma unroll
    for (int r = 0; r < 4; ++r) v[r * 4 + q] = t[r];
  }
}
template <typename T>
__device__ __forceinline__ void st_panel(T* buf, int ld, int B, const T (&v)[16]) {
#pragma unroll
  for (int q = 0; q < 4; ++q) st4(buf + q * ld + 4 * B, v[0 * 4 + q], v[1 * 4 + q], v[2 * 4 + q], v[3 * 4 + q]);
}

// Blocked symmetric Gauss-Jordan sweep over the pivots 0 .. m1−1 (m1 a multiple of 4) of
// the matrix above, held in registers as 4×4 tiles.  SWEEP(k) is
//   d = a_kk;  a_ij ← a_ij − a_ik a_kj / d (i, j ≠ k);  a_ik ← a_ik / d;  a_kk ← −1/d.
// The four pivots of tile K are applied with two barriers: one thread sweeps the pivot tile
// itself (checking each pivot's sign: positive for z rows since Q ≻ 0, negative for ν rows
// since A has full row rank) and publishes, for each pivot k, the row r_k = (pivot-tile
// row k before pivot k)/d_k; the owners of block row/column K replay the four scalar
// sweeps on each of their panel rows, which yields the pivot columns ĉ_k seen by each pivot
// and the new panel values, and publish ĉ and ĉ·D⁻¹; every other tile then takes the
// accumulated update A_IJ −= Σ_k ĉ_Ik ĉ_Jk / d_k.  This is the scalar sweep's arithmetic,
// so the explicit inverse of the pivot tile is never used.  Afterwards the top-left block is
// −K11⁻¹ = −S, the bottom-left block is RE = [G 0]·S and the bottom-right block is −M.
// Writes S and RE to SR (rows 0..m1−1 = S, m1.. = RE, leading dimension ldS), M's strict
// upper triangle to Mb and diag(M) to dM.  Returns false on every thread if a pivot has the
// wrong sign or is not finite.
template <typename T, int SW>
__device__ __noinline__ bool sweep_setup(int n, int p, int m, const T* __restrict__ Q,
                                         const T* __restrict__ A, const T* __restrict__ G,
                                         T* SR, int ldS, T* Mb, int ldM, T* dM, T* cb,
                                         T delta, T zthr) {
  const int tid = threadIdx.x;
  const int nz = padded_nz(n, m), m1 = nz + m, N = m1 + p;
  const int NT = (N + 3) >> 2, ntiles = NT * (NT + 1) / 2, KB = m1 >> 2;
  if (ntiles > SW * NTHREADS) return false;   // register tiles too few (host plans avoid it)
  // cb layout per parity: Ĉ panel [16·NT], Ĉ·D⁻¹ panel [16·NT], pivot rows R [16]; flags.
  const int pstride = 32 * NT + 16;
  int* flag = reinterpret_cast<int*>(cb + 2 * pstride);
  T a[SW][16];
  int tI[SW], tJ[SW];
#pragma unroll
  for (int s = 0; s < SW; ++s) {
    const int t = tid + s * NTHREADS;
    int I = -1, J = 0;
    if (t < ntiles) tile_of(t, I, J);
    tI[s] = I;
    tJ[s] = J;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int c = 0; c < 4; ++c)
        a[s][r * 4 + c] =
            (I >= 0) ? k3_elem(n, nz, m1, N, Q, A, G, 4 * I + r, 4 * J + c, delta) : T(0);
  }
  for (int K = 0; K < KB; ++K) {
    T* Cb = cb + (K & 1) * pstride;
    T* Pb = Cb + 16 * NT;
    T* Rb = Pb + 16 * NT;
    // Phase A: the four scalar sweeps on the pivot tile; publish r_k.
#pragma unroll
    for (int s = 0; s < SW; ++s) {
      if (tI[s] == K && tJ[s] == K) {
        T w[16];
#pragma unroll
        for (int e = 0; e < 16; ++e) w[e] = a[s][e];
        bool good = true;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
          const T d = w[k * 4 + k];
          const int kk = 4 * K + k;
          // z pivots must clear zthr (a singular Q shows as a pivot at rounding level), dummy
          // pivots 0, ν pivots must be negative (A of full row rank)
          good = good && isfinite(d) && (kk < n ? d > zthr : (kk < nz ? d > T(0) : d < T(0)));
          const T dinv = T(1) / d;
#pragma unroll
          for (int q = 0; q < 4; ++q) Rb[k * 4 + q] = (q == k) ? dinv : w[k * 4 + q] * dinv;
#pragma unroll
          for (int r = 0; r < 4; ++r)
#pragma unroll
            for (int c = 0; c < 4; ++c)
              if (r != k && c != k) w[r * 4 + c] = fma(-w[r * 4 + k] * dinv, w[k * 4 + c], w[r * 4 + c]);
#pragma unroll
          for (int r = 0; r < 4; ++r)
            if (r != k) { w[r * 4 + k] *= dinv; w[k * 4 + r] *= dinv; }
          w[k * 4 + k] = -dinv;
        }
#pragma unroll
        for (int e = 0; e < 16; ++e) a[s][e] = w[e];
        flag[K & 1] = good ? 0 : 1;
      }
    }
    __syncthreads();
    if (flag[K & 1]) return false;
    // Phase B: replay the four sweeps on every panel row (rows of blocks I ≠ K).
    {
      T R[16];
      ld16(R, Rb);
#pragma unroll
      for (int s = 0; s < SW; ++s) {
        const int I = tI[s], J = tJ[s];
        if (I < 0 || (I != K && J != K) || (I == K && J == K)) continue;
        const int B = (J == K) ? I : J;   // block index of the panel rows held by this tile
        T ch[16], cd[16];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
          T v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) v[q] = (J == K) ? a[s][r * 4 + q] : a[s][q * 4 + r];
#pragma unroll
          for (int k = 0; k < 4; ++k) {
            const T c = v[k];
            ch[r * 4 + k] = c;
            cd[r * 4 + k] = c * R[k * 4 + k];
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (q != k) v[q] = fma(-c, R[k * 4 + q], v[q]);
            v[k] = c * R[k * 4 + k];
          }
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            if (J == K) a[s][r * 4 + q] = v[q];
            else a[s][q * 4 + r] = v[q];
          }
        }
        st_panel(Cb, 4 * NT, B, ch);
        st_panel(Pb, 4 * NT, B, cd);
      }
    }
    __syncthreads();
    // Phase C: A_IJ −= Σ_k (ĉ_Ik / d_k) ĉ_Jk for I, J ≠ K.
#pragma unroll
    for (int s = 0; s < SW; ++s) {
      const int I = tI[s], J = tJ[s];
      if (I < 0 || I == K || J == K) continue;
      T Pi[16], Cj[16];
      ld_panel(Pi, Pb, 4 * NT, I);
      ld_panel(Cj, Cb, 4 * NT, J);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T acc = a[s][r * 4 + c];
#pragma unroll
          for (int q = 0; q < 4; ++q) acc = fma(-Pi[r * 4 + q], Cj[c * 4 + q], acc);
          a[s][r * 4 + c] = acc;
        }
    }
  }
#pragma unroll
  for (int s = 0; s < SW; ++s) {
    const int I = tI[s], J = tJ[s];
    if (I < 0) continue;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * I + r, j = 4 * J + q;
        if (i >= N || j > i) continue;
        const T v = a[s][r * 4 + q];
        if (i < m1) {
          SR[(size_t)i * ldS + j] = -v;
          SR[(size_t)j * ldS + i] = -v;
        } else if (j < m1) {
          SR[(size_t)i * ldS + j] = v;
        } else if (i == j) {
          dM[i - m1] = -v;
        } else {
          Mb[(size_t)(j - m1) * ldM + (i - m1)] = -v;
        }
      }
  }
  return true;
}

// Blocked Cholesky factorisation M + D(dsh) = L Lᵀ in 4×4 register tiles (right-looking over
// 4-column steps, two barriers per step).  M comes from the strict upper triangle of Mb plus
// dM.  The factor is left in the lower triangle of Mb in the blocked form blk_solve applies:
// L's tiles below the NB×NB diagonal blocks (NB = chol_nb, 32 in FP32 and 16 in FP64) as they
// are, and on each diagonal block its inverse L_BB⁻¹ (lower triangular).  Step K:
//   A: one thread factors the diagonal tile, L_KK = chol(A_KK), and inverts it, V_K = L_KK⁻¹;
//   B: owners form the panel L_IK = A_IK V_Kᵀ (I > K) and the finished block row of the
//      block inverse, X_KJ ← V_K X_KJ (J in K's diagonal block), and publish both;
//   C: A_IJ −= L_IK L_JKᵀ (I ≥ J > K) and, inside K's diagonal block, X_IJ −= L_IK X_KJ.
// The inverse tiles X are owned by threads counted down from the last one, so on most sizes
// they fall on threads without a trailing tile and cost no extra pass.  The owner of the next
// diagonal tile factors it right after its own update.  Padding rows/columns beyond p are the
// identity and never couple to the real ones.  Returns false on every thread if a pivot is
// not positive or not finite.
template <typename T, int CH, bool FULLX = false>
__device__ __noinline__ bool chol_blk(int p, T* Mb, int ldM, const T* dM, const T* dsh, T* cb) {
  // FULLX: the "diagonal block" is the whole matrix, so X = L⁻¹ in full replaces L.
  const int NT = (p + 3) >> 2, ntiles = NT * (NT + 1) / 2;
  const int TB = FULLX ? NT : chol_nb((int)sizeof(T)) / 4;   // tiles along a diagonal block
  const int TBT = TB * (TB + 1) / 2;                          // tiles in a full block's lower triangle
  const int tid = threadIdx.x;
  const int nfull = NT / TB, tlast = NT - nfull * TB;
  const int nxt = nfull * TBT + tlast * (tlast + 1) / 2;
  if (ntiles > CH * NTHREADS || nxt > CH * NTHREADS) return false;   // host plans avoid it
  // cb layout per parity: L panel [16·NT], X block row [16·NT], V_K [16]; flags after both.
  const int pstride = 32 * NT + 16;
  int* flag = reinterpret_cast<int*>(cb + 2 * pstride);
  T a[CH][16], x[CH][16];
  int tI[CH], tJ[CH], xI[CH], xJ[CH];
#pragma unroll
  for (int s = 0; s < CH; ++s) {
    const int t = tid + s * NTHREADS;
    int I = -1, J = 0, XI = -1, XJ = 0;
    if (t < ntiles) tile_of_colmajor(t, NT, I, J);
    const int u = (NTHREADS - 1 - tid) + s * NTHREADS;   // inverse tiles from the top thread
    if (u < nxt) {
      const int b = u / TBT;
      int i, j;
      tile_of(u - b * TBT, i, j);
      XI = b * TB + i;
      XJ = b * TB + j;
    }
    tI[s] = I;
    tJ[s] = J;
    xI[s] = XI;
    xJ[s] = XJ;
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = 4 * I + r, j = 4 * J + q;
        T av = T(0);
        if (I >= 0) {
          if (i >= p || j >= p) {
            av = (i == j) ? T(1) : T(0);
          } else if (i == j) {
            av = dM[i] + dsh[i];
          } else {
            av = Mb[(size_t)min(i, j) * ldM + max(i, j)];
          }
        }
        a[s][r * 4 + q] = av;
        x[s][r * 4 + q] = (XI >= 0 && 4 * XI + r == 4 * XJ + q) ? T(1) : T(0);
      }
  }
  for (int K = 0; K < NT; ++K) {
    T* Lb = cb + (K & 1) * pstride;
    T* Xb = Lb + 16 * NT;
    T* Vb = Xb + 16 * NT;
    // Phase A: Cholesky of the diagonal tile and the inverse of its factor.
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      if (tI[s] == K && tJ[s] == K) {
        T l[16], li[4];
        bool good = true;
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          T d = a[s][c * 4 + c];
#pragma unroll
          for (int q = 0; q < c; ++q) d = fma(-l[c * 4 + q], l[c * 4 + q], d);
          good = good && isfinite(d) && d > T(0);
          const T inv = rsqrt(d);
          li[c] = inv;
          l[c * 4 + c] = d * inv;
#pragma unroll
          for (int r = c + 1; r < 4; ++r) {
            T v = a[s][r * 4 + c];
#pragma unroll
            for (int q = 0; q < c; ++q) v = fma(-l[r * 4 + q], l[c * 4 + q], v);
            l[r * 4 + c] = v * inv;
          }
        }
        T v[16];
#pragma unroll
        for (int c = 0; c < 4; ++c)
#pragma unroll
          for (int r = 0; r < 4; ++r) {
            if (r < c) { v[r * 4 + c] = T(0); continue; }
            T acc = (r == c) ? T(1) : T(0);
#pragma unroll
            for (int q = c; q < r; ++q) acc = fma(-l[r * 4 + q], v[q * 4 + c], acc);
            v[r * 4 + c] = acc * li[r];
          }
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(Vb + 4 * r, v[4 * r], v[4 * r + 1], v[4 * r + 2], v[4 * r + 3]);
        flag[K & 1] = good ? 0 : 1;
      }
    }
    __syncthreads();
    if (flag[K & 1]) return false;
    T V[16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      T row4[4];
      ld4(row4, Vb + 4 * r);
#pragma unroll
      for (int q = 0; q < 4; ++q) V[r * 4 + q] = row4[q];
    }
    // Phase B: panel L_IK = A_IK V_Kᵀ (V_K lower: column c needs q ≤ c), and block row K of
    // the diagonal block's inverse.
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      if (tJ[s] == K && tI[s] > K) {
        T Ln[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q <= c; ++q) acc = fma(a[s][r * 4 + q], V[c * 4 + q], acc);
            Ln[r * 4 + c] = acc;
          }
        st_panel(Lb, 4 * NT, tI[s], Ln);
#pragma unroll
        for (int e = 0; e < 16; ++e) a[s][e] = Ln[e];
      }
      if (xI[s] == K) {
        T Xn[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            T acc = T(0);
#pragma unroll
            for (int q = 0; q <= r; ++q) acc = fma(V[r * 4 + q], x[s][q * 4 + c], acc);
            Xn[r * 4 + c] = acc;
          }
#pragma unroll
        for (int e = 0; e < 16; ++e) x[s][e] = Xn[e];
        T XnT[16];
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) XnT[c * 4 + r] = Xn[r * 4 + c];
        st_panel(Xb, 4 * NT, xJ[s], XnT);
      }
    }
    __syncthreads();
    // Phase C: trailing update, and the block inverse's rows below K in K's block.
#pragma unroll
    for (int s = 0; s < CH; ++s) {
      const int I = tI[s], J = tJ[s];
      if (I > K && J > K) {
        T Li[16], Lj[16];
        ld_panel(Li, Lb, 4 * NT, I);
        ld_panel(Lj, Lb, 4 * NT, J);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            T acc = a[s][r * 4 + c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc = fma(-Li[r * 4 + q], Lj[c * 4 + q], acc);
            a[s][r * 4 + c] = acc;
          }
      }
      const int XI = xI[s], XJ = xJ[s];
      if (XI > K && XJ <= K) {
        T Li[16], XkT[16];   // XkT[c][q] = X_KJ[q][c]
        ld_panel(Li, Lb, 4 * NT, XI);
        ld_panel(XkT, Xb, 4 * NT, XJ);
#pragma unroll
        for (int r = 0; r < 4; ++r)
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            T acc = x[s][r * 4 + c];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc = fma(-Li[r * 4 + q], XkT[c * 4 + q], acc);
            x[s][r * 4 + c] = acc;
          }
      }
    }
  }
  // L below the diagonal blocks, the block inverses on them.
#pragma unroll
  for (int s = 0; s < CH; ++s) {
    const int I = tI[s], J = tJ[s];
    if (I >= 0 && I / TB != J / TB) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 4 * I + r, j = 4 * J + q;
          if (i < p && j < p) Mb[(size_t)i * ldM + j] = a[s][r * 4 + q];
        }
    }
    const int XI = xI[s], XJ = xJ[s];
    if (XI >= 0) {
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int i = 4 * XI + r, j = 4 * XJ + q;
          if (i < p && j <= i) Mb[(size_t)i * ldM + j] = x[s][r * 4 + q];
        }
    }
  }
  __syncthreads();
  return true;
}

// out = Xᵀ(X·rhs) = (M + D)⁻¹ rhs with X = L⁻¹ in the lower triangle of Mb (chol_blk with
// FULLX).
template <typename T>
__device__ __forceinline__ void chol_solve(int p, const T* Mb, int ldM, const T* rhs, T* y,
                                           T* out, T* scr) {
  mv_rows<8>(Mb, ldM, p, p, TRI_LOWER, rhs, [&](int r, T v) { y[r] = v; });
  __syncthreads();
  mv_cols(Mb, ldM, p, p, TRI_LOWER, y, scr, [&](int c, T v) { out[c] = v; });
}

// out = M·x with M symmetric, stored as its strict upper triangle in Mb plus diag in dM.
template <typename T>
__device__ __forceinline__ void mv_sym_upper(int p, const T* Mb, int ldM, const T* dM,
                                             const T* x, T* tmp, T* out, T* scr,
                                             int cap = NTHREADS) {
  mv_rows<8>(Mb, ldM, p, p, TRI_SUPPER, x, [&](int r, T v) { tmp[r] = fma(dM[r], x[r], v); });
  __syncthreads();
  mv_cols(Mb, ldM, p, p, TRI_SUPPER, x, scr, [&](int c, T v) { out[c] = tmp[c] + v; }, cap);
}

// Ask L2 to fetch [ptr, ptr + bytes) (128-byte lines, spread over the block's threads), so
// that later phases find the data there instead of waiting for DRAM one dependent phase at a
// time.  No result depends on it.
__device__ __forceinline__ void prefetch_l2(const void* ptr, size_t bytes) {
  if (!ptr) return;
  const char* c = static_cast<const char*>(ptr);
  for (size_t o = (size_t)threadIdx.x * 128; o < bytes; o += (size_t)NTHREADS * 128)
    asm volatile("prefetch.global.L2 [%0];" :: "l"(c + o));
}

// Asynchronous 16-byte copy global → shared (cp.async), and the wait for all of a thread's.
__device__ __forceinline__ void cp_async16(void* dst_smem, const void* src) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(dst_smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(s), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
}

// Copies `bytes` bytes from global src to shared dst (both 16-byte aligned) with the whole
// block: 16-byte asynchronous copies, the tail by bytes; ends with a barrier.
__device__ __forceinline__ void stage_to_smem(unsigned char* dst, const unsigned char* src,
                                              size_t bytes) {
  const size_t n16 = bytes / 16;
  for (size_t i = threadIdx.x; i < n16; i += NTHREADS) cp_async16(dst + 16 * i, src + 16 * i);
  for (size_t i = 16 * n16 + threadIdx.x; i < bytes; i += NTHREADS) dst[i] = src[i];
  cp_async_wait_all();
  __syncthreads();
}

// Nanoseconds of the GPU's global timer.
__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// s/λ rounded into the factor type, kept finite and non-zero.
template <typename T> __device__ __forceinline__ T ratio_to(T r);
template <> __device__ __forceinline__ float ratio_to<float>(float r) {
  return fminf(fmaxf(r, 1e-30f), 1e30f);
}
template <> __device__ __forceinline__ double ratio_to<double>(double r) {
  return fmin(fmax(r, 1e-300), 1e300);
}

}  // namespace qpk

#include "qp_large.cuh"

namespace qpk {

// ------------------------------------------------------------------ forward kernels
// Body of the forward pass for one instance (one 512-thread block), shared by the
// shared-memory kernel and the global-memory kernel.  SR (= [S; RE], leading dimension
// ldS = m1), Mb (M strict upper / X lower, leading dimension ldM) and dM point to shared or
// global memory; setup() fills them (the setup sweep) and factor(dsh) factors
// M + D(dsh) into X.  With ws_resident the factors already live in the workspace, otherwise
// they are copied there for the backward pass.
template <typename T, typename FS, typename FF, typename FV>
__device__ __forceinline__ void fwd_body(const FwdInst<T>& P, const FwdSmem<T>& L,
                                         unsigned char* sm, T* SR, T* Mb, int ldMb, T* dM,
                                         bool ws_resident, FS setup, FF factor, FV solve) {
  using V = typename Split<T>::V;
  const int tid = threadIdx.x;
  const int n = P.n, p = P.p, m = P.m;
  const int m1 = L.m1, nz = L.nz;
  T* cb = reinterpret_cast<T*>(sm + L.ocb);
  double* dv = reinterpret_cast<double*>(sm + L.odbl);
  double *z = dv, *s = z + n, *lam = s + p, *nu = lam + p;
  double *rz = nu + m, *rl = rz + n, *rn = rl + p;
  double *qd = rn + m, *hd = qd + n, *bd = hd + p;   // q, h, b (constant over the solve)
  V* xs = reinterpret_cast<V*>(sm + L.osplit);
  T* tv = reinterpret_cast<T*>(sm + L.ovec);
  const int p4 = (p + 3) / 4 * 4;   // vector strides keep every vector 16-byte aligned
  T *u = tv, *wv = u + m1, *dzn = wv + m1 + p4, *y = dzn + m1, *dl = y + p4, *dla = dl + p4;
  T *rhs = dla + p4, *rhsa = rhs + p4, *dsh = rhsa + p4, *mdl = dsh + p4, *tmp = mdl + p4;
  T *dsv = tmp + p4, *ccv = dsv + p4;
  float* red = reinterpret_cast<float*>(sm + L.ored);
  double* dred = reinterpret_cast<double*>(sm + L.ored);
  Acc<T>* ascr = reinterpret_cast<Acc<T>*>(sm + L.ocb);
  T* tscr = reinterpret_cast<T*>(sm + L.ocb);
  const int kscr = (int)(L.cbytes / sizeof(Acc<T>));
  const int tcap = (int)(L.cbytes / sizeof(T));   // T elements of the work region
  (void)cb;
  __shared__ int s_timeout;
  const unsigned long long t_start = P.time_limit_ns ? globaltimer_ns() : 0ull;

  const T* Qb = P.Q;
  const T* qb = P.q;
  const T* Gb = p ? P.G : nullptr;
  const T* hb = p ? P.h : nullptr;
  const T* Ab = m ? P.A : nullptr;
  const T* bb = m ? P.b : nullptr;
  WsLayout W;
  W.init(n, nz, p, m, (int)sizeof(T), ws_resident);
  unsigned char* wsb = P.ws;
  T* wSR = reinterpret_cast<T*>(wsb + W.oSR);
  T* wX = reinterpret_cast<T*>(wsb + W.oX);
  double* wIt = reinterpret_cast<double*>(wsb + W.oIt);
  int32_t* wSt = reinterpret_cast<int32_t*>(wsb + W.oSt);
  const int ldS = m1, ldM = ldMb;

  int status = ST_CONV, it = 0, extra = 0, flags = 0;
  float last[4] = {0.f, 0.f, 0.f, 0.f};   // residual norms and μ at the returned iterate
  double cert_scale = 1.0;                 // 1/max(‖λ‖∞, ‖ν‖∞) of an infeasibility certificate

  // Certificate of infeasibility (Farkas' lemma) from the current λ ≥ 0, ν: for any z' with
  // Gz' ≤ h, Az' = b, (Gᵀλ + Aᵀν)ᵀz' ≤ hᵀλ + bᵀν, so −(hᵀλ + bᵀν) > R·‖Gᵀλ + Aᵀν‖₁ rules out
  // feasible points with ‖z'‖∞ ≤ R.  Taken with R = 1e3·(1 + ‖z‖∞): at a feasible KKT point
  // the ratio is at most ‖z‖∞ (Gᵀλ + Aᵀν = −(Qz + q) there), while along a diverging Farkas
  // direction it grows with ‖λ‖ until the FP32 Newton system turns singular (near 1e4 in
  // small examples).  Uses rz/rl/rn and xs as scratch; true on every thread when it holds.
  auto infeasible_cert = [&]() -> bool {
    for (int i = tid; i < n + p + m; i += NTHREADS)
      xs[i] = Split<T>::make(i < n ? 0.0 : (i < n + p ? lam[i - n] : nu[i - n - p]));
    __syncthreads();
    kkt_apply<T>(n, p, m, P.Q, p ? P.G : nullptr, m ? P.A : nullptr, xs, ascr, kscr,
                 [&](int) { return 0.0; }, [&](int) { return 0.0; }, [&](int) { return 0.0; },
                 rz, rl, rn);
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    for (int i = tid; i < p; i += NTHREADS) {
      v[0] -= hd[i] * lam[i];
      v[3] = fmax(v[3], fabs(lam[i]));
    }
    for (int i = tid; i < m; i += NTHREADS) {
      v[0] -= bd[i] * nu[i];
      v[3] = fmax(v[3], fabs(nu[i]));
    }
    for (int i = tid; i < n; i += NTHREADS) {
      v[1] += fabs(rz[i]);
      v[2] = fmax(v[2], fabs(z[i]));
    }
    block_reduce4<R_SUM, R_SUM, R_MAX, R_MAX>(v, dred);
    cert_scale = v[3] > 0.0 ? 1.0 / v[3] : 1.0;
    return v[0] > 0.0 && v[0] > 1e3 * (1.0 + v[2]) * v[1];
  };

  // Setup factorisations.  Q may be only positive semidefinite (§3, Eq. 2): a z pivot at
  // rounding level, below zthr = 1e-5 (FP64: 1e-12) of Q's largest diagonal entry, shows a
  // singular Q, and the setup is repeated with Q + δI, δ = 1e-4 (FP64: 1e-8) of the largest
  // of max_i Q_ii and the squared row norms of G and A.  The Newton systems then carry the
  // regularisation, but the residual they are driven by is the exact one with Q, so the
  // iteration is an inexact Newton method whose fixed point is the exact KKT point; the
  // backward refinement likewise uses Q.
  T delta = T(0);
  float qmx;
  {
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = tid; i < n; i += NTHREADS) v[0] = fmaxf(v[0], fabsf((float)Qb[(size_t)i * n + i]));
    block_reduce4f<R_MAX, R_MAX, R_MAX, R_MAX>(v, red);
    qmx = v[0];
  }
  bool ok = setup(Qb, Ab, Gb, T(0), (T)((sizeof(T) == 4 ? 1e-5f : 1e-12f) * qmx));
  __syncthreads();
  if (!ok) {
    float v[4] = {qmx, 0.f, 0.f, 0.f};
    for (int i = tid; i < p + m; i += NTHREADS) {
      const T* row = i < p ? Gb + (size_t)i * n : Ab + (size_t)(i - p) * n;
      float sq = 0.f;
      for (int j = 0; j < n; ++j) sq = fmaf((float)row[j], (float)row[j], sq);
      v[1] = fmaxf(v[1], sq);
    }
    block_reduce4f<R_MAX, R_MAX, R_MAX, R_MAX>(v, red);
    const float scale = fmaxf(fmaxf(v[0], v[1]), 1e-30f);
    delta = (T)((sizeof(T) == 4 ? 1e-4f : 1e-8f) * scale);
    if (isfinite(scale)) ok = setup(Qb, Ab, Gb, delta, T(0));
    __syncthreads();
    if (ok) flags |= FLAG_REGQ;
  }
  if (!ok) status = ST_NOTPD;

  // Stopping thresholds tol·(1 + ‖q‖∞), tol·(1 + ‖h‖∞), tol·(1 + ‖b‖∞) and mu_tol.
  float tz = 0.f, tl = 0.f, tn = 0.f;
  const float tol = (float)P.tol, mutol = (float)P.mu_tol;
  if (ok) {
    if (!ws_resident)
      for (int i = tid; i < (m1 + p) * m1; i += NTHREADS) wSR[i] = SR[i];
    for (int i = tid; i < n; i += NTHREADS) qd[i] = (double)qb[i];
    for (int i = tid; i < p; i += NTHREADS) hd[i] = (double)hb[i];
    for (int i = tid; i < m; i += NTHREADS) bd[i] = (double)bb[i];
    float v[4] = {0.f, 0.f, 0.f, 0.f};
    for (int i = tid; i < n; i += NTHREADS) v[0] = fmaxf(v[0], fabsf((float)qb[i]));
    for (int i = tid; i < p; i += NTHREADS) v[1] = fmaxf(v[1], fabsf((float)hb[i]));
    for (int i = tid; i < m; i += NTHREADS) v[2] = fmaxf(v[2], fabsf((float)bb[i]));
    block_reduce4f<R_MAX, R_MAX, R_MAX, R_SUM>(v, red);
    tz = tol * (1.f + v[0]);
    tl = tol * (1.f + v[1]);
    tn = tol * (1.f + v[2]);
  }

  if (ok && p == 0) {
    // Equality-constrained QP: [z; ν] = S·[−q; b], then FP64-residual refinement.
    for (int i = tid; i < m1; i += NTHREADS) u[i] = (i < n) ? -qb[i] : (i < nz ? T(0) : bb[i - nz]);
    __syncthreads();
    mv_rows<8>(SR, ldS, m1, m1, TRI_ALL, u, [&](int r, T val) {
      if (r < n) z[r] = (double)val; else if (r >= nz) nu[r - nz] = (double)val;
    });
    __syncthreads();
    for (int rs = 0; rs < 6; ++rs) {
      for (int i = tid; i < n + m; i += NTHREADS) xs[i] = Split<T>::make(i < n ? z[i] : nu[i - n]);
      __syncthreads();
      kkt_apply<T>(n, 0, m, Qb, Gb, Ab, xs, ascr, kscr,
                   [&](int j) { return qd[j]; }, [&](int) { return 0.0; },
                   [&](int i) { return -bd[i]; }, rz, rl, rn);
      float v[4] = {0.f, 0.f, 0.f, 0.f};
      for (int i = tid; i < n; i += NTHREADS) v[0] = ropf<R_MAX>(v[0], fabsf((float)rz[i]));
      for (int i = tid; i < m; i += NTHREADS) v[1] = ropf<R_MAX>(v[1], fabsf((float)rn[i]));
      block_reduce4f<R_MAX, R_MAX, R_MAX, R_SUM>(v, red);
      last[0] = v[0];
      last[2] = v[1];
      if (!isfinite(v[0]) || !isfinite(v[1])) { status = ST_NUM; break; }
      if (v[0] <= 0.01f * tz && v[1] <= 0.01f * tn) break;
      for (int i = tid; i < m1; i += NTHREADS) u[i] = (i < n) ? (T)(-rz[i]) : (i < nz ? T(0) : (T)(-rn[i - nz]));
      __syncthreads();
      mv_rows<8>(SR, ldS, m1, m1, TRI_ALL, u, [&](int r, T val) {
        if (r < n) z[r] += (double)val; else if (r >= nz) nu[r - nz] += (double)val;
      });
      __syncthreads();
    }
  } else if (ok) {
    // ---- initial point: the KKT solve with D(s/λ) = I, then shift s and λ positive.
    for (int i = tid; i < p; i += NTHREADS) dsh[i] = T(1);
    for (int i = tid; i < m1; i += NTHREADS) u[i] = (i < n) ? -qb[i] : (i < nz ? T(0) : bb[i - nz]);
    __syncthreads();
    ok = factor(dsh);
    if (!ok) status = ST_NOTPD;
    if (ok) {
      if (!mv_rows_xreg<8>(SR, ldS, m1 + p, m1, u, [&](int r, T val) { wv[r] = val; }))
        mv_rows<8>(SR, ldS, m1 + p, m1, TRI_ALL, u, [&](int r, T val) { wv[r] = val; });
      __syncthreads();
      for (int i = tid; i < p; i += NTHREADS) rhs[i] = wv[m1 + i] - hb[i];
      __syncthreads();
      solve(rhs, y, dl, tscr);
      mv_cols(SR + (size_t)m1 * ldS, ldS, p, m1, TRI_ALL, dl, tscr,
              [&](int c, T val) { dzn[c] = wv[c] - val; }, tcap);
      float v[4] = {-INFINITY, 0.f, -INFINITY, 0.f};
      for (int i = tid; i < n; i += NTHREADS) z[i] = (double)dzn[i];
      for (int i = tid; i < m; i += NTHREADS) nu[i] = (double)dzn[nz + i];
      for (int i = tid; i < p; i += NTHREADS) {
        const float lh = (float)dl[i];
        v[0] = fmaxf(v[0], lh);          // max(−s) with s = −λ̂
        v[1] += lh * lh;
        v[2] = fmaxf(v[2], -lh);         // max(−λ) with λ = λ̂
      }
      block_reduce4f<R_MAX, R_SUM, R_MAX, R_SUM>(v, red);
      const float nrm = sqrtf(v[1]);
      const double shs = (v[0] >= -1e-8f * fmaxf(nrm, 1.f)) ? 1.0 + (double)v[0] : 0.0;
      const double shl = (v[2] >= -1e-8f * fmaxf(nrm, 1.f)) ? 1.0 + (double)v[2] : 0.0;
      for (int i = tid; i < p; i += NTHREADS) {
        const double lh = (double)dl[i];
        s[i] = -lh + shs;
        lam[i] = lh + shl;
      }
      __syncthreads();

      // ---- interior point iterations
      float lam_max = 0.f, lam_check = INFINITY;   // ‖λ‖∞ and the level that triggers a
                                                    // certificate check (1e3 × its first value)
      bool loop_notpd = false;                      // a Newton step's factorisation failed
      // Residual precision (FP32 factors only): the plain FP32 operator while the previous
      // iteration's μ is above 1e5·mu_tol, the FP64-accurate one from then on.  Convergence
      // is only ever declared on an FP64-accurate residual.
      bool exact = sizeof(T) == 8;
      float mu_prev = INFINITY;
      // The KKT residual at the current iterate and its norms (v[0..2]) and μ·p (v[3]).
      auto residual = [&](bool fast, float (&v)[4]) {
        for (int i = tid; i < n + p + m; i += NTHREADS)
          xs[i] = Split<T>::make(i < n ? z[i] : (i < n + p ? lam[i - n] : nu[i - n - p]));
        __syncthreads();
        if (fast)
          kkt_apply_fast<T>(n, p, m, Qb, Gb, Ab, xs, tscr, tcap,
                            [&](int j) { return qd[j]; },
                            [&](int i) { return s[i] - hd[i]; },
                            [&](int i) { return -bd[i]; }, rz, rl, rn);
        else
          kkt_apply<T>(n, p, m, Qb, Gb, Ab, xs, ascr, kscr,
                       [&](int j) { return qd[j]; },
                       [&](int i) { return s[i] - hd[i]; },
                       [&](int i) { return -bd[i]; }, rz, rl, rn);
        v[0] = v[1] = v[2] = v[3] = 0.f;
        for (int i = tid; i < n; i += NTHREADS) v[0] = ropf<R_MAX>(v[0], fabsf((float)rz[i]));
        for (int i = tid; i < p; i += NTHREADS) {
          v[1] = ropf<R_MAX>(v[1], fabsf((float)rl[i]));
          v[3] += (float)s[i] * (float)lam[i];
        }
        for (int i = tid; i < m; i += NTHREADS) v[2] = ropf<R_MAX>(v[2], fabsf((float)rn[i]));
        block_reduce4f<R_MAX, R_MAX, R_MAX, R_SUM>(v, red);
      };
      for (it = 0;; ++it) {
        if (lam_max > lam_check) {
          if (infeasible_cert()) {
            status = ST_INFEAS;
            break;
          }
          lam_check *= 1e3f;
        }
        if (!exact && mu_prev <= 1e5f * mutol) exact = true;
        float v[4];
        residual(!exact, v);
        if (!exact && v[0] <= tz && v[1] <= tl && v[2] <= tn && v[3] / (float)p <= mutol) {
          exact = true;             // the stopping test is only taken on the exact residual
          residual(false, v);
        }
        const float mu = v[3] / (float)p;
        mu_prev = mu;
        last[0] = v[0];
        last[1] = v[1];
        last[2] = v[2];
        last[3] = mu;
        if (!isfinite(v[0]) || !isfinite(v[1]) || !isfinite(v[2]) || !isfinite(mu)) {
          status = ST_NUM;
          break;
        }
        if (v[0] <= tz && v[1] <= tl && v[2] <= tn && mu <= mutol) {
          // FP32 path: also require every complementarity pair with max(λ_i, s_i) > 1e-5 to
          // be resolved, min/max ≤ 1e-5 (at most 4 more iterations).  At finite μ a barely
          // resolved pair keeps s_i/λ_i of order μ/max² instead of 0 or ∞ in the system the
          // backward pass reuses, and the gradient inherits that bias; pairs below the floor
          // (degenerate, both tending to 0) are exempt.
          bool resolved = true;
          if constexpr (sizeof(T) == 4) {
            if (extra < 4) {
              float w[4] = {0.f, 0.f, 0.f, 0.f};
              for (int i = tid; i < p; i += NTHREADS) {
                const float si = (float)s[i], li = (float)lam[i];
                const float hi = fmaxf(si, li);
                if (hi > 1e-5f) w[0] = fmaxf(w[0], fminf(si, li) / hi);
              }
              block_reduce4f<R_MAX, R_MAX, R_MAX, R_MAX>(w, red);
              resolved = w[0] <= 1e-5f;
              ++extra;
            }
          }
          if (resolved) {
            status = ST_CONV;
            break;
          }
        }
        if (it >= P.max_iter) {
          status = ST_MAXIT;
          break;
        }
        if (P.time_limit_ns) {
          if (tid == 0) s_timeout = (globaltimer_ns() - t_start > P.time_limit_ns) ? 1 : 0;
          __syncthreads();
          const int out = s_timeout;
          __syncthreads();
          if (out) {
            status = ST_TIMEOUT;
            break;
          }
        }
        for (int i = tid; i < p; i += NTHREADS) dsh[i] = ratio_to<T>((T)s[i] / (T)lam[i]);
        for (int i = tid; i < m1; i += NTHREADS) u[i] = (i < n) ? (T)(-rz[i]) : (i < nz ? T(0) : (T)(-rn[i - nz]));
        __syncthreads();
        if (!factor(dsh)) {
          status = ST_NOTPD;
          loop_notpd = true;
          break;
        }
        // Affine-scaling (predictor) direction, Eq. 9.
        if (!mv_rows_xreg<8>(SR, ldS, m1 + p, m1, u, [&](int r, T val) { wv[r] = val; }))
          mv_rows<8>(SR, ldS, m1 + p, m1, TRI_ALL, u, [&](int r, T val) { wv[r] = val; });
        __syncthreads();
        for (int i = tid; i < p; i += NTHREADS) rhsa[i] = wv[m1 + i] + (T)(rl[i] - s[i]);
        __syncthreads();
        solve(rhsa, y, dla, tscr);
        mv_sym_upper(p, Mb, ldM, dM, dla, tmp, mdl, tscr, tcap);
        // Δs from the complementarity row where s ≤ λ and from the primal row
        // GΔz + Δs = −r_λ (with GΔz = RE·u − MΔλ) elsewhere: the first multiplies the
        // FP32 error of Δλ by s/λ, which is large exactly where the second is safe.
        float w4[4] = {INFINITY, 0.f, 0.f, 0.f};
        for (int i = tid; i < p; i += NTHREADS) {
          const T si = (T)s[i], li = (T)lam[i], d = dla[i];
          const T dsai = (si <= li) ? -si - dsh[i] * d : (T)(-rl[i]) - wv[m1 + i] + mdl[i];
          dsv[i] = dsai;
          if (dsai < T(0)) w4[0] = fminf(w4[0], (float)(-si / dsai));
          if (d < T(0)) w4[0] = fminf(w4[0], (float)(-li / d));
          w4[1] = fmaxf(w4[1], (float)li);
        }
        block_reduce4f<R_MIN, R_MAX, R_SUM, R_SUM>(w4, red);
        const float a_aff = fminf(1.f, w4[0]);
        lam_max = w4[1];
        if (it == 0) lam_check = 1e3f * fmaxf(1.f, lam_max);
        float w5[4] = {0.f, 0.f, 0.f, 0.f};
        for (int i = tid; i < p; i += NTHREADS) {
          const T si = (T)s[i], li = (T)lam[i];
          w5[0] += (float)((si + (T)a_aff * dsv[i]) * (li + (T)a_aff * dla[i]));
        }
        block_reduce4f<R_SUM, R_SUM, R_SUM, R_SUM>(w5, red);
        const float mu_aff = w5[0] / (float)p;
        const float sr = mu_aff / mu;
        const T smu = (T)(sr * sr * sr * mu);
        // Centering-plus-corrector (Eq. 10) folded into one combined solve.
        for (int i = tid; i < p; i += NTHREADS) {
          const T cc = smu - dsv[i] * dla[i];
          ccv[i] = cc;
          rhs[i] = rhsa[i] + cc / (T)lam[i];
        }
        __syncthreads();
        solve(rhs, y, dl, tscr);
        mv_cols(SR + (size_t)m1 * ldS, ldS, p, m1, TRI_ALL, dl, tscr,
                [&](int c, T val) { dzn[c] = wv[c] - val; }, tcap);
        mv_sym_upper(p, Mb, ldM, dM, dl, tmp, mdl, tscr, tcap);
        float w6[4] = {INFINITY, 0.f, 0.f, 0.f};
        for (int i = tid; i < p; i += NTHREADS) {
          const T si = (T)s[i], li = (T)lam[i], d = dl[i];
          const T dsi = (si <= li) ? -si + ccv[i] / li - dsh[i] * d
                                   : (T)(-rl[i]) - wv[m1 + i] + mdl[i];
          dsv[i] = dsi;
          if (dsi < T(0)) w6[0] = fminf(w6[0], (float)(-si / dsi));
          if (d < T(0)) w6[0] = fminf(w6[0], (float)(-li / d));
        }
        block_reduce4f<R_MIN, R_SUM, R_SUM, R_SUM>(w6, red);
        const double alpha = (double)fminf(1.f, 0.99f * w6[0]);
        for (int i = tid; i < n; i += NTHREADS) z[i] += alpha * (double)dzn[i];
        for (int i = tid; i < m; i += NTHREADS) nu[i] += alpha * (double)dzn[nz + i];
        for (int i = tid; i < p; i += NTHREADS) {
          s[i] += alpha * (double)dsv[i];
          lam[i] += alpha * (double)dl[i];
        }
        __syncthreads();
      }
      // An interior point loop that ran out of steps or time, or whose Newton system became
      // singular, may be facing infeasible data (λ diverging along a Farkas direction).
      if ((status == ST_MAXIT || status == ST_TIMEOUT || loop_notpd) && infeasible_cert())
        status = ST_INFEAS;
      // Factorisation at the returned iterate: the one the backward pass reuses.
      if (status == ST_CONV || status == ST_MAXIT || status == ST_TIMEOUT) {
        for (int i = tid; i < p; i += NTHREADS) dsh[i] = ratio_to<T>((T)s[i] / (T)lam[i]);
        __syncthreads();
        if (!factor(dsh)) status = ST_NOTPD;
      }
      // Near-degenerate point: some pair with max(λ_i, s_i) ≤ 1e-5·max(1, max_j max(λ_j, s_j)).
      if (status == ST_CONV || status == ST_MAXIT || status == ST_TIMEOUT) {
        float w[4] = {INFINITY, 0.f, 0.f, 0.f};
        for (int i = tid; i < p; i += NTHREADS) {
          const float mx = fmaxf((float)s[i], (float)lam[i]);
          w[0] = fminf(w[0], mx);
          w[1] = fmaxf(w[1], mx);
        }
        block_reduce4f<R_MIN, R_MAX, R_SUM, R_SUM>(w, red);
        if (w[0] <= 1e-5f * fmaxf(1.f, w[1])) flags |= FLAG_NEARDEG;
      }
    }
  }

  // ---- outputs and the state kept for the backward pass
  const bool bad = (status == ST_NOTPD || status == ST_NUM);
  const double qnan = __longlong_as_double(0x7ff8000000000000LL);
  // An infeasibility certificate is returned scaled to max(‖λ‖∞, ‖ν‖∞) = 1.
  const double dsc = status == ST_INFEAS ? cert_scale : 1.0;
  for (int i = tid; i < n; i += NTHREADS) {
    const double v = bad ? qnan : z[i];
    P.z[i] = (T)v;
    wIt[i] = v;
  }
  for (int i = tid; i < p; i += NTHREADS) {
    const double vs = bad ? qnan : s[i], vl = bad ? qnan : lam[i] * dsc;
    if (P.lam) P.lam[i] = (T)vl;
    wIt[n + i] = vs;
    wIt[n + p + i] = vl;
  }
  for (int i = tid; i < m; i += NTHREADS) {
    const double v = bad ? qnan : nu[i] * dsc;
    if (P.nu) P.nu[i] = (T)v;
    wIt[n + 2 * p + i] = v;
  }
  if (!bad && !ws_resident)
    for (int i = tid; i < p * p; i += NTHREADS) wX[i] = Mb[(size_t)(i / p) * ldM + i % p];
  if (tid == 0) {
    wSt[0] = status | flags;
    wSt[1] = STAMP_MAGIC;
    wSt[2] = n;
    wSt[3] = p;
    wSt[4] = m;
    wSt[5] = (int32_t)sizeof(T) | (ws_resident ? 256 : 0);
    wSt[6] = nz;
    wSt[7] = stamp_hash(P.Q, p ? P.G : nullptr, m ? P.A : nullptr);
    if (P.status) *P.status = status;
    if (P.iters) *P.iters = it;
    if (P.resid) {
      P.resid[0] = last[0];
      P.resid[1] = last[1];
      P.resid[2] = last[2];
      P.resid[3] = last[3];
    }
  }
}


template <typename T>
__device__ __forceinline__ FwdInst<T> fixed_inst(const FwdParams<T>& P, int bi) {
  const int n = P.n, p = P.p, m = P.m;
  FwdInst<T> I;
  I.n = n; I.p = p; I.m = m; I.nz = P.nz;
  I.Q = P.Q + (size_t)bi * n * n;
  I.q = P.q + (size_t)bi * n;
  I.G = p ? P.G + (size_t)bi * p * n : nullptr;
  I.h = p ? P.h + (size_t)bi * p : nullptr;
  I.A = m ? P.A + (size_t)bi * m * n : nullptr;
  I.b = m ? P.b + (size_t)bi * m : nullptr;
  I.z = P.z + (size_t)bi * n;
  I.lam = P.lam ? P.lam + (size_t)bi * p : nullptr;
  I.nu = P.nu ? P.nu + (size_t)bi * m : nullptr;
  I.status = P.status ? P.status + bi : nullptr;
  I.iters = P.iters ? P.iters + bi : nullptr;
  I.resid = P.resid ? P.resid + 4 * (size_t)bi : nullptr;
  I.ws = P.ws + (size_t)bi * P.ws_inst;
  I.tol = P.tol; I.mu_tol = P.mu_tol; I.max_iter = P.max_iter;
  I.time_limit_ns = P.time_limit_ns;
  return I;
}

// One instance on the shared-memory path (factors in shared memory, register tiles).
template <typename T, int SW, int CH>
__device__ __forceinline__ void fwd_smem_path(const FwdInst<T>& I, unsigned char* sm) {
  FwdSmem<T> L;
  L.init(I.n, I.nz, I.p, I.m, false);
  T* SR = reinterpret_cast<T*>(sm + L.oSR);
  T* Mb = reinterpret_cast<T*>(sm + L.oMb);
  T* dM = reinterpret_cast<T*>(sm + L.odM);
  T* cb = reinterpret_cast<T*>(sm + L.ocb);
  const int n = I.n, p = I.p, m = I.m;
  const int tcap = (int)(L.cbytes / sizeof(T));
  fwd_body<T>(I, L, sm, SR, Mb, L.ldM, dM, false,
      [&](const T* Qb, const T* Ab, const T* Gb, T delta, T zthr) {
        return sweep_setup<T, SW>(n, p, m, Qb, Ab, Gb, SR, L.ldS, Mb, L.ldM, dM, cb, delta, zthr);
      },
      [&](const T* dsh) { return chol_blk<T, CH, true>(p, Mb, L.ldM, dM, dsh, cb); },
      [&](const T* rhs, T* y, T* out, T* scr) { chol_solve(p, Mb, L.ldM, rhs, y, out, scr); });
}

// One instance on the global-memory path (factors in the workspace, see qp_large.cuh).  TC:
// whether the setup sweep may take its rank-64 updates on the tensor cores (qp_tc.cuh).  The
// fixed-size kernel does; the persistent packed kernel does not (its tensor-core variant raised
// a GPU fault whose cause was not found), so its workspace has no panel-tile region.
template <typename T, bool TC>
__device__ __forceinline__ void fwd_global_path(const FwdInst<T>& I, unsigned char* sm) {
  FwdSmem<T> L;
  L.init(I.n, I.nz, I.p, I.m, true);
  const int n = I.n, p = I.p, m = I.m, nz = I.nz;
  WsLayout W;
  W.init(n, nz, p, m, (int)sizeof(T), true, TC);
  T* SR = reinterpret_cast<T*>(I.ws + W.oSR);
  T* Mb = reinterpret_cast<T*>(I.ws + W.oX);
  T* dM = reinterpret_cast<T*>(I.ws + W.odM);
  T* Aw = reinterpret_cast<T*>(I.ws + W.oAw);
  T* pan = reinterpret_cast<T*>(I.ws + W.oPan);
  T* cb = reinterpret_cast<T*>(sm + L.ocb);
  const int tcap = (int)(L.cbytes / sizeof(T));
  fwd_body<T>(I, L, sm, SR, Mb, p > 0 ? p : 1, dM, true,
      [&](const T* Qb, const T* Ab, const T* Gb, T delta, T zthr) {
        return gsweep_setup<T>(n, nz, p, m, Qb, Ab, Gb, SR, Mb, dM, pan, L.span_smem != 0, cb,
                               delta, zthr,
                               TC && L.tc_sweep ? reinterpret_cast<T*>(I.ws + W.oTc) : nullptr);
      },
      [&](const T* dsh) {
        // Small Schur complements: the register-tile routine (M read from and X written to
        // the workspace, panels in shared memory); otherwise the blocked global routine.
        const int NT = (p + 3) >> 2, nt = NT * (NT + 1) / 2, ldM = p > 0 ? p : 1;
        if (nt <= NTHREADS) return chol_blk<T, 1, true>(p, Mb, ldM, dM, dsh, cb);
        if constexpr (sizeof(T) == 4) {
          if (reg_chol_ok(p, 4)) return chol_blk<T, 2, true>(p, Mb, ldM, dM, dsh, cb);
        }
        return gchol_factor<T>(p, Mb, dM, dsh, Aw, pan, L.pan_smem != 0, cb);
      },
      [&](const T* rhs, T* y, T* out, T* scr) {
        const int ldM = p > 0 ? p : 1;
        if (reg_chol_ok(p, (int)sizeof(T))) chol_solve(p, Mb, ldM, rhs, y, out, scr);
        else blk_solve(p, Mb, ldM, rhs, y, out, scr);
      });
}

// Fixed-size batch, shared-memory path: one block per instance.
template <typename T, int SW, int CH>
__global__ void __launch_bounds__(NTHREADS, 1) qp_fwd_kernel(const FwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char sm[];
  fwd_smem_path<T, SW, CH>(fixed_inst(P, blockIdx.x), sm);
}

// Fixed-size batch, global-memory path.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, 1) qp_fwd_large_kernel(const FwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char sm[];
  fwd_global_path<T, true>(fixed_inst(P, blockIdx.x), sm);
}

// Packed batch of uneven sizes, persistent: blocks take instances from an atomic counter in
// the order of the descriptor array (largest estimated cost first), and each instance runs
// the path its own size selects, so its result does not depend on the mix.  MODE selects the
// code compiled in: PK_SMEM the shared-memory path alone (register-allocated on its own, as
// the fixed-size kernel is), PK_BOTH both paths.  The host runs a batch's global-path
// instances in a PK_BOTH kernel and its shared-memory-path instances in a PK_SMEM kernel
// beside it, each over its own descriptor range.
enum : int { PK_SMEM = 0, PK_BOTH = 1 };
template <typename T, int SW, int CH, int MODE>
__global__ void __launch_bounds__(NTHREADS, 1) qp_fwd_packed_kernel(const PackedFwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(P.counter, 1);
    __syncthreads();
    const int k = s_idx;
    __syncthreads();
    if (k >= P.B) break;
    const PackedDesc d = P.desc[k];
    FwdInst<T> I;
    I.n = d.n; I.p = d.nineq; I.m = d.neq; I.nz = d.nz;
    I.Q = P.Q + d.oQ; I.q = P.q + d.oq;
    I.G = d.nineq ? P.G + d.oG : nullptr;
    I.h = d.nineq ? P.h + d.oh : nullptr;
    I.A = d.neq ? P.A + d.oA : nullptr;
    I.b = d.neq ? P.b + d.ob : nullptr;
    I.z = P.z + d.oz;
    I.lam = P.lam ? P.lam + d.olam : nullptr;
    I.nu = P.nu ? P.nu + d.onu : nullptr;
    I.status = P.status ? P.status + d.id : nullptr;
    I.iters = P.iters ? P.iters + d.id : nullptr;
    I.resid = P.resid ? P.resid + 4 * (size_t)d.id : nullptr;
    I.ws = P.ws + d.ows;
    I.tol = P.tol; I.mu_tol = P.mu_tol; I.max_iter = P.max_iter;
    I.time_limit_ns = P.time_limit_ns;
    const bool glob = (d.flags & 1) != 0;
    if (glob && MODE == PK_SMEM) {
      // Not reached (the host gives each kernel only instances of its own path); should it
      // happen, the instance is marked failed rather than run on the wrong path.
      if (threadIdx.x == 0) {
        WsLayout W;
        W.init(I.n, I.nz, I.p, I.m, (int)sizeof(T), glob);
        reinterpret_cast<int32_t*>(I.ws + W.oSt)[0] = ST_NUM;
        if (I.status) *I.status = ST_NUM;
      }
    } else if constexpr (MODE == PK_BOTH) {
      if (glob) fwd_global_path<T, false>(I, sm);
      else fwd_smem_path<T, SW, CH>(I, sm);
    } else {
      fwd_smem_path<T, SW, CH>(I, sm);
    }
    __syncthreads();
  }
}

// One 16-byte streaming store (evict-first: the gradients are not read again here) of the
// first 16 / sizeof(T) entries of v.
__device__ __forceinline__ void st16_stream(float* o, const float (&v)[4]) {
  __stcs(reinterpret_cast<float4*>(o), make_float4(v[0], v[1], v[2], v[3]));
}
__device__ __forceinline__ void st16_stream(double* o, const double (&v)[4]) {
  __stcs(reinterpret_cast<double2*>(o), make_double2(v[0], v[1]));
}

// ------------------------------------------------------------------ backward kernel
template <typename T>
__device__ __forceinline__ void bwd_body(const BwdInst<T>& P, unsigned char* sm) {
  using V = typename Split<T>::V;
  const int tid = threadIdx.x;
  const int n = P.n, p = P.p, m = P.m, nz = P.nz, m1 = nz + m;
  BwdSmem<T> L;
  L.init(n, nz, p, m, P.staged != 0);
  double* dv = reinterpret_cast<double*>(sm + L.odbl);
  double *z = dv, *s = z + n, *lam = s + p, *nu = lam + p;
  double *dz = nu + m, *dlt = dz + n, *dnu = dlt + p;
  double *rz = dnu + m, *rl = rz + n, *rn = rl + p;
  V* xs = reinterpret_cast<V*>(sm + L.osplit);
  T* tv = reinterpret_cast<T*>(sm + L.ovec);
  const int p4 = (p + 3) / 4 * 4;   // vector strides keep every vector 16-byte aligned
  T *u = tv, *wv = u + m1, *dzn = wv + m1 + p4, *y = dzn + m1, *dl = y + p4, *rhs = dl + p4;
  Acc<T>* ascr = reinterpret_cast<Acc<T>*>(sm + L.oscr);
  T* tscr = reinterpret_cast<T*>(sm + L.oscr);
  const int tcap = (int)(8 * 4 * NTHREADS / sizeof(T));   // T elements of the scratch
  float* red = reinterpret_cast<float*>(sm + L.ored);

  WsLayout W;
  W.init(n, nz, p, m, (int)sizeof(T), P.large != 0);
  const unsigned char* wsb = P.ws;
  const T* SR = reinterpret_cast<const T*>(wsb + W.oSR);
  const T* X = reinterpret_cast<const T*>(wsb + W.oX);
  const bool stage = P.staged != 0;
  const double* wIt = reinterpret_cast<const double*>(wsb + W.oIt);
  const T* Qb = P.Q;
  const T* Gb = p ? P.G : nullptr;
  const T* Ab = m ? P.A : nullptr;
  // The stamp the forward pass left: trusted only if it names this instance's sizes, element
  // type, kernel path and Q/G/A buffers.
  const int32_t* stp = reinterpret_cast<const int32_t*>(wsb + W.oSt);
  const bool stamped = stp[1] == STAMP_MAGIC && stp[2] == n && stp[3] == p && stp[4] == m &&
                       stp[5] == ((int32_t)sizeof(T) | (P.large ? 256 : 0)) && stp[6] == nz &&
                       stp[7] == stamp_hash(Qb, Gb, Ab);
  const int sword = stamped ? stp[0] : ST_NOFWD;
  const int status = sword & 0xff;
  if (tid == 0 && P.status) *P.status = sword;
  const T* gz = P.dl_dz;
  const T* gl = P.dl_dlam;   // may be null: zero
  const T* gn = P.dl_dnu;    // may be null: zero

  if (status == ST_NOTPD || status == ST_NUM || status == ST_NOFWD || status == ST_INFEAS) {
    const T qn = (T)__longlong_as_double(0x7ff8000000000000LL);
    if (P.dQ) for (int i = tid; i < n * n; i += NTHREADS) P.dQ[i] = qn;
    if (P.dq) for (int i = tid; i < n; i += NTHREADS) P.dq[i] = qn;
    if (P.dG) for (int i = tid; i < p * n; i += NTHREADS) P.dG[i] = qn;
    if (P.dh) for (int i = tid; i < p; i += NTHREADS) P.dh[i] = qn;
    if (P.dA) for (int i = tid; i < m * n; i += NTHREADS) P.dA[i] = qn;
    if (P.db) for (int i = tid; i < m; i += NTHREADS) P.db[i] = qn;
    return;
  }
  // S/RE and X into shared memory when the host planned room for them (they are read by two
  // S/RE products, two REᵀ products and four products with X).
  if (stage) {
    stage_to_smem(sm + L.oSR, wsb + W.oSR, (size_t)(m1 + p) * m1 * sizeof(T));
    stage_to_smem(sm + L.oX, wsb + W.oX, (size_t)p * p * sizeof(T));
    SR = reinterpret_cast<const T*>(sm + L.oSR);
    X = reinterpret_cast<const T*>(sm + L.oX);
  }
  // Everything else read below from global memory: Q, G, A (refinement residual).
  if (!stage) prefetch_l2(X, (size_t)p * p * sizeof(T));
  prefetch_l2(Qb, (size_t)n * n * sizeof(T));
  prefetch_l2(Gb, (size_t)p * n * sizeof(T));
  prefetch_l2(Ab, (size_t)m * n * sizeof(T));
  for (int i = tid; i < n + 2 * p + m; i += NTHREADS) dv[i] = wIt[i];
  for (int i = tid; i < m1; i += NTHREADS)
    u[i] = (i < n) ? -gz[i] : ((i >= nz && gn) ? -gn[i - nz] : T(0));
  __syncthreads();

  // K_sym [d_z; d_s; d̃_λ; d_ν] = [−∂ℓ/∂z; 0; −∂ℓ/∂λ; −∂ℓ/∂ν]  (Eq. 11; the last two blocks
  // are zero for a loss of z* alone), reduced form:
  //   (M + D(s/λ)) d̃_λ = RE·u + ∂ℓ/∂λ,  [d_z; d_ν] = S·u − REᵀ d̃_λ,  u = [−∂ℓ/∂z; −∂ℓ/∂ν].
  if (!mv_rows_xreg<8>(SR, m1, m1 + p, m1, u, [&](int r, T val) { wv[r] = val; }))
    mv_rows<8>(SR, m1, m1 + p, m1, TRI_ALL, u, [&](int r, T val) { wv[r] = val; });
  __syncthreads();
  const T* rhs0 = wv + m1;
  if (gl) {
    for (int i = tid; i < p; i += NTHREADS) rhs[i] = wv[m1 + i] + gl[i];
    __syncthreads();
    rhs0 = rhs;
  }
  // The global-memory path leaves the blocked factor instead of X = L⁻¹ for large p.
  const bool blk = P.large && !reg_chol_ok(p, (int)sizeof(T));
  if (p > 0) {
    if (blk) blk_solve(p, X, p, rhs0, y, dl, tscr);
    else chol_solve(p, X, p, rhs0, y, dl, tscr);
  }
  mv_cols(SR + (size_t)m1 * m1, m1, p, m1, TRI_ALL, dl, tscr,
          [&](int c, T val) { dzn[c] = wv[c] - val; }, tcap);
  if (p == 0)
    for (int i = tid; i < m1; i += NTHREADS) dzn[i] = wv[i];
  __syncthreads();
  for (int i = tid; i < n; i += NTHREADS) dz[i] = (double)dzn[i];
  for (int i = tid; i < m; i += NTHREADS) dnu[i] = (double)dzn[nz + i];
  for (int i = tid; i < p; i += NTHREADS) dlt[i] = (double)dl[i];
  __syncthreads();

  // Iterative refinement with the FP64-accurate residual of the reduced system
  //   ρ_z = Q d_z + Gᵀ d̃_λ + Aᵀ d_ν + ∂ℓ/∂z,  ρ_λ = G d_z − D(s/λ) d̃_λ,  ρ_ν = A d_z.
  // With a factorisation of relative accuracy δ the correction shrinks by about κδ per
  // step and ‖correction_k‖/‖d‖ estimates that rate, so the error left after a step is
  // about that ratio times the correction: refinement stops once, in each of the three
  // blocks (d_z, d_ν, d̃_λ), the correction is below 1e-3·max(‖block‖∞, 1e-3·‖∂ℓ/∂z‖∞)
  // (at most P.refine steps).  Well-conditioned systems stop after the first step;
  // near-singular A Q⁻¹ Aᵀ blocks take more.
  // This thread's part of max(‖∂ℓ/∂z‖∞, ‖∂ℓ/∂λ‖∞, ‖∂ℓ/∂ν‖∞), reduced with the first step's
  // norms.
  float gpart = 0.f, gfloor = 0.f;
  for (int i = tid; i < n; i += NTHREADS) gpart = fmaxf(gpart, fabsf((float)gz[i]));
  if (gl) for (int i = tid; i < p; i += NTHREADS) gpart = fmaxf(gpart, fabsf((float)gl[i]));
  if (gn) for (int i = tid; i < m; i += NTHREADS) gpart = fmaxf(gpart, fabsf((float)gn[i]));
  for (int rs = 0; rs < P.refine; ++rs) {
    for (int i = tid; i < n + p + m; i += NTHREADS)
      xs[i] = Split<T>::make(i < n ? dz[i] : (i < n + p ? dlt[i - n] : dnu[i - n - p]));
    __syncthreads();
    kkt_apply<T>(n, p, m, Qb, Gb, Ab, xs, ascr, 4 * NTHREADS, [&](int j) { return (double)gz[j]; },
                 [&](int i) { return -(s[i] / lam[i]) * dlt[i] + (gl ? (double)gl[i] : 0.0); },
                 [&](int i) { return gn ? (double)gn[i] : 0.0; },
                 rz, rl, rn);
    for (int i = tid; i < m1; i += NTHREADS) u[i] = (i < n) ? (T)(-rz[i]) : (i < nz ? T(0) : (T)(-rn[i - nz]));
    __syncthreads();
    {
      // [S; RE]·u, with the right-hand side RE·u + ρ_λ of the Schur system formed as each
      // row of RE·u lands
      auto epi = [&](int r, T val) {
        wv[r] = val;
        if (r >= m1) rhs[r - m1] = val + (T)rl[r - m1];
      };
      if (!mv_rows_xreg<8>(SR, m1, m1 + p, m1, u, epi)) mv_rows<8>(SR, m1, m1 + p, m1, TRI_ALL, u, epi);
    }
    __syncthreads();
    if (p > 0) {
      if (blk) blk_solve(p, X, p, rhs, y, dl, tscr);
      else chol_solve(p, X, p, rhs, y, dl, tscr);
    }
    mv_cols(SR + (size_t)m1 * m1, m1, p, m1, TRI_ALL, dl, tscr,
            [&](int c, T val) { dzn[c] = wv[c] - val; }, tcap);
    if (p == 0)
      for (int i = tid; i < m1; i += NTHREADS) dzn[i] = wv[i];
    __syncthreads();
    // v[0..2]: the corrections' norms, v[3..5]: the updated blocks' norms, v[6]: the
    // upstream gradient's norm (first step)
    float v[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, rs == 0 ? gpart : 0.f, 0.f};
    for (int i = tid; i < n; i += NTHREADS) {
      dz[i] += (double)dzn[i];
      v[0] = ropf<R_MAX>(v[0], fabsf((float)dzn[i]));
      v[3] = ropf<R_MAX>(v[3], fabsf((float)dz[i]));
    }
    for (int i = tid; i < m; i += NTHREADS) {
      dnu[i] += (double)dzn[nz + i];
      v[1] = ropf<R_MAX>(v[1], fabsf((float)dzn[nz + i]));
      v[4] = ropf<R_MAX>(v[4], fabsf((float)dnu[i]));
    }
    for (int i = tid; i < p; i += NTHREADS) {
      dlt[i] += (double)dl[i];
      v[2] = ropf<R_MAX>(v[2], fabsf((float)dl[i]));
      v[5] = ropf<R_MAX>(v[5], fabsf((float)dlt[i]));
    }
    block_reduce8f_max(v, red);
    if (rs == 0) gfloor = 1e-3f * v[6];
    bool done = true;
#pragma unroll
    for (int k = 0; k < 3; ++k) done = done && (v[k] <= 1e-3f * fmaxf(v[3 + k], gfloor));
    if (done || !isfinite(v[0] + v[1] + v[2])) break;
  }

  // Gradients of Eq. 8 with d̃_λ = D(λ*) d_λ, formed in the factor precision T from
  // rounded copies of the six vectors (the outer products need no more).
  T* vz = wv;                       // reuse: z, d_z (n each), λ, d̃_λ (p each), ν, d_ν (m each)
  T* vdz = vz + n;
  T* vl = y;
  T* vdl = rhs;
  T* vnu = u;
  T* vdnu = u + m;
  for (int i = tid; i < n; i += NTHREADS) { vz[i] = (T)z[i]; vdz[i] = (T)dz[i]; }
  for (int i = tid; i < p; i += NTHREADS) { vl[i] = (T)lam[i]; vdl[i] = (T)dlt[i]; }
  for (int i = tid; i < m; i += NTHREADS) { vnu[i] = (T)nu[i]; vdnu[i] = (T)dnu[i]; }
  __syncthreads();
  // Rows of dQ (scale ½), dG and dA as one sequence of n + p + m rows of
  // scale·(a_i z_jᵀ + c_i d_z,jᵀ); each thread keeps one 16-byte column group of z and d_z in
  // registers and writes that group of every k-th row with one streaming store.
  const int VW = 16 / (int)sizeof(T), nv = n / VW;
  const bool vec = n % VW == 0 && nv <= NTHREADS &&
      ((((uintptr_t)P.dQ) | ((uintptr_t)P.dG) | ((uintptr_t)P.dA)) & 15) == 0;
  auto row_of = [&](int r, T*& o, T& a, T& c, T& sc) {
    if (r < n) { o = P.dQ ? P.dQ + (size_t)r * n : nullptr; a = vdz[r]; c = vz[r]; sc = T(0.5); }
    else if (r < n + p) {
      const int i = r - n;
      o = P.dG ? P.dG + (size_t)i * n : nullptr; a = vdl[i]; c = vl[i]; sc = T(1);
    } else {
      const int i = r - n - p;
      o = P.dA ? P.dA + (size_t)i * n : nullptr; a = vdnu[i]; c = vnu[i]; sc = T(1);
    }
  };
  if (vec) {
    const int rpp = NTHREADS / nv, g = tid % nv, r0 = tid / nv;
    if (r0 < rpp) {
      T zj[4], dj[4];
#pragma unroll
      for (int e = 0; e < VW; ++e) { zj[e] = vz[g * VW + e]; dj[e] = vdz[g * VW + e]; }
      for (int r = r0; r < n + p + m; r += rpp) {
        T* o; T a, c, sc;
        row_of(r, o, a, c, sc);
        if (!o) continue;
        T v[4];
#pragma unroll
        for (int e = 0; e < VW; ++e) v[e] = sc * fma(a, zj[e], c * dj[e]);
        st16_stream(o + g * VW, v);
      }
    }
  } else {
    for (int r = 0; r < n + p + m; ++r) {
      T* o; T a, c, sc;
      row_of(r, o, a, c, sc);
      if (o)
        for (int j = tid; j < n; j += NTHREADS) o[j] = sc * fma(a, vz[j], c * vdz[j]);
    }
  }
  if (P.dq) for (int i = tid; i < n; i += NTHREADS) P.dq[i] = vdz[i];
  if (P.dh) for (int i = tid; i < p; i += NTHREADS) P.dh[i] = -vdl[i];
  if (P.db) for (int i = tid; i < m; i += NTHREADS) P.db[i] = -vdnu[i];
}


template <typename T>
__global__ void __launch_bounds__(NTHREADS, 1) qp_bwd_kernel(const BwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int bi = blockIdx.x, n = P.n, p = P.p, m = P.m;
  BwdInst<T> I;
  I.n = n; I.p = p; I.m = m; I.nz = P.nz; I.large = P.large; I.staged = P.staged;
  I.Q = P.Q + (size_t)bi * n * n;
  I.G = p ? P.G + (size_t)bi * p * n : nullptr;
  I.A = m ? P.A + (size_t)bi * m * n : nullptr;
  I.dl_dz = P.dl_dz + (size_t)bi * n;
  I.dQ = P.dQ ? P.dQ + (size_t)bi * n * n : nullptr;
  I.dq = P.dq ? P.dq + (size_t)bi * n : nullptr;
  I.dG = P.dG ? P.dG + (size_t)bi * p * n : nullptr;
  I.dh = P.dh ? P.dh + (size_t)bi * p : nullptr;
  I.dA = P.dA ? P.dA + (size_t)bi * m * n : nullptr;
  I.db = P.db ? P.db + (size_t)bi * m : nullptr;
  I.ws = P.ws + (size_t)bi * P.ws_inst;
  I.refine = P.refine;
  I.dl_dlam = P.dl_dlam ? P.dl_dlam + (size_t)bi * p : nullptr;
  I.dl_dnu = P.dl_dnu ? P.dl_dnu + (size_t)bi * m : nullptr;
  I.status = P.status ? P.status + bi : nullptr;
  bwd_body<T>(I, sm);
}

// Backward pass of a packed batch, persistent like its forward kernel.
template <typename T>
__global__ void __launch_bounds__(NTHREADS, 1) qp_bwd_packed_kernel(const PackedBwdParams<T> P) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_idx;
  for (;;) {
    if (threadIdx.x == 0) s_idx = atomicAdd(P.counter, 1);
    __syncthreads();
    const int k = s_idx;
    __syncthreads();
    if (k >= P.B) break;
    const PackedDesc d = P.desc[k];
    BwdInst<T> I;
    I.n = d.n; I.p = d.nineq; I.m = d.neq; I.nz = d.nz; I.large = d.flags & 1; I.staged = 0;
    I.Q = P.Q + d.oQ;
    I.G = d.nineq ? P.G + d.oG : nullptr;
    I.A = d.neq ? P.A + d.oA : nullptr;
    I.dl_dz = P.dl_dz + d.oq;
    I.dQ = P.dQ ? P.dQ + d.oQ : nullptr;
    I.dq = P.dq ? P.dq + d.oq : nullptr;
    I.dG = P.dG ? P.dG + d.oG : nullptr;
    I.dh = P.dh ? P.dh + d.oh : nullptr;
    I.dA = P.dA ? P.dA + d.oA : nullptr;
    I.db = P.db ? P.db + d.ob : nullptr;
    I.ws = P.ws + d.ows;
    I.refine = P.refine;
    I.dl_dlam = nullptr;   // the packed entry takes ∂ℓ/∂z* only
    I.dl_dnu = nullptr;
    I.status = P.status ? P.status + d.id : nullptr;
    bwd_body<T>(I, sm);
    __syncthreads();
  }
}

}  // namespace qpk
