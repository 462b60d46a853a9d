// qp_large.cuh -- factorisation routines of the global-memory path, used when the KKT blocks
// of an instance do not fit in shared memory.  Same method and same results layout as the
// register-tile routines in qp_device.cuh (S and RE in SR, M in the strict upper triangle of
// Mb plus dM, X = L⁻¹ in the lower triangle of Mb), but the matrices live in the instance's
// global workspace (L2-resident during the solve) and pivots are taken in blocks of LNB: one
// warp handles the pivot block in shared memory, all threads then transform the panel and
// apply the rank-LNB update, with three barriers per pivot block.
#pragma once

namespace qpk {

constexpr int LNB = 16;   // pivot block of the global-memory path
static_assert(LNB == 16, "FwdSmem sizes the shared Cholesky panels for 16-wide blocks");

// Shared-memory scratch of the large routines (elements of T): pivot block, its per-pivot
// rows, and two flags.
constexpr int LARGE_SMEM_ELEMS = 2 * LNB * LNB + 16;

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// C(i, j) −= Σ_{q<NQ} Pa[q·ldp + i] · Pb[q·ldp + j] over the rectangle [i0, i1) × [j0, j1)
// (i0, j0 multiples of 4), in 4×4 register micro-tiles spread over the block's threads.
// `cref(i, j)` returns a reference to C(i, j); `keep(i, j)` selects the entries to update
// (a tile is skipped when keep_tile(ti, tj) is false).  Panels are padded so that reading
// the four rows i..i+3 of a tile at the edge stays inside their allocation.
template <typename T, int NQ, typename CR, typename KT, typename KE>
__device__ __forceinline__ void tile_rank_update(int i0, int i1, int j0, int j1, const T* Pa,
                                                 const T* Pb, int ldp, CR cref,
                                                 KT keep_tile, KE keep) {
  const int ti_n = (i1 - i0 + 3) / 4, tj_n = (j1 - j0 + 3) / 4;
  for (int t = threadIdx.x; t < ti_n * tj_n; t += NTHREADS) {
    const int ti = t / tj_n, tj = t - ti * tj_n;
    const int ib = i0 + 4 * ti, jb = j0 + 4 * tj;
    if (!keep_tile(ib, jb)) continue;
    T c[16];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ib + r, j = jb + q;
        c[r * 4 + q] = (i < i1 && j < j1 && keep(i, j)) ? cref(i, j) : T(0);
      }
#pragma unroll
    for (int q = 0; q < NQ; ++q) {
      T a[4], b[4];
      ld4(a, Pa + (size_t)q * ldp + ib);
      ld4(b, Pb + (size_t)q * ldp + jb);
#pragma unroll
      for (int r = 0; r < 4; ++r)
#pragma unroll
        for (int cc = 0; cc < 4; ++cc) c[r * 4 + cc] = fma(-a[r], b[cc], c[r * 4 + cc]);
    }
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int i = ib + r, j = jb + q;
        if (i < i1 && j < j1 && keep(i, j)) cref(i, j) = c[r * 4 + q];
      }
  }
}

// Blocked symmetric Gauss-Jordan sweep over the first m1 pivots (m1 = nz + neq, a multiple of
// LNB) of [[Q̃, Aᵀ, Gᵀ], [A, 0, 0], [G, 0, 0]] held in global memory:
//   rows 0..m1−1 of SR (full square, both triangles) = the z/ν block,
//   rows m1.. of SR (nineq × m1)                     = the λ-by-(z, ν) block,
//   strict upper triangle of Mb plus dM               = the λ-by-λ block.
// Each pivot block replays the scalar sweeps of its LNB pivots on every panel row (the
// pivot columns of a row), publishes ĉ and ĉ·D⁻¹ to `pan` (q-major, ld = N), and every
// other entry takes the accumulated update a_ij −= Σ_q (ĉ_iq/d_q) ĉ_jq.  Afterwards the
// blocks are negated where the swept matrix holds −S and −M, so SR = [S; RE] and Mb/dM
// hold M exactly as the register-tile sweep leaves them.
template <typename T>
__device__ __noinline__ bool gsweep_setup(int n, int nz, int p, int m, const T* __restrict__ Q,
                                          const T* __restrict__ A, const T* __restrict__ G,
                                          T* SR, T* Mb, T* dM, T* pan, T* sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m1 = nz + m, N = m1 + p, ldS = m1, ldM = p > 0 ? p : 1;
  T* sB = sm;                  // pivot block (LNB × LNB), swept in place
  T* sR = sm + LNB * LNB;      // r_k rows
  int* flag = reinterpret_cast<int*>(sm + 2 * LNB * LNB);
  const int ldp = round4(N);
  T* panC = pan;               // ĉ, q-major: panC[q·ldp + i]
  T* panP = pan + (size_t)LNB * ldp;

  for (int e = tid; e < (m1 + p) * m1; e += NTHREADS) {
    const int i = e / m1, j = e - i * m1;
    SR[e] = k3_elem(n, nz, m1, N, Q, A, G, i, j);
  }
  for (int e = tid; e < p * p; e += NTHREADS) Mb[e] = T(0);
  for (int e = tid; e < p; e += NTHREADS) dM[e] = T(0);
  __syncthreads();

  for (int k0 = 0; k0 < m1; k0 += LNB) {
    // Phase A (warp 0): scalar sweeps of the pivot block, recording r_k.
    if (warp == 0) {
      for (int e = lane; e < LNB * LNB; e += 32)
        sB[e] = SR[(size_t)(k0 + e / LNB) * ldS + k0 + e % LNB];
      __syncwarp();
      bool good = true;
      for (int k = 0; k < LNB; ++k) {
        const T d = sB[k * LNB + k];
        good = good && isfinite(d) && ((k0 + k) < nz ? d > T(0) : d < T(0));
        const T dinv = T(1) / d;
        if (lane < LNB) sR[k * LNB + lane] = (lane == k) ? dinv : sB[k * LNB + lane] * dinv;
        T upd[LNB * LNB / 32];
#pragma unroll
        for (int u = 0; u < LNB * LNB / 32; ++u) {
          const int e = lane + 32 * u, r = e / LNB, c = e % LNB;
          T v = sB[e];
          if (r != k && c != k) v = fma(-sB[r * LNB + k] * dinv, sB[k * LNB + c], v);
          else if (r == k && c == k) v = -dinv;
          else v = v * dinv;
          upd[u] = v;
        }
        __syncwarp();
#pragma unroll
        for (int u = 0; u < LNB * LNB / 32; ++u) sB[lane + 32 * u] = upd[u];
        __syncwarp();
      }
      for (int e = lane; e < LNB * LNB; e += 32)
        SR[(size_t)(k0 + e / LNB) * ldS + k0 + e % LNB] = sB[e];
      if (lane == 0) flag[0] = good ? 0 : 1;
    }
    __syncthreads();
    if (flag[0]) return false;
    // Phase B: replay the sweeps on every panel row.
    for (int i = tid; i < N; i += NTHREADS) {
      if (i >= k0 && i < k0 + LNB) continue;
      T v[LNB];
#pragma unroll
      for (int q = 0; q < LNB; ++q) v[q] = (i < m1) ? SR[(size_t)i * ldS + k0 + q] : SR[(size_t)i * ldS + k0 + q];
#pragma unroll
      for (int k = 0; k < LNB; ++k) {
        const T c = v[k];
        panC[(size_t)k * ldp + i] = c;
        panP[(size_t)k * ldp + i] = c * sR[k * LNB + k];
#pragma unroll
        for (int q = 0; q < LNB; ++q)
          if (q != k) v[q] = fma(-c, sR[k * LNB + q], v[q]);
        v[k] = c * sR[k * LNB + k];
      }
#pragma unroll
      for (int q = 0; q < LNB; ++q) {
        SR[(size_t)i * ldS + k0 + q] = v[q];
        if (i < m1) SR[(size_t)(k0 + q) * ldS + i] = v[q];
      }
    }
    __syncthreads();
    // Phase C: rank-LNB update of every entry outside the pivot rows/columns.
    // (a) z/ν block (full square) and λ-by-(z, ν) block: rows 0..N−1, columns 0..m1−1.
    tile_rank_update<T, LNB>(0, N, 0, m1, panP, panC, ldp,
        [&](int i, int j) -> T& { return SR[(size_t)i * ldS + j]; },
        [&](int ib, int jb) { return !(ib >= k0 && ib < k0 + LNB) && !(jb >= k0 && jb < k0 + LNB); },
        [&](int, int) { return true; });
    // (b) λ-by-λ block, upper triangle with diagonal.
    tile_rank_update<T, LNB>(m1, N, m1, N, panP, panC, ldp,
        [&](int i, int j) -> T& {
          const int a = i - m1, b = j - m1;
          return (a == b) ? dM[a] : Mb[(size_t)a * ldM + b];
        },
        [&](int ib, int jb) { return jb + 3 >= ib; },
        [&](int i, int j) { return j >= i; });
    __syncthreads();
  }
  // Negate the z/ν block (it holds −S) and the λ-by-λ block (it holds −M).
  for (int e = tid; e < m1 * m1; e += NTHREADS) SR[e] = -SR[e];
  for (int e = tid; e < p * p; e += NTHREADS) {
    const int a = e / p, b = e - a * p;
    if (b > a) Mb[e] = -Mb[e];
  }
  for (int e = tid; e < p; e += NTHREADS) dM[e] = -dM[e];
  __syncthreads();
  return true;
}

// Blocked Cholesky factorisation M + D(dsh) = L Lᵀ in the global work matrix Aw (lower
// triangle), with X = L⁻¹ built in the lower triangle of Mb (whose strict upper triangle
// keeps M).  Block K of LNB columns: warp 0 factors the diagonal block and inverts its factor
// in registers (lane r holds row r; pivots and rows are exchanged by shuffles), giving
// V = L_KK⁻¹; all threads form the panel L_IK = A_IK Vᵀ and the new block row
// X_KJ ← V X_KJ in shared memory (columns beyond a short last block are zero); then
// A_IJ −= L_IK L_JKᵀ (I ≥ J > K) and X_IJ −= L_IK X_KJ (I > K ≥ J) in register micro-tiles.
// The two panels live in `sm` after its LARGE_SMEM_ELEMS scratch elements when `pan_in_sm`
// (then `sm` holds LARGE_SMEM_ELEMS + 2·LNB·round4(p) elements), else in the global `pan`.
// Returns false on every thread on a non-positive pivot.
template <typename T>
__device__ __noinline__ bool gchol_inv(int p, T* Mb, const T* dM, const T* dsh, T* Aw, T* pan,
                                       bool pan_in_sm, T* sm) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldM = p > 0 ? p : 1;
  T* sV = sm;                  // V = L_KK⁻¹ (LNB × LNB)
  int* flag = reinterpret_cast<int*>(sm + 2 * LNB * LNB);
  const int ldp = round4(p);
  T* panL = pan_in_sm ? sm + LARGE_SMEM_ELEMS : pan;   // panel, q-major: panL[q·ldp + i]
  T* panX = panL + (size_t)LNB * ldp;                   // new block row of X: panX[r·ldp + j]

  for (int e = tid; e < p * p; e += NTHREADS) {
    const int i = e / p, j = e - i * p;
    if (j > i) continue;
    Aw[e] = (i == j) ? dM[i] + dsh[i] : Mb[(size_t)j * ldM + i];
    Mb[e] = (i == j) ? T(1) : T(0);
  }
  __syncthreads();
  for (int k0 = 0; k0 < p; k0 += LNB) {
    const int nb = min(LNB, p - k0);
    // Phase A (warp 0, lanes 0..LNB−1 hold the rows): Cholesky of the diagonal block with
    // V = L_KK⁻¹ accumulated alongside (rows beyond nb are the identity).
    if (warp == 0) {
      const int r = lane;
      T a[LNB], x[LNB];
#pragma unroll
      for (int c = 0; c < LNB; ++c) {
        a[c] = (r < nb && c <= r) ? Aw[(size_t)(k0 + r) * p + k0 + c] : ((r == c) ? T(1) : T(0));
        x[c] = (r == c) ? T(1) : T(0);
      }
      bool good = true;
#pragma unroll
      for (int k = 0; k < LNB; ++k) {
        const T d = __shfl_sync(0xffffffffu, a[k], k);
        good = good && isfinite(d) && d > T(0);
        const T inv = rsqrt(d);
        const T l = a[k] * inv;            // l_rk (r > k)
#pragma unroll
        for (int j = k + 1; j < LNB; ++j) {
          const T lj = __shfl_sync(0xffffffffu, l, j);
          if (r > k && j <= r) a[j] = fma(-l, lj, a[j]);
        }
#pragma unroll
        for (int q = 0; q <= k; ++q) {
          const T xk = __shfl_sync(0xffffffffu, x[q], k) * inv;
          if (r == k) x[q] = xk;
          else if (r > k) x[q] = fma(-l, xk, x[q]);
        }
      }
      if (r < LNB) {
#pragma unroll
        for (int c = 0; c < LNB; ++c) sV[r * LNB + c] = (c <= r) ? x[c] : T(0);
      }
      if (lane == 0) flag[0] = good ? 0 : 1;
    }
    __syncthreads();
    if (flag[0]) return false;
    // Phase B: panel rows (shared memory) and the new block row of X (shared + global).
    for (int i = k0 + nb + tid; i < p; i += NTHREADS) {
      T a[LNB];
#pragma unroll
      for (int q = 0; q < LNB; ++q) a[q] = (q < nb) ? Aw[(size_t)i * p + k0 + q] : T(0);
#pragma unroll
      for (int c = 0; c < LNB; ++c) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < LNB; ++q) acc = fma(a[q], sV[c * LNB + q], acc);
        panL[(size_t)c * ldp + i] = acc;
      }
    }
    for (int j = tid; j < k0 + nb; j += NTHREADS) {
      T xo[LNB];
#pragma unroll
      for (int q = 0; q < LNB; ++q)
        xo[q] = (q < nb && j <= k0 + q) ? Mb[(size_t)(k0 + q) * ldM + j] : T(0);
#pragma unroll
      for (int r = 0; r < LNB; ++r) {
        T acc = T(0);
#pragma unroll
        for (int q = 0; q < LNB; ++q) acc = fma(sV[r * LNB + q], xo[q], acc);
        panX[(size_t)r * ldp + j] = acc;
        if (r < nb && j <= k0 + r) Mb[(size_t)(k0 + r) * ldM + j] = acc;
      }
    }
    __syncthreads();
    // Phase C: trailing update of Aw and of the rows of X below the block.
    const int t0 = k0 + nb;
    if (t0 < p) {
      tile_rank_update<T, LNB>(t0, p, t0, p, panL, panL, ldp,
          [&](int i, int j) -> T& { return Aw[(size_t)i * p + j]; },
          [&](int ib, int jb) { return jb <= ib + 3; },
          [&](int i, int j) { return j <= i; });
      tile_rank_update<T, LNB>(t0, p, 0, t0, panL, panX, ldp,
          [&](int i, int j) -> T& { return Mb[(size_t)i * ldM + j]; },
          [&](int, int) { return true; },
          [&](int, int) { return true; });
    }
    __syncthreads();
  }
  return true;
}

}  // namespace qpk
