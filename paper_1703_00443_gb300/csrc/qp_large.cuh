// qp_large.cuh -- factorisation routines of the global-memory path, used when the KKT blocks
// of an instance do not fit in shared memory.  Same method and same results layout as the
// register-tile routines in qp_device.cuh (S and RE in SR, M in the strict upper triangle of
// Mb plus dM, the Cholesky factor in the lower triangle of Mb), but the matrices live in the instance's
// global workspace (L2-resident during the solve).  Pivots are taken in blocks: one warp
// handles the pivot block, all threads then form the panel and apply the rank-block update
// to the trailing matrix (LNB = 16 columns per block in the setup sweep, chol_nb columns in
// the per-iteration Cholesky, whose current block column and panel stay in shared memory).
#pragma once

namespace qpk {

constexpr int LNB = 16;   // pivot block of the global-memory path

// Shared-memory scratch of the large routines (elements of T): pivot block, its per-pivot
// rows, and two flags.
constexpr int LARGE_SMEM_ELEMS = 2 * LNB * LNB + 16;

__host__ __device__ inline int round4(int x) { return (x + 3) & ~3; }

// Blocked symmetric Gauss-Jordan sweep over the first m1 pivots (m1 = nz + neq, a multiple of
// LNB) of [[Q̃, Aᵀ, Gᵀ], [A, 0, 0], [G, 0, 0]] held in global memory:
//   rows 0..m1−1 of SR (full square, both triangles) = the z/ν block,
//   rows m1.. of SR (nineq × m1)                     = the λ-by-(z, ν) block,
//   strict upper triangle of Mb plus dM               = the λ-by-λ block.
// Each pivot block replays the scalar sweeps of its LNB pivots on every panel row (the
// pivot columns of a row, read and written as 16-byte vectors), publishes ĉ and ĉ·D⁻¹ to
// the panels (q-major, ld = round8(N); in shared memory after the pivot scratch when
// `pan_in_sm`, else in the global `pan`), and every other entry takes the accumulated update
// a_ij −= Σ_q (ĉ_iq/d_q) ĉ_jq in 8×4 register micro-tiles.  Afterwards the blocks are
// negated where the swept matrix holds −S and −M, so SR = [S; RE] and Mb/dM hold M exactly
// as the register-tile sweep leaves them.
template <typename T>
__device__ __noinline__ bool gsweep_setup(int n, int nz, int p, int m, const T* __restrict__ Q,
                                          const T* __restrict__ A, const T* __restrict__ G,
                                          T* SR, T* Mb, T* dM, T* pan, bool pan_in_sm, T* sm,
                                          T delta, T zthr, T* tcp) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int m1 = nz + m, N = m1 + p, ldS = m1, ldM = p > 0 ? p : 1;
  const bool mvec = (p & 3) == 0;   // rows of Mb 16-byte aligned
  T* sB = sm;                  // pivot block (LNB × LNB), swept in place
  T* sR = sm + LNB * LNB;      // r_k rows
  int* flag = reinterpret_cast<int*>(sm + 2 * LNB * LNB);
  const int ldp = (N + 7) & ~7;
  T* panC = pan_in_sm ? sm + LARGE_SMEM_ELEMS : pan;   // ĉ, q-major: panC[q·ldp + i]
  T* panP = panC + (size_t)LNB * ldp;                  // ĉ·D⁻¹

  for (int e = tid; e < (m1 + p) * m1; e += NTHREADS) {
    const int i = e / m1, j = e - i * m1;
    SR[e] = k3_elem(n, nz, m1, N, Q, A, G, i, j, delta);
  }
  for (int e = tid; e < p * p; e += NTHREADS) Mb[e] = T(0);
  for (int e = tid; e < p; e += NTHREADS) dM[e] = T(0);
  __syncthreads();

  const int RT = (N + 7) >> 3, CT = m1 >> 2;           // tiles of the SR region
  const int RTp = (p + 7) >> 3, CTp = (p + 3) >> 2;    // tile rows / columns of the λλ block
  int kstart = 0;
#if defined(__CUDA_ARCH__) || defined(QP_HOST_EMULATION)
  if constexpr (sizeof(T) == 4) {
    // FP32 with the workspace's panel tiles: every pivot in 64-pivot superblocks on the
    // tensor cores (the last one partial), none left for the 16-pivot blocks below.  Not for
    // the regularised retry of a singular Q (delta > 0): its Schur complements are
    // ill-conditioned by construction, and the backward refinement needs the FP32 sweep's
    // accuracy there (3×TF32 products carry about 10× the FP32 rounding error).
    if (tcp != nullptr && delta == T(0)) {
      const int nsb = (m1 + TC_KB - 1) / TC_KB;
      if (!tc_sweep_superblocks(n, nz, p, m, nsb, SR, Mb, ldM, dM, tcp,
                                reinterpret_cast<unsigned char*>(sm), zthr))
        return false;
      kstart = m1;
    }
  }
#endif
  for (int k0 = kstart; k0 < m1; k0 += LNB) {
    // Phase A (warp 0): scalar sweeps of the pivot block, recording r_k.
    if (warp == 0) {
      for (int e = lane; e < LNB * LNB; e += 32)
        sB[e] = SR[(size_t)(k0 + e / LNB) * ldS + k0 + e % LNB];
      __syncwarp();
      bool good = true;
      for (int k = 0; k < LNB; ++k) {
        const T d = sB[k * LNB + k];
        const int kk = k0 + k;
        good = good && isfinite(d) && (kk < n ? d > zthr : (kk < nz ? d > T(0) : d < T(0)));
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
      T* row = SR + (size_t)i * ldS + k0;
      T v[LNB];
#pragma unroll
      for (int q = 0; q < LNB; q += 4) {
        T t4[4];
        ld4(t4, row + q);
        v[q] = t4[0]; v[q + 1] = t4[1]; v[q + 2] = t4[2]; v[q + 3] = t4[3];
      }
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
      for (int q = 0; q < LNB; q += 4) st4(row + q, v[q], v[q + 1], v[q + 2], v[q + 3]);
      if (i < m1) {
#pragma unroll
        for (int q = 0; q < LNB; ++q) SR[(size_t)(k0 + q) * ldS + i] = v[q];
      }
    }
    __syncthreads();
    // Phase C: rank-LNB update of every entry outside the pivot rows/columns, 8×4 tiles.
    // (a) z/ν block (full square) and λ-by-(z, ν) block: rows 0..N−1, columns 0..m1−1.
    for (int t = tid; t < RT * CT; t += NTHREADS) {
      const int R = t / CT, ib = 8 * R, jb = 4 * (t - R * CT);
      if ((ib >= k0 && ib < k0 + LNB) || (jb >= k0 && jb < k0 + LNB)) continue;
      T c[32];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        T t4[4] = {T(0), T(0), T(0), T(0)};
        if (ib + rr < N) ld4(t4, SR + (size_t)(ib + rr) * ldS + jb);
#pragma unroll
        for (int q = 0; q < 4; ++q) c[rr * 4 + q] = t4[q];
      }
#pragma unroll 4
      for (int q = 0; q < LNB; ++q) {
        T a0[4], a1[4], b[4];
        ld4(a0, panP + (size_t)q * ldp + ib);
        ld4(a1, panP + (size_t)q * ldp + ib + 4);
        ld4(b, panC + (size_t)q * ldp + jb);
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            c[rr * 4 + cc] = fma(-a0[rr], b[cc], c[rr * 4 + cc]);
            c[(rr + 4) * 4 + cc] = fma(-a1[rr], b[cc], c[(rr + 4) * 4 + cc]);
          }
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr)
        if (ib + rr < N)
          st4(SR + (size_t)(ib + rr) * ldS + jb, c[rr * 4], c[rr * 4 + 1], c[rr * 4 + 2], c[rr * 4 + 3]);
    }
    // (b) λ-by-λ block, upper triangle with diagonal: tile row R (rows 8R..8R+7) holds the
    // CTp − 2R tiles of columns 8R..p−1; F(R) = R·(CTp + 1 − R) tiles precede it.
    const int ntp = RTp * (CTp + 1 - RTp);
    for (int t = tid; t < ntp; t += NTHREADS) {
      int lo = 0, hi = RTp - 1;
      while (lo < hi) {   // largest R with F(R) ≤ t
        const int mid = (lo + hi + 1) >> 1;
        if (mid * (CTp + 1 - mid) <= t) lo = mid; else hi = mid - 1;
      }
      const int R = lo, ia = 8 * R, jb = 4 * (2 * R + (t - R * (CTp + 1 - R)));
      T c[32];
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int a = ia + rr;
        if (mvec && a < p && jb > a) {
          T t4[4];
          ld4(t4, Mb + (size_t)a * ldM + jb);
#pragma unroll
          for (int q = 0; q < 4; ++q) c[rr * 4 + q] = t4[q];
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int b = jb + q;
            c[rr * 4 + q] = (a < p && b < p && b >= a) ? ((a == b) ? dM[a] : Mb[(size_t)a * ldM + b])
                                                      : T(0);
          }
        }
      }
#pragma unroll 4
      for (int q = 0; q < LNB; ++q) {
        T a0[4], a1[4], b[4];
        ld4(a0, panP + (size_t)q * ldp + m1 + ia);
        ld4(a1, panP + (size_t)q * ldp + m1 + ia + 4);
        ld4(b, panC + (size_t)q * ldp + m1 + jb);
#pragma unroll
        for (int rr = 0; rr < 4; ++rr)
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) {
            c[rr * 4 + cc] = fma(-a0[rr], b[cc], c[rr * 4 + cc]);
            c[(rr + 4) * 4 + cc] = fma(-a1[rr], b[cc], c[(rr + 4) * 4 + cc]);
          }
      }
#pragma unroll
      for (int rr = 0; rr < 8; ++rr) {
        const int a = ia + rr;
        if (mvec && a < p && jb > a) {
          st4(Mb + (size_t)a * ldM + jb, c[rr * 4], c[rr * 4 + 1], c[rr * 4 + 2], c[rr * 4 + 3]);
        } else {
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int b = jb + q;
            if (a < p && b < p && b >= a) {
              if (a == b) dM[a] = c[rr * 4 + q];
              else Mb[(size_t)a * ldM + b] = c[rr * 4 + q];
            }
          }
        }
      }
    }
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

// Shared scratch of gchol_factor before its panels (elements of T): two parity buffers of the
// pivot block's factor columns and reciprocal pivots, and a flag word.
__host__ __device__ constexpr int gchol_scratch(int nb) { return 2 * nb * nb + 2 * nb + 16; }

// Cholesky of the pivot block of the global-memory factorisation, in registers of warp 0
// (lane r holds row r): A_KK from the block column staged in Sb (Sb[c·ldp + i] = A(i, k0+c))
// becomes L_KK, published by columns: sLT[k·NB + j] = L(k+1+j, k) for k+1+j < NB and 0
// beyond (each column shifted up to start at its first sub-diagonal entry), and
// sInv[k] = 1/L(k, k).  Rows beyond nb are the identity.  Each column step shifts the row
// left by one, so the pivot column is always a[0] and the loop needs no unrolling; pivots and
// columns travel by shuffles.  flag[0] = 1 on a non-positive or non-finite pivot.
template <typename T, int NB>
__device__ __noinline__ void gchol_pivot_block(int k0, int nb, const T* Sb, int ldp, T* sLT,
                                               T* sInv, int* flag) {
  static_assert(NB <= 32, "one lane per row");
  const int r = threadIdx.x & 31;
  T a[NB];
#pragma unroll
  for (int c = 0; c < NB; ++c)
    a[c] = (r < nb && c <= r) ? Sb[(size_t)c * ldp + k0 + r] : ((r == c) ? T(1) : T(0));
  bool good = true;
#pragma unroll 1
  for (int k = 0; k < NB; ++k) {
    const T d = __shfl_sync(0xffffffffu, a[0], k);
    good = good && isfinite(d) && d > T(0);
    const T inv = rsqrt(d);
    const T l = (r > k) ? a[0] * inv : T(0);   // l_rk below the pivot
    const T lsh = __shfl_down_sync(0xffffffffu, l, k + 1);
    if (r < NB) sLT[k * NB + r] = (r + k + 1 < NB) ? lsh : T(0);
    if (r == 0) sInv[k] = inv;
#pragma unroll
    for (int jj = 1; jj < NB; ++jj) {
      const T lj = __shfl_sync(0xffffffffu, l, (k + jj) & 31);
      if (k + jj <= r) a[jj] = fma(-l, lj, a[jj]);
    }
#pragma unroll
    for (int jj = 0; jj + 1 < NB; ++jj) a[jj] = a[jj + 1];
    a[NB - 1] = T(0);
  }
  if (r == 0) flag[0] = good ? 0 : 1;
}

// V_K = L_KK⁻¹ from the published columns of the pivot block (sLT, sInv), by one warp: lane c
// forms column c by forward substitution, and the lower triangle of the diagonal block of Mb
// (rows and columns k0..k0+nb−1) receives it.
template <typename T, int NB>
__device__ __noinline__ void gchol_invert_block(int k0, int nb, const T* sLT, const T* sInv,
                                                T* Mb, int ldM) {
  const int c = threadIdx.x & 31;
  T x[NB];
#pragma unroll
  for (int r = 0; r < NB; ++r) x[r] = (r == c) ? T(1) : T(0);
#pragma unroll
  for (int q = 0; q < NB; ++q) {
    x[q] *= sInv[q];   // V(q, c), zero above the diagonal
#pragma unroll
    for (int m4 = 0; q + 1 + 4 * m4 < NB; ++m4) {
      T w[4];
      ld4(w, sLT + q * NB + 4 * m4);
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = q + 1 + 4 * m4 + e;
        if (r < NB) x[r] = fma(-w[e], x[q], x[r]);
      }
    }
  }
  if (c < nb) {
#pragma unroll
    for (int r = 0; r < NB; ++r)
      if (r >= c && r < nb) Mb[(size_t)(k0 + r) * ldM + k0 + c] = x[r];
  }
}

// Blocked Cholesky factorisation M + D(dsh) = L Lᵀ for Schur complements too large for the
// register tiles.  The factor is left in the lower triangle of Mb (whose strict upper
// triangle keeps M): the inverted diagonal blocks V_K = L_KK⁻¹ and, below them, the panels
// L_IK; blk_solve applies it.  The trailing matrix lives in the global work matrix Aw (lower
// triangle, row stride round4(p)); the current block column S, the panel P and the pivot
// block's columns live in shared memory (or, for very large p, S and P in the global `pan`).
// Block K = columns [k0, k0 + NB), t0 = k0 + NB, block column K staged in S:
//   A: warp 0 factors the diagonal block from S (gchol_pivot_block);
//   B: one thread per row i ≥ t0 solves L_KK l_iᵀ = a_iᵀ (row i of the panel L_IK) by forward
//      substitution, shifting the row through registers so the results come out in order;
//      P[c][i] and Mb[i][k0 + c] receive it;
//   C: every lower-triangle entry of the trailing matrix takes A_IJ −= L_IK L_JKᵀ in 8×4
//      register micro-tiles (tile row t0/8 + R holds the 2R + 2 tiles of columns
//      t0..t0+8R+7).  Tiles of block column K + 1 go to S instead of Aw: they are final and
//      only the next pivot block and panel read them.  Meanwhile warp 0 takes the tiles of the
//      next diagonal block and then runs step A of block K + 1, and warp 1 inverts L_KK into
//      the diagonal block of Mb (the pivot columns are double-buffered by block parity).
// NB is 32 for FP32 and 16 for FP64 (register room of the pivot block).  Returns false on
// every thread on a non-positive pivot.
template <typename T>
__device__ __noinline__ bool gchol_factor(int p, T* Mb, const T* dM, const T* dsh, T* Aw,
                                          T* pan, bool pan_in_sm, T* sm) {
  constexpr int NB = chol_nb((int)sizeof(T));
  constexpr int ND = (NB / 8) * (NB / 8 + 1);      // tiles of one diagonal block
  static_assert(ND <= 32, "one diagonal tile per lane of warp 0");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int ldM = p > 0 ? p : 1, ldA = round4(p), ldp = (p + 7) & ~7;
  const bool mvec = (p & 3) == 0;                   // rows of Mb 16-byte aligned
  T* sLT = sm;                                      // 2 × NB × NB pivot columns
  T* sInv = sm + 2 * NB * NB;                       // 2 × NB reciprocal pivots
  int* flag = reinterpret_cast<int*>(sm + 2 * NB * NB + 2 * NB);
  T* P = pan_in_sm ? sm + gchol_scratch(NB) : pan;  // panel: P[c·ldp + i]
  T* S = P + (size_t)NB * ldp;                      // block column: S[c·ldp + i] = A(i, k0 + c)

  for (int e = tid; e < p * p; e += NTHREADS) {
    const int i = e / p, j = e - i * p;
    if (j > i) continue;
    const T v = (i == j) ? dM[i] + dsh[i] : Mb[(size_t)j * ldM + i];
    if (j < NB) S[(size_t)j * ldp + i] = v;
    else Aw[(size_t)i * ldA + j] = v;
  }
  __syncthreads();
  if (warp == 0) gchol_pivot_block<T, NB>(0, min(NB, p), S, ldp, sLT, sInv, flag);
  __syncthreads();
  for (int k0 = 0, par = 0; k0 < p; k0 += NB, par ^= 1) {
    const int nb = min(NB, p - k0), t0 = k0 + nb;
    const T* cLT = sLT + par * NB * NB;
    const T* cInv = sInv + par * NB;
    if (flag[0]) return false;
    // Phase B: row i of the panel by forward substitution with L_KK.
    for (int i = t0 + tid; i < p; i += NTHREADS) {
      T a[NB];
#pragma unroll
      for (int q = 0; q < NB; ++q) a[q] = S[(size_t)q * ldp + i];
#pragma unroll 1
      for (int c = 0; c < NB; ++c) {
        const T l = a[0] * cInv[c];
        const T* col = cLT + c * NB;
#pragma unroll
        for (int j = 0; j + 1 < NB; j += 4) {
          T w[4];
          ld4(w, col + j);
#pragma unroll
          for (int e = 0; e < 4; ++e)
            if (j + e + 1 < NB) a[j + e] = fma(-l, w[e], a[j + e + 1]);
        }
        a[NB - 1] = l;
      }
#pragma unroll
      for (int c = 0; c < NB; ++c) P[(size_t)c * ldp + i] = a[c];
      T* mrow = Mb + (size_t)i * ldM + k0;
      if (mvec) {
#pragma unroll
        for (int c = 0; c < NB; c += 4) st4(mrow + c, a[c], a[c + 1], a[c + 2], a[c + 3]);
      } else {
#pragma unroll
        for (int c = 0; c < NB; ++c) mrow[c] = a[c];
      }
    }
    __syncthreads();
    // Phase C, with step A of block K + 1 in warp 0 and the inverse of L_KK in warp 1.
    if (warp == 1) gchol_invert_block<T, NB>(k0, nb, cLT, cInv, Mb, ldM);
    if (t0 < p) {
      const int t1 = t0 + NB;
      const long long ntile = (long long)((p - t0 + 7) >> 3) * (((p - t0 + 7) >> 3) + 1);
      auto tile = [&](long long u) {
        int R = (int)((sqrtf(4.0f * (float)u + 1.0f) - 1.0f) * 0.5f);
        while ((long long)(R + 1) * (R + 2) <= u) ++R;
        while ((long long)R * (R + 1) > u) --R;
        const int ib = t0 + 8 * R, jb = t0 + 4 * (int)(u - (long long)R * (R + 1));
        const bool stage = jb < t1;
        T c[32];
#pragma unroll
        for (int rr = 0; rr < 8; ++rr) {
          const int i = ib + rr;
          if (i < p && jb + 3 <= i) {
            T t4[4];
            ld4(t4, Aw + (size_t)i * ldA + jb);
#pragma unroll
            for (int q = 0; q < 4; ++q) c[rr * 4 + q] = t4[q];
          } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              c[rr * 4 + q] = (i < p && jb + q <= i) ? Aw[(size_t)i * ldA + jb + q] : T(0);
          }
        }
#pragma unroll 4
        for (int q = 0; q < NB; ++q) {
          T a0[4], a1[4], b[4];
          ld4(a0, P + (size_t)q * ldp + ib);
          ld4(a1, P + (size_t)q * ldp + ib + 4);
          ld4(b, P + (size_t)q * ldp + jb);
#pragma unroll
          for (int rr = 0; rr < 4; ++rr)
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
              c[rr * 4 + cc] = fma(-a0[rr], b[cc], c[rr * 4 + cc]);
              c[(rr + 4) * 4 + cc] = fma(-a1[rr], b[cc], c[(rr + 4) * 4 + cc]);
            }
        }
        if (stage) {
          // Block column K + 1: S[(jb − t0 + q)·ldp + i].
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int i = ib + rr;
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (i < p && jb + q <= i) S[(size_t)(jb - t0 + q) * ldp + i] = c[rr * 4 + q];
          }
        } else {
#pragma unroll
          for (int rr = 0; rr < 8; ++rr) {
            const int i = ib + rr;
            if (i < p && jb + 3 <= i) {
              st4(Aw + (size_t)i * ldA + jb, c[rr * 4], c[rr * 4 + 1], c[rr * 4 + 2], c[rr * 4 + 3]);
            } else {
#pragma unroll
              for (int q = 0; q < 4; ++q)
                if (i < p && jb + q <= i) Aw[(size_t)i * ldA + jb + q] = c[rr * 4 + q];
            }
          }
        }
      };
      if (warp == 0) {
        // The tiles of the next diagonal block come first in the order (tile rows 0..NB/8−1).
        if (lane < ND && lane < ntile) tile(lane);
        __syncwarp();
        gchol_pivot_block<T, NB>(t0, min(NB, p - t0), S, ldp, sLT + (par ^ 1) * NB * NB,
                                 sInv + (par ^ 1) * NB, flag);
      } else if (warp >= 2) {
        for (long long u = ND + (tid - 64); u < ntile; u += NTHREADS - 64) tile(u);
      }
    }
    __syncthreads();
  }
  return true;
}

// out = (L Lᵀ)⁻¹ rhs with the factor of gchol_factor or chol_blk in the lower triangle of Mb (inverted
// diagonal blocks V_K, panels L_IK below them); y receives L⁻¹ rhs.  Forward substitution
// y_K = V_K (rhs_K − Σ_{J<K} L_KJ y_J) by block rows, then back substitution
// out_K = V_Kᵀ (y_K − Σ_{I>K} L_IKᵀ out_I) by block columns, two barriers per block each way.
// In each block step every thread issues its loads of V_K (staged to shared memory, row
// stride NB + 1) together with its partial-sum loads, eight at a time, so the step waits for
// memory about once.  `scr` holds BLK_SOLVE_SCR elements; y, out and scr are shared memory;
// ends with a barrier.
static_assert(BLK_SOLVE_SCR * 8 <= 8 * 4 * NTHREADS, "solve scratch within the 16 KB work region");
template <typename T>
__device__ __noinline__ void blk_solve(int p, const T* Mb, int ldM, const T* rhs, T* y, T* out,
                                       T* scr) {
  constexpr int NB = chol_nb((int)sizeof(T));
  constexpr int TPR = NTHREADS / NB;   // threads per row of the forward block step
  constexpr int VS = NB + 1;           // row stride of the staged V_K
  constexpr int VPT = (NB * NB + NTHREADS - 1) / NTHREADS;
  static_assert(TPR == 16 || TPR == 32, "row groups within a warp");
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  T* t = scr;                       // NB values
  T* part = scr + 32;               // NWARPS × 32 partial sums
  T* sVb = part + 32 * NWARPS;      // V_K, NB × VS
  auto load_v = [&](int k0, int nb, T (&vv)[VPT]) {
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NTHREADS, r = idx / NB, q = idx - r * NB;
      vv[e] = (idx < NB * NB && r < nb && q <= r) ? Mb[(size_t)(k0 + r) * ldM + k0 + q] : T(0);
    }
  };
  auto store_v = [&](const T (&vv)[VPT]) {
#pragma unroll
    for (int e = 0; e < VPT; ++e) {
      const int idx = tid + e * NTHREADS, r = idx / NB, q = idx - r * NB;
      if (idx < NB * NB) sVb[r * VS + q] = vv[e];
    }
  };
  for (int k0 = 0; k0 < p; k0 += NB) {
    const int nb = min(NB, p - k0);
    T vv[VPT];
    load_v(k0, nb, vv);
    {
      const int r = tid / TPR, h = tid - r * TPR;
      T acc = T(0);
      if (r < nb) {
        const T* row = Mb + (size_t)(k0 + r) * ldM;
#pragma unroll 8
        for (int j = h; j < k0; j += TPR) acc = fma(row[j], y[j], acc);
      }
#pragma unroll
      for (int off = TPR / 2; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
      if (h == 0 && r < nb) t[r] = rhs[k0 + r] - acc;
    }
    store_v(vv);
    __syncthreads();
    if (warp == 0 && lane < nb) {
      T v = T(0);
#pragma unroll
      for (int q = 0; q < NB; ++q) v = fma(sVb[lane * VS + q], t[q], v);
      y[k0 + lane] = v;
    }
    __syncthreads();
  }
  for (int k0 = ((p - 1) / NB) * NB; p > 0 && k0 >= 0; k0 -= NB) {
    const int nb = min(NB, p - k0), t0 = k0 + nb;
    const int c = (NB == 32) ? lane : (lane & 15);
    T vv[VPT];
    load_v(k0, nb, vv);
    {
      T acc = T(0);
      const int rstep = (NB == 32) ? NWARPS : 2 * NWARPS;
      const int r0 = (NB == 32) ? warp : 2 * warp + (lane >> 4);
      if (c < nb) {
#pragma unroll 8
        for (int i = t0 + r0; i < p; i += rstep) acc = fma(Mb[(size_t)i * ldM + k0 + c], out[i], acc);
      }
      part[warp * 32 + lane] = acc;
    }
    store_v(vv);
    __syncthreads();
    if (warp == 0) {
      T u = T(0);
#pragma unroll
      for (int w = 0; w < NWARPS; ++w) {
        u += part[w * 32 + c];
        if (NB != 32) u += part[w * 32 + 16 + c];
      }
      u = (c < nb) ? y[k0 + c] - u : T(0);
      T x = T(0);
#pragma unroll
      for (int r = 0; r < NB; ++r) x = fma(sVb[r * VS + c], __shfl_sync(0xffffffffu, u, r), x);
      if (lane < nb && lane < NB) out[k0 + lane] = x;
    }
    __syncthreads();
  }
}

}  // namespace qpk
