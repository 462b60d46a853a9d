// qp_abi.cu -- the C ABI declared in include/qp_gb300.h: argument checks, kernel-variant
// choice and launches.  No device memory is allocated here; the caller owns every buffer.
#include <stdint.h>

#include <algorithm>
#include <mutex>
#include <vector>

#include "qp_gb300.h"
#include "qp_launch.cuh"

namespace {

constexpr int kDefaultSmemOptin = 232448;  // 227 KiB, used when no device is visible

int max_smem_optin() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) {
    cudaGetLastError();
    return kDefaultSmemOptin;
  }
  if (cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) {
    cudaGetLastError();
    return kDefaultSmemOptin;
  }
  return v;
}

bool dims_ok(int B, int n, int nineq, int neq) {
  return B >= 0 && n >= 1 && n <= 2048 && nineq >= 0 && neq >= 0 && neq <= n;
}

int tiles_of(int N) {
  const int NT = (N + 3) / 4;
  return NT * (NT + 1) / 2;
}

// Smallest compiled (SW, CH) variant whose register tiles cover the sweep matrix (order
// nz + neq + nineq, with nz the padded variable count) and the nineq×nineq Schur complement.
bool pick_variant(int dtype, int n, int nineq, int neq, int* SW, int* CH) {
  const int t3 = tiles_of(qpk::padded_nz(n, neq) + neq + nineq), tp = tiles_of(nineq);
  const int sws[3] = {1, 2, 4};
  const int esz = dtype == QP_F32 ? 4 : 8;
  for (int ch = 1; ch <= 2; ++ch) {
    if (ch * qpk::NTHREADS < tp) continue;
    for (int i = 0; i < 3; ++i) {
      const int sw = sws[i];
      if (sw * qpk::NTHREADS < t3) continue;
      if (!qpk::fwd_variant_exists(esz, sw, ch)) continue;
      *SW = sw;
      *CH = ch;
      return true;
    }
  }
  return false;
}

size_t fwd_smem(int dtype, int n, int nz, int nineq, int neq, bool large) {
  if (dtype == QP_F32) {
    qpk::FwdSmem<float> L;
    L.init(n, nz, nineq, neq, large);
    return L.total;
  }
  qpk::FwdSmem<double> L;
  L.init(n, nz, nineq, neq, large);
  return L.total;
}

size_t bwd_smem(int dtype, int n, int nz, int nineq, int neq, bool staged = false) {
  if (dtype == QP_F32) {
    qpk::BwdSmem<float> L;
    L.init(n, nz, nineq, neq, staged);
    return L.total;
  }
  qpk::BwdSmem<double> L;
  L.init(n, nz, nineq, neq, staged);
  return L.total;
}

// Kernel path for a size: the shared-memory kernel when a register-tile variant covers it and
// its factors fit in shared memory, else the global-memory kernel.  A pure function of the
// sizes and the device's shared-memory limit, so forward and backward always agree.
struct Plan {
  bool ok = false, large = false, bstaged = false;
  int sw = 0, ch = 0, nz = 0;
  size_t fsmem = 0, bsmem = 0, bsmem_staged = 0, ws = 0;
};

// force: 0 automatic, 1 global-memory path, 2 shared-memory path (ok = false if impossible).
// packed: the instance runs in the persistent packed kernel (no tensor-core sweep, so no
// panel-tile region in its workspace).
Plan make_plan(int dtype, int n, int nineq, int neq, int force_global = 0, bool packed = false) {
  Plan pl;
  const size_t lim = (size_t)max_smem_optin();
  int sw = 0, ch = 0;
  const int nz4 = qpk::padded_nz(n, neq);
  const bool smem_ok = pick_variant(dtype, n, nineq, neq, &sw, &ch) &&
                       fwd_smem(dtype, n, nz4, nineq, neq, false) <= lim;
  if (force_global == 2 && !smem_ok) return pl;
  if (force_global != 1 && smem_ok) {
    pl.large = false;
    pl.sw = sw;
    pl.ch = ch;
    pl.nz = nz4;
  } else {
    pl.large = true;
    pl.nz = n + ((qpk::LNB - (n + neq) % qpk::LNB) % qpk::LNB);
  }
  pl.fsmem = fwd_smem(dtype, n, pl.nz, nineq, neq, pl.large);
  pl.bsmem = bwd_smem(dtype, n, pl.nz, nineq, neq);
  // The fixed-size backward kernel stages S/RE and X in shared memory when they fit there.
  if (!pl.large) {
    const size_t st = bwd_smem(dtype, n, pl.nz, nineq, neq, true);
    if (st <= lim) {
      pl.bsmem_staged = st;
      pl.bstaged = true;
    }
  }
  qpk::WsLayout W;
  W.init(n, pl.nz, nineq, neq, dtype == QP_F32 ? 4 : 8, pl.large, !packed);
  pl.ws = W.inst;
  pl.ok = pl.fsmem <= lim && pl.bsmem <= lim;
  return pl;
}

}  // namespace

static_assert(sizeof(qp_instance_desc) == sizeof(qpk::PackedDesc), "descriptor layout");

// Non-blocking side streams, each with a fork/join event pair, created on first use (host-side
// resources, not device memory) and kept for the life of the process.  A caller's stream
// gets its own side stream (up to kSideSlots per device; beyond that, streams share slots by
// hash), so packed calls issued on different streams do not queue behind one another.
struct SideStream {
  cudaStream_t owner = nullptr;   // the caller stream this slot serves
  bool used = false;
  cudaStream_t s = nullptr;
  cudaEvent_t fork = nullptr, join = nullptr;
  std::mutex mu;
};
constexpr int kSideSlots = 16;

SideStream* side_stream(cudaStream_t owner) {
  static std::mutex mu;
  static SideStream slots[64][kSideSlots];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
    cudaGetLastError();
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  SideStream* row = slots[dev];
  SideStream* x = nullptr;
  for (int i = 0; i < kSideSlots && !x; ++i)
    if (row[i].used && row[i].owner == owner) x = &row[i];
  for (int i = 0; i < kSideSlots && !x; ++i)
    if (!row[i].used) x = &row[i];
  if (!x) x = &row[(reinterpret_cast<uintptr_t>(owner) >> 4) % kSideSlots];
  if (!x->used) {
    if (cudaStreamCreateWithFlags(&x->s, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&x->join, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      return nullptr;
    }
    x->used = true;
    x->owner = owner;
  }
  return x;
}

int num_sms() {
  int dev = 0, v = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
    cudaGetLastError();
    return 152;
  }
  return v;
}

// Rough relative cost of one instance (FMA counts of the setup sweep, ~12 interior point
// iterations and the backward solve; the global path runs about 3× slower per FMA); used
// only to order the work queue largest first.
double est_cost(int n, int nz, int p, int m, bool large) {
  const double m1 = nz + m, N = m1 + p;
  const double c = m1 * N * N + 12.0 * (p * (double)p * p / 3.0 + 2.0 * n * N) + N * N;
  return large ? 3.0 * c : c;
}

namespace qpk {
bool fwd_variant_exists(int esz, int SW, int CH) {
  if (esz == 4) return (CH == 1 && (SW == 1 || SW == 2 || SW == 4)) || (CH == 2 && SW == 4);
  return CH == 1 && (SW == 1 || SW == 2);
}
}  // namespace qpk

extern "C" {

void qp_default_options(int dtype, qp_options* opt) {
  if (!opt) return;
  if (dtype == QP_F64) {
    opt->tol = 1e-12;
    opt->mu_tol = 1e-13;
    opt->max_iter = 100;
  } else {
    opt->tol = 1e-10;
    opt->mu_tol = 1e-11;
    opt->max_iter = 50;
  }
  opt->refine = 4;
  opt->path = 0;
  opt->time_limit_us = 0;
}

size_t qp_workspace_bytes(int dtype, int B, int n, int nineq, int neq) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(B, n, nineq, neq)) return 0;
  return (size_t)B * make_plan(dtype, n, nineq, neq).ws;
}

size_t qp_workspace_bytes_opt(const qp_options* opt, int dtype, int B, int n, int nineq,
                              int neq) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(B, n, nineq, neq)) return 0;
  return (size_t)B * make_plan(dtype, n, nineq, neq, opt ? opt->path : 0).ws;
}

int qp_supported(int dtype, int n, int nineq, int neq) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(1, n, nineq, neq)) return QP_EINVAL;
  return make_plan(dtype, n, nineq, neq).ok ? QP_OK : QP_EUNSUPPORTED;
}

int qp_uses_global_path(int dtype, int n, int nineq, int neq) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(1, n, nineq, neq)) return -1;
  return make_plan(dtype, n, nineq, neq).large ? 1 : 0;
}

int qp_uses_tensor_cores(const qp_options* opt, int dtype, int n, int nineq, int neq) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(1, n, nineq, neq)) return -1;
  const Plan pl = make_plan(dtype, n, nineq, neq, opt ? opt->path : 0);
  if (!pl.ok) return -1;
  return pl.large && qpk::tc_sweep_ok(n, pl.nz, nineq, neq, dtype == QP_F32 ? 4 : 8) ? 1 : 0;
}

int qp_forward(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
               const void* Q, const void* q, const void* G, const void* h, const void* A,
               const void* b, void* z, void* lam, void* nu, int32_t* status, int32_t* iters,
               double* resid, void* workspace, size_t workspace_bytes, void* stream) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(B, n, nineq, neq)) return QP_EINVAL;
  if (B == 0) return QP_OK;
  if (!Q || !q || !z || !workspace) return QP_EINVAL;
  if (nineq > 0 && (!G || !h)) return QP_EINVAL;
  if (neq > 0 && (!A || !b)) return QP_EINVAL;
  if (((uintptr_t)workspace) % 256 != 0) return QP_EINVAL;
  qp_options o;
  if (opt) o = *opt; else qp_default_options(dtype, &o);
  if (o.max_iter < 0 || o.path < 0 || o.path > 1 || o.time_limit_us < 0) return QP_EINVAL;
  const unsigned long long tl_ns = 1000ull * (unsigned long long)o.time_limit_us;
  const Plan pl = make_plan(dtype, n, nineq, neq, o.path);
  if (workspace_bytes < (size_t)B * pl.ws) return QP_ENOSPACE;
  if (!pl.ok) return QP_EUNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (dtype == QP_F32) {
    qpk::FwdParams<float> P{B, n, nineq, neq, pl.nz,
                            (const float*)Q, (const float*)q, (const float*)G, (const float*)h,
                            (const float*)A, (const float*)b, (float*)z, (float*)lam, (float*)nu,
                            status, iters, resid, (unsigned char*)workspace,
                            pl.ws, o.tol, o.mu_tol, o.max_iter, tl_ns};
    e = pl.large ? qpk::launch_fwd_large_f32(P, pl.fsmem, st)
                 : qpk::launch_fwd_f32(P, pl.sw, pl.ch, pl.fsmem, st);
  } else {
    qpk::FwdParams<double> P{B, n, nineq, neq, pl.nz,
                             (const double*)Q, (const double*)q, (const double*)G, (const double*)h,
                             (const double*)A, (const double*)b, (double*)z, (double*)lam,
                             (double*)nu, status, iters, resid, (unsigned char*)workspace,
                             pl.ws, o.tol, o.mu_tol, o.max_iter, tl_ns};
    e = pl.large ? qpk::launch_fwd_large_f64(P, pl.fsmem, st)
                 : qpk::launch_fwd_f64(P, pl.sw, pl.ch, pl.fsmem, st);
  }
  return e == cudaSuccess ? QP_OK : QP_ECUDA;
}

int qp_backward(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
                const void* Q, const void* G, const void* A, const void* workspace,
                size_t workspace_bytes, const void* dl_dz, void* dQ, void* dq, void* dG,
                void* dh, void* dA, void* db, void* stream) {
  return qp_backward_ext(opt, dtype, B, n, nineq, neq, Q, G, A, workspace, workspace_bytes,
                         dl_dz, nullptr, nullptr, dQ, dq, dG, dh, dA, db, nullptr, stream);
}

int qp_backward_ext(const qp_options* opt, int dtype, int B, int n, int nineq, int neq,
                    const void* Q, const void* G, const void* A, const void* workspace,
                    size_t workspace_bytes, const void* dl_dz, const void* dl_dlam,
                    const void* dl_dnu, void* dQ, void* dq, void* dG, void* dh, void* dA,
                    void* db, int32_t* status, void* stream) {
  if ((dtype != QP_F32 && dtype != QP_F64) || !dims_ok(B, n, nineq, neq)) return QP_EINVAL;
  if (B == 0) return QP_OK;
  if (!Q || !dl_dz || !workspace) return QP_EINVAL;
  if (nineq > 0 && !G) return QP_EINVAL;
  if (neq > 0 && !A) return QP_EINVAL;
  if (((uintptr_t)workspace) % 256 != 0) return QP_EINVAL;
  qp_options o;
  if (opt) o = *opt; else qp_default_options(dtype, &o);
  if (o.refine < 0 || o.refine > 4 || o.path < 0 || o.path > 1) return QP_EINVAL;
  const Plan pl = make_plan(dtype, n, nineq, neq, o.path);
  if (workspace_bytes < (size_t)B * pl.ws) return QP_ENOSPACE;
  if (!pl.ok) return QP_EUNSUPPORTED;
  const size_t smem = pl.bstaged ? pl.bsmem_staged : pl.bsmem;
  const int staged = pl.bstaged ? 1 : 0;
  cudaStream_t st = (cudaStream_t)stream;
  cudaError_t e;
  if (dtype == QP_F32) {
    qpk::BwdParams<float> P{B, n, nineq, neq, pl.nz, pl.large ? 1 : 0, staged,
                            (const float*)Q, (const float*)G, (const float*)A,
                            (const float*)dl_dz, (float*)dQ, (float*)dq, (float*)dG, (float*)dh,
                            (float*)dA, (float*)db, (const unsigned char*)workspace,
                            pl.ws, o.refine, (const float*)dl_dlam, (const float*)dl_dnu,
                            status};
    e = qpk::launch_bwd_f32(P, smem, st);
  } else {
    qpk::BwdParams<double> P{B, n, nineq, neq, pl.nz, pl.large ? 1 : 0, staged,
                             (const double*)Q, (const double*)G,
                             (const double*)A, (const double*)dl_dz, (double*)dQ, (double*)dq,
                             (double*)dG, (double*)dh, (double*)dA, (double*)db,
                             (const unsigned char*)workspace, pl.ws, o.refine,
                             (const double*)dl_dlam, (const double*)dl_dnu, status};
    e = qpk::launch_bwd_f64(P, smem, st);
  }
  return e == cudaSuccess ? QP_OK : QP_ECUDA;
}

int qp_packed_plan(const qp_options* opt, int dtype, int B, const int32_t* dims,
                   qp_instance_desc* desc, qp_packed_sizes* sizes) {
  return qp_packed_plan_ex(opt, dtype, B, dims, nullptr, nullptr, desc, sizes);
}

int qp_packed_plan_ex(const qp_options* opt, int dtype, int B, const int32_t* dims,
                      const int8_t* path_hint, const float* cost, qp_instance_desc* desc,
                      qp_packed_sizes* sizes) {
  if ((dtype != QP_F32 && dtype != QP_F64) || B < 0 || !sizes || (B > 0 && (!dims || !desc)))
    return QP_EINVAL;
  qp_options o;
  if (opt) o = *opt; else qp_default_options(dtype, &o);
  const int esz = dtype == QP_F32 ? 4 : 8;
  qp_packed_sizes S{};
  int64_t oQ = 0, oq = 0, oG = 0, oh = 0, oA = 0, ob = 0;
  int64_t ows = 256;   // first 256 bytes: the two work-queue counters
  int sw_need = 1, ch_need = 1;
  size_t fsm = 0, bsm = 0;
  std::vector<std::pair<double, int>> order;
  for (int i = 0; i < B; ++i) {
    const int n = dims[3 * i], p = dims[3 * i + 1], m = dims[3 * i + 2];
    if (!dims_ok(1, n, p, m)) return QP_EINVAL;
    const int hint = path_hint ? path_hint[i] : 0;
    if (hint < 0 || hint > 2) return QP_EINVAL;
    const Plan pl = make_plan(dtype, n, p, m, hint ? hint : o.path, true);
    if (!pl.ok) return QP_EUNSUPPORTED;
    qp_instance_desc& d = desc[i];
    d.n = n; d.nineq = p; d.neq = m; d.id = i; d.nz = pl.nz; d.flags = pl.large ? 1 : 0;
    d.oQ = oQ; d.oq = oq; d.oG = oG; d.oh = oh; d.oA = oA; d.ob = ob;
    d.oz = oq; d.olam = oh; d.onu = ob; d.ows = ows;
    // Offsets padded to multiples of 4 elements keep every instance's rows 16-byte aligned.
    auto r4 = [](int64_t x) { return (x + 3) & ~int64_t(3); };
    oQ += r4((int64_t)n * n); oq += r4(n); oG += r4((int64_t)p * n); oh += r4(p);
    oA += r4((int64_t)m * n); ob += r4(m);
    ows += (int64_t)pl.ws;
    if (!pl.large) {
      sw_need = std::max(sw_need, pl.sw);
      ch_need = std::max(ch_need, pl.ch);
    } else {
      ++S.n_global;
    }
    fsm = std::max(fsm, pl.fsmem);
    bsm = std::max(bsm, pl.bsmem);
    order.push_back({cost ? (double)cost[i] : est_cost(n, pl.nz, p, m, pl.large), i});
  }
  // Register-tile variant covering every shared-memory-path instance.
  int sw = 0, ch = 0;
  const int sws[3] = {1, 2, 4};
  for (int c = ch_need; c <= 2 && !sw; ++c)
    for (int k = 0; k < 3; ++k)
      if (sws[k] >= sw_need && qpk::fwd_variant_exists(esz, sws[k], c)) { sw = sws[k]; ch = c; break; }
  if (!sw) return QP_EUNSUPPORTED;
  // Execution order: global-path instances first, then shared-memory-path ones (the two run
  // as separate kernels), each part largest estimated cost first (longest-processing-time).
  std::vector<qp_instance_desc> tmp(desc, desc + B);
  std::stable_sort(order.begin(), order.end(),
                   [&](const std::pair<double, int>& x, const std::pair<double, int>& y) {
                     const int gx = tmp[x.second].flags & 1, gy = tmp[y.second].flags & 1;
                     return gx != gy ? gx > gy : x.first > y.first;
                   });
  for (int k = 0; k < B; ++k) desc[k] = tmp[order[k].second];
  S.nQ = oQ; S.nq = oq; S.nG = oG; S.nh = oh; S.nA = oA; S.nb = ob;
  S.nz = oq; S.nlam = oh; S.nnu = ob;
  S.ws_bytes = ows;
  S.fwd_smem = (int64_t)fsm; S.bwd_smem = (int64_t)bsm;
  S.sw = sw; S.ch = ch;
  *sizes = S;
  return QP_OK;
}

int qp_forward_packed(const qp_options* opt, int dtype, int B, const qp_instance_desc* desc,
                      const qp_packed_sizes* sizes, const void* Q, const void* q,
                      const void* G, const void* h, const void* A, const void* b, void* z,
                      void* lam, void* nu, int32_t* status, int32_t* iters, double* resid,
                      void* workspace, size_t workspace_bytes, void* stream) {
  if ((dtype != QP_F32 && dtype != QP_F64) || B < 0 || !sizes) return QP_EINVAL;
  if (B == 0) return QP_OK;
  if (!desc || !Q || !q || !z || !workspace) return QP_EINVAL;
  if ((sizes->nG > 0 && (!G || !h)) || (sizes->nA > 0 && (!A || !b))) return QP_EINVAL;
  if (((uintptr_t)workspace) % 256 != 0) return QP_EINVAL;
  if ((int64_t)workspace_bytes < sizes->ws_bytes) return QP_ENOSPACE;
  if ((size_t)sizes->fwd_smem > (size_t)max_smem_optin()) return QP_EUNSUPPORTED;
  qp_options o;
  if (opt) o = *opt; else qp_default_options(dtype, &o);
  if (o.max_iter < 0 || o.time_limit_us < 0) return QP_EINVAL;
  const unsigned long long tl_ns = 1000ull * (unsigned long long)o.time_limit_us;
  cudaStream_t st = (cudaStream_t)stream;
  // Work-queue counters: bytes 0..3 the shared-memory-path kernel's, 4..7 the backward's,
  // 8..11 the kernel of the global-path instances.
  if (cudaMemsetAsync(workspace, 0, 16, st) != cudaSuccess) return QP_ECUDA;
  const int nsm = num_sms(), ng = std::min(std::max(sizes->n_global, 0), B), ns = B - ng;
  auto launch = [&](int mode, int off, int cnt, int grid, int ctr_byte, cudaStream_t s) {
    if (dtype == QP_F32) {
      qpk::PackedFwdParams<float> P{cnt, (const qpk::PackedDesc*)desc + off,
                                    (int*)((char*)workspace + ctr_byte),
                                    (const float*)Q, (const float*)q, (const float*)G,
                                    (const float*)h, (const float*)A, (const float*)b, (float*)z,
                                    (float*)lam, (float*)nu, status, iters, resid,
                                    (unsigned char*)workspace, o.tol, o.mu_tol, o.max_iter, tl_ns};
      return qpk::launch_fwd_packed_f32(P, sizes->sw, sizes->ch, (size_t)sizes->fwd_smem, grid,
                                        mode, s);
    }
    qpk::PackedFwdParams<double> P{cnt, (const qpk::PackedDesc*)desc + off,
                                   (int*)((char*)workspace + ctr_byte),
                                   (const double*)Q, (const double*)q, (const double*)G,
                                   (const double*)h, (const double*)A, (const double*)b,
                                   (double*)z, (double*)lam, (double*)nu, status, iters, resid,
                                   (unsigned char*)workspace, o.tol, o.mu_tol, o.max_iter, tl_ns};
    return qpk::launch_fwd_packed_f64(P, sizes->sw, sizes->ch, (size_t)sizes->fwd_smem, grid,
                                      mode, s);
  };
  cudaError_t e;
  if (ns == 0) {
    e = launch(qpk::PK_BOTH, 0, ng, std::min(ng, nsm), 8, st);
  } else if (ng == 0) {
    e = launch(qpk::PK_SMEM, 0, ns, std::min(ns, nsm), 0, st);
  } else {
    // Both kinds: the global-path instances (first in the descriptor array) in the combined
    // kernel on `stream`, launched first so that its blocks take the SMs first; the
    // shared-memory-path instances in the shared-memory-only kernel on a side stream forked
    // from `stream` and joined back to it.  Each block of either kernel holds its SM until its
    // queue runs dry, so as global-path blocks finish, shared-memory-path blocks take their
    // SMs: the hardware block scheduler balances the two queues without a fixed split.
    SideStream* ss = side_stream(st);
    if (!ss) return QP_ECUDA;
    std::lock_guard<std::mutex> lk(ss->mu);
    if (cudaEventRecord(ss->fork, st) != cudaSuccess) return QP_ECUDA;
    e = launch(qpk::PK_BOTH, 0, ng, std::min(ng, nsm), 8, st);
    if (e != cudaSuccess) return QP_ECUDA;
    if (cudaStreamWaitEvent(ss->s, ss->fork, 0) != cudaSuccess) return QP_ECUDA;
    e = launch(qpk::PK_SMEM, ng, ns, std::min(ns, nsm), 0, ss->s);
    if (cudaEventRecord(ss->join, ss->s) != cudaSuccess ||
        cudaStreamWaitEvent(st, ss->join, 0) != cudaSuccess)
      return QP_ECUDA;
  }
  return e == cudaSuccess ? QP_OK : QP_ECUDA;
}

int qp_backward_packed(const qp_options* opt, int dtype, int B, const qp_instance_desc* desc,
                       const qp_packed_sizes* sizes, const void* Q, const void* G,
                       const void* A, void* workspace, size_t workspace_bytes,
                       const void* dl_dz, void* dQ, void* dq, void* dG, void* dh, void* dA,
                       void* db, int32_t* status, void* stream) {
  if ((dtype != QP_F32 && dtype != QP_F64) || B < 0 || !sizes) return QP_EINVAL;
  if (B == 0) return QP_OK;
  if (!desc || !Q || !dl_dz || !workspace) return QP_EINVAL;
  if ((sizes->nG > 0 && !G) || (sizes->nA > 0 && !A)) return QP_EINVAL;
  if (((uintptr_t)workspace) % 256 != 0) return QP_EINVAL;
  if ((int64_t)workspace_bytes < sizes->ws_bytes) return QP_ENOSPACE;
  if ((size_t)sizes->bwd_smem > (size_t)max_smem_optin()) return QP_EUNSUPPORTED;
  qp_options o;
  if (opt) o = *opt; else qp_default_options(dtype, &o);
  if (o.refine < 0 || o.refine > 4) return QP_EINVAL;
  cudaStream_t st = (cudaStream_t)stream;
  // The backward counter is the second int of the workspace (the forward leaves it alone).
  if (cudaMemsetAsync((char*)workspace + 4, 0, 4, st) != cudaSuccess) return QP_ECUDA;
  const int grid = std::min(B, num_sms());
  int* ctr = (int*)((char*)workspace + 4);
  cudaError_t e;
  if (dtype == QP_F32) {
    qpk::PackedBwdParams<float> P{B, (const qpk::PackedDesc*)desc, ctr, (const float*)Q,
                                  (const float*)G, (const float*)A, (const float*)dl_dz,
                                  (float*)dQ, (float*)dq, (float*)dG, (float*)dh, (float*)dA,
                                  (float*)db, (const unsigned char*)workspace, o.refine,
                                  status};
    e = qpk::launch_bwd_packed_f32(P, (size_t)sizes->bwd_smem, grid, st);
  } else {
    qpk::PackedBwdParams<double> P{B, (const qpk::PackedDesc*)desc, ctr, (const double*)Q,
                                   (const double*)G, (const double*)A, (const double*)dl_dz,
                                   (double*)dQ, (double*)dq, (double*)dG, (double*)dh,
                                   (double*)dA, (double*)db, (const unsigned char*)workspace,
                                   o.refine, status};
    e = qpk::launch_bwd_packed_f64(P, (size_t)sizes->bwd_smem, grid, st);
  }
  return e == cudaSuccess ? QP_OK : QP_ECUDA;
}

const char* qp_strerror(int code) {
  switch (code) {
    case QP_OK: return "ok";
    case QP_EINVAL: return "invalid argument (dtype, sizes, null or misaligned pointer)";
    case QP_ENOSPACE: return "workspace smaller than qp_workspace_bytes()";
    case QP_EUNSUPPORTED: return "problem size beyond what the compiled kernels handle";
    case QP_ECUDA: return "CUDA launch or attribute call failed";
    default: return "unknown error code";
  }
}

}  // extern "C"
