// qp_launch.cuh -- host-side launchers shared by the translation units of the library.
#pragma once

#include <cuda_runtime.h>

#include <map>
#include <mutex>
#include <utility>

#include "qp_device.cuh"

namespace qpk {

// Tile-slot variants compiled for the forward kernel (sweep slots SW, Cholesky slots CH).
// Each slot holds one 4×4 tile per thread, so a variant covers symmetric matrices with
// up to SW·512 (resp. CH·512) lower-triangular tiles.
bool fwd_variant_exists(int esz, int SW, int CH);

// Each forward-kernel variant is compiled in an object file of its own (qp_fwd_variant.cu,
// built once per variant with -DQP_T/-DQP_SW/-DQP_CH/-DQP_KIND), so the variants compile in
// parallel; the dispatch functions below pick one at run time.
template <typename T, int SW, int CH>
cudaError_t launch_fwd_v(const FwdParams<T>& P, size_t smem, cudaStream_t st);
template <typename T>
cudaError_t launch_fwd_large_v(const FwdParams<T>& P, size_t smem, cudaStream_t st);
template <typename T, int SW, int CH, int MODE>
cudaError_t launch_fwd_packed_v(const PackedFwdParams<T>& P, size_t smem, int grid, cudaStream_t st);

cudaError_t launch_fwd_f32(const FwdParams<float>& P, int SW, int CH, size_t smem, cudaStream_t st);
cudaError_t launch_fwd_f64(const FwdParams<double>& P, int SW, int CH, size_t smem, cudaStream_t st);
cudaError_t launch_fwd_large_f32(const FwdParams<float>& P, size_t smem, cudaStream_t st);
cudaError_t launch_fwd_large_f64(const FwdParams<double>& P, size_t smem, cudaStream_t st);
cudaError_t launch_fwd_packed_f32(const PackedFwdParams<float>& P, int SW, int CH, size_t smem,
                                  int grid, int mode, cudaStream_t st);
cudaError_t launch_fwd_packed_f64(const PackedFwdParams<double>& P, int SW, int CH, size_t smem,
                                  int grid, int mode, cudaStream_t st);
cudaError_t launch_bwd_packed_f32(const PackedBwdParams<float>& P, size_t smem, int grid, cudaStream_t st);
cudaError_t launch_bwd_packed_f64(const PackedBwdParams<double>& P, size_t smem, int grid, cudaStream_t st);
cudaError_t launch_bwd_f32(const BwdParams<float>& P, size_t smem, cudaStream_t st);
cudaError_t launch_bwd_f64(const BwdParams<double>& P, size_t smem, cudaStream_t st);

// Raise a kernel's dynamic shared-memory limit to at least `smem` on the current device.
// The attribute is set once per (device, kernel, new maximum) and remembered: setting it
// is a host-side call that can wait for work in flight, so repeating it before every
// launch would keep launches on different streams from overlapping.
inline cudaError_t set_smem_limit(const void* kernel, size_t smem) {
  static std::mutex mu;
  static std::map<std::pair<int, const void*>, size_t> done;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  std::lock_guard<std::mutex> lk(mu);
  size_t& have = done[{dev, kernel}];
  if (have >= smem) return cudaSuccess;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) have = smem;
  return e;
}

template <typename K>
inline cudaError_t prepare_smem(K kernel, size_t smem) {
  if (smem <= 48 * 1024) return cudaSuccess;
  return set_smem_limit(reinterpret_cast<const void*>(kernel), smem);
}

}  // namespace qpk
