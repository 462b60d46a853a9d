// FP32 forward-kernel variants (FP32 factors, FP64-accurate residuals and iterate).
#include "qp_launch.cuh"

namespace qpk {

template <int SW, int CH>
static cudaError_t go(const FwdParams<float>& P, size_t smem, cudaStream_t st) {
  auto k = qp_fwd_kernel<float, SW, CH>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fwd_f32(const FwdParams<float>& P, int SW, int CH, size_t smem, cudaStream_t st) {
  if (SW == 1 && CH == 1) return go<1, 1>(P, smem, st);
  if (SW == 2 && CH == 1) return go<2, 1>(P, smem, st);
  if (SW == 4 && CH == 1) return go<4, 1>(P, smem, st);
  if (SW == 4 && CH == 2) return go<4, 2>(P, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_large_f32(const FwdParams<float>& P, size_t smem, cudaStream_t st) {
  auto k = qp_fwd_large_kernel<float>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

template <int SW, int CH>
static cudaError_t gop(const PackedFwdParams<float>& P, size_t smem, int grid, int mode,
                       cudaStream_t st) {
  auto k = mode == PK_BOTH ? qp_fwd_packed_kernel<float, SW, CH, PK_BOTH>
                           : qp_fwd_packed_kernel<float, SW, CH, PK_SMEM>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_fwd_packed_f32(const PackedFwdParams<float>& P, int SW, int CH, size_t smem,
                                  int grid, int mode, cudaStream_t st) {
  if (SW == 1 && CH == 1) return gop<1, 1>(P, smem, grid, mode, st);
  if (SW == 2 && CH == 1) return gop<2, 1>(P, smem, grid, mode, st);
  if (SW == 4 && CH == 1) return gop<4, 1>(P, smem, grid, mode, st);
  if (SW == 4 && CH == 2) return gop<4, 2>(P, smem, grid, mode, st);
  return cudaErrorInvalidValue;
}

}  // namespace qpk
