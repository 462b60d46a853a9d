// FP32 forward-kernel dispatch (FP32 factors, FP64-accurate residuals and iterate).  The
// kernels themselves are compiled one variant per object file from qp_fwd_variant.cu.
#include "qp_launch.cuh"

namespace qpk {

cudaError_t launch_fwd_f32(const FwdParams<float>& P, int SW, int CH, size_t smem, cudaStream_t st) {
  if (SW == 1 && CH == 1) return launch_fwd_v<float, 1, 1>(P, smem, st);
  if (SW == 2 && CH == 1) return launch_fwd_v<float, 2, 1>(P, smem, st);
  if (SW == 4 && CH == 1) return launch_fwd_v<float, 4, 1>(P, smem, st);
  if (SW == 4 && CH == 2) return launch_fwd_v<float, 4, 2>(P, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_large_f32(const FwdParams<float>& P, size_t smem, cudaStream_t st) {
  return launch_fwd_large_v<float>(P, smem, st);
}

template <int SW, int CH>
static cudaError_t gop(const PackedFwdParams<float>& P, size_t smem, int grid, int mode,
                       cudaStream_t st) {
  return mode == PK_BOTH ? launch_fwd_packed_v<float, SW, CH, PK_BOTH>(P, smem, grid, st)
                         : launch_fwd_packed_v<float, SW, CH, PK_SMEM>(P, smem, grid, st);
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
