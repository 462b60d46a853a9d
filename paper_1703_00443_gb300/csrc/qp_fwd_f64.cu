// FP64 forward-kernel dispatch (everything in FP64).  The kernels themselves are compiled
// one variant per object file from qp_fwd_variant.cu.
#include "qp_launch.cuh"

namespace qpk {

cudaError_t launch_fwd_f64(const FwdParams<double>& P, int SW, int CH, size_t smem, cudaStream_t st) {
  if (SW == 1 && CH == 1) return launch_fwd_v<double, 1, 1>(P, smem, st);
  if (SW == 2 && CH == 1) return launch_fwd_v<double, 2, 1>(P, smem, st);
  return cudaErrorInvalidValue;
}

cudaError_t launch_fwd_large_f64(const FwdParams<double>& P, size_t smem, cudaStream_t st) {
  return launch_fwd_large_v<double>(P, smem, st);
}

template <int SW, int CH>
static cudaError_t gop(const PackedFwdParams<double>& P, size_t smem, int grid, int mode,
                       cudaStream_t st) {
  return mode == PK_BOTH ? launch_fwd_packed_v<double, SW, CH, PK_BOTH>(P, smem, grid, st)
                         : launch_fwd_packed_v<double, SW, CH, PK_SMEM>(P, smem, grid, st);
}

cudaError_t launch_fwd_packed_f64(const PackedFwdParams<double>& P, int SW, int CH, size_t smem,
                                  int grid, int mode, cudaStream_t st) {
  if (SW == 1 && CH == 1) return gop<1, 1>(P, smem, grid, mode, st);
  if (SW == 2 && CH == 1) return gop<2, 1>(P, smem, grid, mode, st);
  return cudaErrorInvalidValue;
}

}  // namespace qpk
