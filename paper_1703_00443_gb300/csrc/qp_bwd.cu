// Backward (adjoint) kernels, FP32 and FP64.
#include "qp_launch.cuh"

namespace qpk {

cudaError_t launch_bwd_f32(const BwdParams<float>& P, size_t smem, cudaStream_t st) {
  auto k = qp_bwd_kernel<float>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_bwd_f64(const BwdParams<double>& P, size_t smem, cudaStream_t st) {
  auto k = qp_bwd_kernel<double>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_bwd_packed_f32(const PackedBwdParams<float>& P, size_t smem, int grid, cudaStream_t st) {
  auto k = qp_bwd_packed_kernel<float>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

cudaError_t launch_bwd_packed_f64(const PackedBwdParams<double>& P, size_t smem, int grid, cudaStream_t st) {
  auto k = qp_bwd_packed_kernel<double>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}

}  // namespace qpk
