// One forward-kernel variant per object file.  The build compiles this file once per
// variant with -DQP_T=<float|double> -DQP_KIND=<0 fixed-size, 1 global-memory, 2 packed
// shared-memory-only, 3 packed both paths> and, for kinds 0, 2 and 3, -DQP_SW/-DQP_CH (the
// register-tile slots of the sweep and of the Cholesky).
#include "qp_launch.cuh"

#if !defined(QP_T) || !defined(QP_KIND)
#error "qp_fwd_variant.cu needs -DQP_T and -DQP_KIND"
#endif

namespace qpk {

#if QP_KIND == 0
template <typename T, int SW, int CH>
cudaError_t launch_fwd_v(const FwdParams<T>& P, size_t smem, cudaStream_t st) {
  auto k = qp_fwd_kernel<T, SW, CH>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}
template cudaError_t launch_fwd_v<QP_T, QP_SW, QP_CH>(const FwdParams<QP_T>&, size_t, cudaStream_t);
#elif QP_KIND == 1
template <typename T>
cudaError_t launch_fwd_large_v(const FwdParams<T>& P, size_t smem, cudaStream_t st) {
  auto k = qp_fwd_large_kernel<T>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<P.B, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}
template cudaError_t launch_fwd_large_v<QP_T>(const FwdParams<QP_T>&, size_t, cudaStream_t);
#elif QP_KIND == 2 || QP_KIND == 3
template <typename T, int SW, int CH, int MODE>
cudaError_t launch_fwd_packed_v(const PackedFwdParams<T>& P, size_t smem, int grid, cudaStream_t st) {
  auto k = qp_fwd_packed_kernel<T, SW, CH, MODE>;
  cudaError_t e = prepare_smem(k, smem);
  if (e != cudaSuccess) return e;
  k<<<grid, NTHREADS, smem, st>>>(P);
  return cudaGetLastError();
}
template cudaError_t launch_fwd_packed_v<QP_T, QP_SW, QP_CH, (QP_KIND == 3 ? PK_BOTH : PK_SMEM)>(
    const PackedFwdParams<QP_T>&, size_t, int, cudaStream_t);
#else
#error "unknown QP_KIND"
#endif

}  // namespace qpk
