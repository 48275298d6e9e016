// sweep_grad.cu -- the batch kernel in gradient mode (FP64): it rebuilds the
// accumulators A(R) of each batch exactly as the sweep does, then scatters the
// derivative of E_PT2 with respect to h and the packed integrals (recomputing
// the matrix elements; nothing is stored from the forward sweep).
#include "sweep_impl.cuh"

namespace qp {

template __global__ void batch_kernel<1, double, true>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<2, double, true>(const __grid_constant__ SweepParams);

cudaError_t launch_batch_grad(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<1, double, true><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<2, double, true><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace qp
