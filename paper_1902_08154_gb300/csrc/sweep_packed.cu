// sweep_packed.cu -- the FP64 batch kernels that gather the integrals from
// the packed array (the compound index of Algorithm hash) instead of the
// context's four-index layout: used by the no-allocation entry point, whose
// only copy of the integrals is the caller's packed one.
#include "sweep_impl.cuh"

namespace qp {

template __global__ void batch_kernel<1, double, false, false, false>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<2, double, false, false, false>(const __grid_constant__ SweepParams);

cudaError_t launch_batch_packed(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    batch_kernel<1, double, false, false, false><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    batch_kernel<2, double, false, false, false><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

int batch_blocks_per_sm_packed(int nint, size_t smem) {
  int n = 0;
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<1, double, false, false, false>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double, false, false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, double, false, false, false>, kThreads, smem);
  }
  return n;
}

}  // namespace qp
