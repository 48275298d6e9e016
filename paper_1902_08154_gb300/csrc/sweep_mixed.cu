// sweep_mixed.cu -- the mixed-precision batch kernels (FP32 integral gathers and
// products, FP64 accumulation, denominators and reductions); see sweep_impl.cuh.
#include "sweep_impl.cuh"

namespace qp {

template __global__ void batch_kernel<1, float>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<2, float>(const __grid_constant__ SweepParams);

cudaError_t launch_batch_mixed(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<1, float><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<2, float><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

cudaError_t launch_wave_multi_mixed(int nint, const MultiWaveInline& m, int total_slots, int grid, size_t smem,
                                    cudaStream_t st) {
  return multi_wave_launch<float>(nint, m, total_slots, grid, smem, st);
}

cudaError_t launch_compact_multi_mixed(int nint, const SweepParams* ps, int n, int grid, cudaStream_t st) {
  return multi_compact_launch<float>(nint, ps, n, grid, st);
}

int batch_multi_blocks_per_sm_mixed(int nint, size_t smem) { return multi_blocks_per_sm<float>(nint, smem); }

int batch_blocks_per_sm_mixed(int nint, size_t smem) {
  int n = 0;
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<1, float>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, float>, kThreads, smem);
  }
  return n;
}

}  // namespace qp
