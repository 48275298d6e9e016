// sweep_states.cu -- the batch kernel in multi-state form (FP64): one
// accumulator per state, the per-state PT2 sums and the selection by the
// multi-state criterion of Angeli et al. (Sec. "Selected CI").
#include "sweep_impl.cuh"

namespace qp {

template __global__ void batch_kernel<1, double, false, true>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<2, double, false, true>(const __grid_constant__ SweepParams);

// Dynamic shared memory of the multi-state form: nst accumulators of
// max_cells doubles, the ban bitmap (rounded to 8 bytes), the group's
// per-state coefficients, c_I per state and the weights.
size_t states_smem(int max_cells, int nst) {
  const size_t ban_words = (size_t)(((max_cells + 31) / 32 + 1) & ~1);
  return sizeof(double) * (size_t)max_cells * (size_t)nst + sizeof(uint32_t) * ban_words +
         sizeof(double) * (size_t)(kGroup * kMaxStates + 2 * kMaxStates);
}

int batch_blocks_per_sm_states(int nint, size_t smem) {
  int n = 0;
  cudaError_t e;
  if (nint == 1) {
    e = cudaFuncSetAttribute(batch_kernel<1, double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<1, double, false, true>, kThreads, smem);
  } else {
    e = cudaFuncSetAttribute(batch_kernel<2, double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)smem);
    if (e == cudaSuccess)
      e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, double, false, true>, kThreads, smem);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

cudaError_t launch_batch_states(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    batch_kernel<1, double, false, true><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    batch_kernel<2, double, false, true><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

}  // namespace qp
