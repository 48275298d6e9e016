// sweep.cu -- the FP64 sweep kernels (prep, batch) and their launch helpers;
// the kernels themselves are in sweep_impl.cuh, the mixed-precision batch
// kernels in sweep_mixed.cu.
#include "sweep_impl.cuh"

namespace qp {

template __global__ void prep_kernel<1>(const __grid_constant__ SweepParams);
template __global__ void prep_kernel<2>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<1, double>(const __grid_constant__ SweepParams);
template __global__ void batch_kernel<2, double>(const __grid_constant__ SweepParams);
template __global__ void grad_gen_kernel<1>(const __grid_constant__ SweepParams);
template __global__ void grad_gen_kernel<2>(const __grid_constant__ SweepParams);

cudaError_t launch_batch_grad(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);

cudaError_t launch_grad_gen(int nint, const SweepParams& p, int ngen, cudaStream_t st) {
  if (nint == 1) grad_gen_kernel<1><<<ngen, kThreads, 0, st>>>(p);
  else grad_gen_kernel<2><<<ngen, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_batch_mixed(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);
int batch_blocks_per_sm_mixed(int nint, size_t smem);

cudaError_t launch_prep(int nint, const SweepParams& p, int slots, cudaStream_t st) {
  if (nint == 1) prep_kernel<1><<<slots, kThreads, 0, st>>>(p);
  else prep_kernel<2><<<slots, kThreads, 0, st>>>(p);
  return cudaGetLastError();
}

cudaError_t launch_batch(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (p.mixed) return launch_batch_mixed(nint, p, grid, smem, st);
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<1, double><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_kernel<2, double><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

int batch_blocks_per_sm(int nint, int mixed, size_t smem) {
  if (mixed) return batch_blocks_per_sm_mixed(nint, smem);
  int n = 0;
  if (nint == 1) {
    cudaFuncSetAttribute(batch_kernel<1, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<1, double>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(batch_kernel<2, double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_kernel<2, double>, kThreads, smem);
  }
  return n;
}

int sweep_threads() { return kThreads; }

}  // namespace qp
