// sweep.cu -- the FP64 sweep kernels (prep, batch) and their launch helpers;
// the kernels themselves are in sweep_impl.cuh, the mixed-precision batch
// kernels in sweep_mixed.cu.
#include "sweep_impl.cuh"

namespace qp {

// Per generator of the wave and per state: eps_I and sum A^2/D^2 from the
// items' slots, added in item order with Neumaier's compensation, so that
// they are the same bits on every run and every grid size.
__device__ __forceinline__ void reduce_items(const SweepParams& p, const int t) {
  const int nst = p.nst > 1 ? p.nst : 1;
  if (t >= p.wave_slots * nst) return;
  const int slot = t / nst, st = t - slot * nst;
  const int g = p.meta[slot].g;
  const double* its = p.it_sum + (size_t)slot * p.nper * p.it_stride + 2 * st;
  double se = 0.0, ce = 0.0, ss = 0.0, cs = 0.0;
  for (int j = 0; j < p.nper; j++) {
    const double ve = its[(size_t)j * p.it_stride], vs = its[(size_t)j * p.it_stride + 1];
    double u = se + ve;
    ce += (fabs(se) >= fabs(ve)) ? (se - u) + ve : (ve - u) + se;
    se = u;
    u = ss + vs;
    cs += (fabs(ss) >= fabs(vs)) ? (ss - u) + vs : (vs - u) + ss;
    ss = u;
  }
  if (g < 0) return;
  p.eps[(size_t)st * p.ndet + g] = se + ce;
  p.s2[(size_t)st * p.ndet + g] = ss + cs;
}

__global__ void reduce_items_kernel(const __grid_constant__ SweepParams p) {
  reduce_items(p, blockIdx.x * blockDim.x + threadIdx.x);
}

// Instance blockIdx.y of a multi-instance wave.
__global__ void reduce_items_multi_kernel(const SweepParams* __restrict__ ps) {
  reduce_items(ps[blockIdx.y], blockIdx.x * blockDim.x + threadIdx.x);
}

cudaError_t launch_reduce_items(const SweepParams& p, cudaStream_t st) {
  const int n = p.wave_slots * (p.nst > 1 ? p.nst : 1);
  if (n > 0) reduce_items_kernel<<<(n + 127) / 128, 128, 0, st>>>(p);
  return cudaGetLastError();
}

// max_slots: the most slots any of the n instances has in this wave (one
// state each).
cudaError_t launch_reduce_items_multi(const SweepParams* ps, int n, int max_slots, cudaStream_t st) {
  if (n > 0 && max_slots > 0) reduce_items_multi_kernel<<<dim3((max_slots + 127) / 128, n), 128, 0, st>>>(ps);
  return cudaGetLastError();
}

cudaError_t launch_wave_multi_mixed(int nint, const MultiWaveInline& m, int total_slots, int grid, size_t smem,
                                    cudaStream_t st);
cudaError_t launch_compact_multi_mixed(int nint, const SweepParams* ps, int n, int grid, cudaStream_t st);
int batch_multi_blocks_per_sm_mixed(int nint, size_t smem);

// The prep and batch launches of one wave of several instances: the prep
// kernel reads the pieces' parameters from the device table m.ps, the batch
// kernel from its own parameters mi.
cudaError_t launch_wave_multi(int nint, int mixed, const MultiWave& m, const MultiWaveInline& mi, int total_slots,
                              int grid, size_t smem, cudaStream_t st) {
  if (total_slots <= 0) return cudaSuccess;
  if (nint == 1) prep_multi_kernel<1><<<total_slots, kThreads, 0, st>>>(m);
  else prep_multi_kernel<2><<<total_slots, kThreads, 0, st>>>(m);
  if (mixed) return launch_wave_multi_mixed(nint, mi, total_slots, grid, smem, st);
  return multi_wave_launch<double>(nint, mi, total_slots, grid, smem, st);
}

cudaError_t launch_compact_multi(int nint, int mixed, const SweepParams* ps, int n, int grid, cudaStream_t st) {
  if (mixed) return launch_compact_multi_mixed(nint, ps, n, grid, st);
  return multi_compact_launch<double>(nint, ps, n, grid, st);
}

int batch_multi_blocks_per_sm(int nint, int mixed, size_t smem) {
  if (mixed) return batch_multi_blocks_per_sm_mixed(nint, smem);
  return multi_blocks_per_sm<double>(nint, smem);
}

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
