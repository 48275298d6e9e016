// peaks.cu -- measured throughput of the two pipes that bound the EN-PT2
// sweep on this GPU: the FP64 pipe (the arithmetic of A_alpha, H_aa, 1/D and
// e_alpha) and the integer pipe (XOR / POPC / add of the excitation-degree
// tests and phases).  The sweep's roofline is reported against these
// measured rates instead of a rate derived from the nominal FP64 figure.
//
// Each kernel runs many independent dependency chains per thread over a
// persistent grid (a multiple of the SM count), so that the pipe, not
// latency, limits it.  One operation = one FMA (FP64) or one XOR, POPC or
// add (integer).  Besides the rate per second, the kernels report the rate
// per SM clock (from clock64 around the loop), which does not depend on the
// clock the GPU happened to run at.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

constexpr int kChains = 8;

__global__ void __launch_bounds__(256) dfma_kernel(int iters, double b, double c, double* sink,
                                                   unsigned long long* cycles) {
  double a[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) a[k] = 1.0 + 1e-3 * (threadIdx.x + k);
  const long long t0 = clock64();
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int k = 0; k < kChains; k++) a[k] = fma(a[k], b, c);
  }
  const long long t1 = clock64();
  double s = 0.0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s += a[k];
  if (s == 1234.5678) sink[0] = s;  // never true; keeps the chains alive
  if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

// Per step and chain: x = popc(x ^ y) + (x ^ z) -- two XOR, one POPC, one
// add (4 operations), the shape of the degree tests of the sweep.
__global__ void __launch_bounds__(256) int_kernel(int iters, uint32_t y, uint32_t z, uint32_t* sink,
                                                  unsigned long long* cycles) {
  uint32_t x[kChains];
#pragma unroll
  for (int k = 0; k < kChains; k++) x[k] = threadIdx.x * 2654435761u + k;
  const long long t0 = clock64();
  for (int i = 0; i < iters; i++) {
#pragma unroll
    for (int u = 0; u < 4; u++)
#pragma unroll
      for (int k = 0; k < kChains; k++) x[k] = (uint32_t)__popc(x[k] ^ y) + (x[k] ^ (z + (uint32_t)k));
  }
  const long long t1 = clock64();
  uint32_t s = 0;
#pragma unroll
  for (int k = 0; k < kChains; k++) s ^= x[k];
  if (s == 0x9E3779B9u && y == z) sink[0] = s;
  if (threadIdx.x == 0) atomicMax(cycles, (unsigned long long)(t1 - t0));
}

template <typename Launch>
int time_kernel(Launch&& launch, int reps, double* best_ms) {
  cudaEvent_t a, b;
  if (cudaEventCreate(&a) != cudaSuccess || cudaEventCreate(&b) != cudaSuccess) return -6;
  double best = 1e30;
  for (int r = 0; r < reps; r++) {
    cudaEventRecord(a, 0);
    launch();
    cudaEventRecord(b, 0);
    if (cudaEventSynchronize(b) != cudaSuccess) return -6;
    float ms = 0.f;
    cudaEventElapsedTime(&ms, a, b);
    if (r > 0 && ms < best) best = ms;  // the first run is a warm-up
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (cudaGetLastError() != cudaSuccess) return -6;
  *best_ms = best;
  return 0;
}

}  // namespace

// out[0] = operations per second (1e9), out[1] = operations per SM clock,
// out[2] = kernel milliseconds (best of reps), out[3] = SM clock in MHz
// implied by clock64 cycles / kernel time.  kind 0: FP64 FMA; kind 1:
// integer XOR/POPC/add.  Returns 0 or a negative error code.
extern "C" int qp_peak_measure(int kind, int iters, int reps, double* out) {
  int dev = 0, nsm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return -6;
  if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return -6;
  const int threads = 256, blocks = nsm * 8;
  void* sink = nullptr;
  unsigned long long* cyc = nullptr;
  if (cudaMalloc(&sink, 64) != cudaSuccess) return -5;
  if (cudaMalloc(&cyc, 8) != cudaSuccess) {
    cudaFree(sink);
    return -5;
  }
  if (cudaMemset(cyc, 0, 8) != cudaSuccess) {
    cudaFree(sink);
    cudaFree(cyc);
    return -6;
  }
  double ms = 0.0;
  int rc;
  if (kind == 0) {
    rc = time_kernel([&] { dfma_kernel<<<blocks, threads>>>(iters, 0.9999999, 1e-9, (double*)sink, cyc); }, reps, &ms);
  } else {
    rc = time_kernel([&] { int_kernel<<<blocks, threads>>>(iters, 0x5bd1e995u, 0x1b873593u, (uint32_t*)sink, cyc); },
                     reps, &ms);
  }
  unsigned long long cycles = 0;
  if (rc == 0 && cudaMemcpy(&cycles, cyc, 8, cudaMemcpyDeviceToHost) != cudaSuccess) rc = -6;
  cudaFree(sink);
  cudaFree(cyc);
  if (rc) return rc;
  const double per_thread = (double)iters * 4 * kChains * (kind == 0 ? 1 : 4);
  const double ops = per_thread * threads * blocks;
  out[0] = ops / (ms * 1e-3) / 1e9;
  out[2] = ms;
  // SM clocks over the kernel: the longest block's clock64 interval times the
  // rounds in which the 8 blocks per SM run (1 when all are resident)
  int per_sm = 0;
  if (kind == 0)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, dfma_kernel, threads, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, int_kernel, threads, 0);
  out[1] = out[3] = 0.0;
  if (per_sm > 0 && cycles > 0) {
    const double sm_cycles = (double)cycles * (double)((8 + per_sm - 1) / per_sm);
    out[1] = ops / ((double)nsm * sm_cycles);
    out[3] = sm_cycles / (ms * 1e-3) / 1e6;
  }
  return 0;
}
