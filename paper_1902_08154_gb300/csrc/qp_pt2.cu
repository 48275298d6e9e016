// qp_pt2.cu -- C ABI of the EN-PT2 + selection sweep (include/qp_pt2.h):
// context set-up, input validation, generator ranking, the persistent sweep
// launch, the fixed-order E_PT2 reduction and the merge of the selection.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_segmented_radix_sort.cuh>
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "../../include/qp_pt2.h"
#include "common.cuh"

namespace qp {
cudaError_t launch_prep(int nint, const SweepParams& p, int slots, cudaStream_t st);
cudaError_t launch_batch(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);
int batch_blocks_per_sm(int nint, int mixed, size_t smem);
int sweep_threads();
cudaError_t launch_batch_grad(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_grad_gen(int nint, const SweepParams& p, int ngen, cudaStream_t st);
size_t states_smem(int max_cells, int nst);
int batch_blocks_per_sm_states(int nint, size_t smem);
cudaError_t launch_batch_states(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_reduce_items(const SweepParams& p, cudaStream_t st);
cudaError_t launch_reduce_items_multi(const SweepParams* ps, int n, int max_slots, cudaStream_t st);
cudaError_t launch_wave_multi(int nint, int mixed, const MultiWave& m, const MultiWaveInline& mi, int total_slots,
                              int grid, size_t smem, cudaStream_t st);
cudaError_t launch_compact_multi(int nint, int mixed, const SweepParams* ps, int n, int grid, cudaStream_t st);
int batch_multi_blocks_per_sm(int nint, int mixed, size_t smem);
}  // namespace qp

using namespace qp;

static thread_local std::string g_last_error;

static int fail(int code, const std::string& msg) {
  g_last_error = msg;
  return code;
}

#define CUDA_TRY(expr)                                                                     \
  do {                                                                                     \
    cudaError_t e_ = (expr);                                                               \
    if (e_ != cudaSuccess)                                                                 \
      return fail(e_ == cudaErrorMemoryAllocation ? QP_ENOMEM : QP_ECUDA,                  \
                  std::string(#expr) + ": " + cudaGetErrorString(e_));                     \
  } while (0)

// device error flags
// (16 and 32: the no-allocation entry point's symmetry check, the selection's
// candidate space; 64: coefficients times integrals beyond the exact
// accumulator's range)
enum : int { kErrOcc = 1, kErrDup = 2, kErrCoef = 4, kErrBucket = 8, kErrRange = 64, kErrTimeout = 128 };

// device memory allowed for the per-generator records and buckets of a wave
static const size_t kWaveBudget = (size_t)4 << 30;

// ---------------------------------------------------------------------------
// Small kernels
// ---------------------------------------------------------------------------
// The integrals in the batch kernel's four-index layout (eri4_index):
// entry i = ((p * norb + r) * norb + q) * norb + s holds (pq|rs); the FP32
// copy for the mixed-precision numerator when e4f is set.
__global__ void eri4_kernel(int norb, const double* eri, double* e4d, float* e4f) {
  const int64_t n = norb, i = blockIdx.x * 256ll + threadIdx.x;
  if (i >= n * n * n * n) return;
  const int s = (int)(i % n), q = (int)((i / n) % n), r = (int)((i / (n * n)) % n), p = (int)(i / (n * n * n));
  const double v = eri[qp::eri_index(p, q, r, s)];
  e4d[i] = v;
  if (e4f) e4f[i] = (float)v;
}

__global__ void to_f32_kernel(int64_t n, const double* in, float* out) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = (float)in[i];
}

__global__ void jk_kernel(int norb, const double* eri, double* Jm, double* Km) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= norb * norb) return;
  int p = x / norb, q = x % norb;
  Jm[x] = eri[eri_index(p, p, q, q)];
  Km[x] = eri[eri_index(p, q, q, p)];
}

// Occupation counts, bits beyond norb, finite coefficients; key hashes for
// the duplicate check; generator sort keys.
__global__ void validate_kernel(int64_t ndet, int nint, int norb, int na, int nb, const uint64_t* dets,
                            const double* coefs, unsigned long long* hkey, int32_t* hidx,
                            unsigned long long* rkey, int32_t* ridx, int* err, unsigned long long* cmax) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndet) return;
  const int nw = 2 * nint;
  const uint64_t* d = dets + i * nw;
  int bad = 0;
  uint64_t hk = 0;
  for (int s = 0; s < 2; s++) {
    int n = 0;
    for (int w = 0; w < nint; w++) {
      uint64_t x = d[s * nint + w];
      n += __popcll(x);
      int lo = norb - 64 * w;  // bits >= lo of this word are beyond norb
      if (lo < 64) {
        uint64_t beyond = lo <= 0 ? ~0ull : ~((1ull << lo) - 1);
        if (x & beyond) bad = 1;
      }
    }
    if (n != (s == 0 ? na : nb)) bad = 1;
  }
  for (int w = 0; w < nw; w++) hk = splitmix64(hk ^ d[w]);
  if (bad) atomicOr(err, kErrOcc);
  const double c = coefs[i];
  if (!isfinite(c)) atomicOr(err, kErrCoef);
  else atomicMax(cmax, (unsigned long long)__double_as_longlong(fabs(c)));  // max |c_I|, as bits
  hkey[i] = hk;
  hidx[i] = (int32_t)i;
  // decreasing c^2 == increasing ~bits(c*c); the radix sort is stable, so
  // ties keep increasing input index
  const double c2 = c * c;
  rkey[i] = ~(unsigned long long)__double_as_longlong(c2);
  ridx[i] = (int32_t)i;
}

// Bits of max |x| over n values (non-negative doubles order as their bits).
__global__ void absmax_kernel(int64_t n, const double* x, unsigned long long* out) {
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(x[i]));
    m = b > m ? b : m;
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0) atomicMax(out, m);
}

__global__ void dup_kernel(int64_t ndet, int nint, const uint64_t* dets, const unsigned long long* hs,
                           const int32_t* hi, int* err) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ndet) return;
  const int nw = 2 * nint;
  for (int64_t j = i + 1; j < ndet && hs[j] == hs[i]; j++) {
    bool same = true;
    for (int w = 0; w < nw; w++) same &= dets[(int64_t)hi[i] * nw + w] == dets[(int64_t)hi[j] * nw + w];
    if (same) atomicOr(err, kErrDup);
  }
}

__global__ void rank_kernel(int64_t ndet, const int32_t* order, int32_t* rank_of) {
  int64_t g = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (g < ndet) rank_of[order[g]] = (int32_t)g;
}

struct DevResult {
  double e_pt2, s2;
  long long na, ncon;
};

// Several states: every coefficient finite, and per state (blockIdx.y) the
// bits of max_I |c_Is| (non-negative doubles order as their bit patterns).
__global__ void state_scan_kernel(int64_t ndet, const double* coefs, unsigned long long* cmax, int* err) {
  const int s = blockIdx.y;
  unsigned long long m = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < ndet; i += (int64_t)gridDim.x * blockDim.x) {
    const double c = coefs[(size_t)s * ndet + i];
    if (!isfinite(c)) atomicOr(err, kErrCoef);
    else {
      const unsigned long long b = (unsigned long long)__double_as_longlong(fabs(c));
      m = b > m ? b : m;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    const unsigned long long v = __shfl_xor_sync(0xffffffffu, m, o);
    m = v > m ? v : m;
  }
  if ((threadIdx.x & 31) == 0 && m) atomicMax(&cmax[s], m);
}

// One block: fixed-order sums over generators (rank order), each thread a
// contiguous slice with Neumaier compensation, then a fixed tree.
__global__ void finalize_kernel(int64_t ndet, const double* eps, const double* s2, const long long* na,
                                const long long* nc, DevResult* out) {
  __shared__ double se[1024], ce[1024], ss[1024];
  __shared__ long long sa[1024], sc[1024];
  const int t = threadIdx.x, nt = blockDim.x;
  const int64_t per = (ndet + nt - 1) / nt;
  const int64_t b = t * per, e = (b + per < ndet) ? b + per : ndet;
  double s = 0, c = 0, q = 0;
  long long x = 0, y = 0;
  for (int64_t i = b; i < e; i++) {
    double v = eps[i], tt = s + v;
    if (fabs(s) >= fabs(v)) c += (s - tt) + v;
    else c += (v - tt) + s;
    s = tt;
    q += s2[i];
    x += na[i];
    y += nc[i];
  }
  se[t] = s;
  ce[t] = c;
  ss[t] = q;
  sa[t] = x;
  sc[t] = y;
  __syncthreads();
  for (int o = nt / 2; o > 0; o >>= 1) {
    if (t < o) {
      se[t] += se[t + o];
      ce[t] += ce[t + o];
      ss[t] += ss[t + o];
      sa[t] += sa[t + o];
      sc[t] += sc[t + o];
    }
    __syncthreads();
  }
  if (t == 0) {
    out->e_pt2 = se[0] + ce[0];
    out->s2 = ss[0];
    out->na = sa[0];
    out->ncon = sc[0];
  }
}

// Gather the CTAs' selection buffers, dropping entries below the global
// threshold (they cannot be among the k best).
__global__ void gather_kernel(int grid, int nint, int64_t cap, const int* tk_cnt, const double* tk_e,
                              const double* tk_a, const uint64_t* tk_key, const unsigned long long* tau,
                              double* ce, double* ca, uint64_t* ck, int* ncand, int64_t cand_cap, int* err) {
  const int b = blockIdx.x;
  const int nw = 2 * nint;
  const int n = tk_cnt[b];
  const unsigned long long t = *tau;
  for (int i = threadIdx.x; i < n; i += blockDim.x) {
    const size_t src = (size_t)b * cap + i;
    const double e = tk_e[src];
    if ((unsigned long long)__double_as_longlong(fabs(e)) < t) continue;
    const int o = atomicAdd(ncand, 1);
    if (o >= cand_cap) {  // more candidates than the space planned for them
      atomicOr(err, 32);
      atomicSub(ncand, 1);
      continue;
    }
    ce[o] = e;
    ca[o] = tk_a[src];
    for (int w = 0; w < nw; w++) ck[(size_t)o * nw + w] = tk_key[src * nw + w];
  }
}

// sort key of pass w: w < nw: key word w; w == nw: ~bits(|e|)
__global__ void sortkey_kernel(int n, int nint, int w, const double* ce, const uint64_t* ck,
                               const int32_t* perm, unsigned long long* keys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nw = 2 * nint, j = perm[i];
  keys[i] = (w < nw) ? ck[(size_t)j * nw + w] : ~(unsigned long long)__double_as_longlong(fabs(ce[j]));
}

__global__ void iota_kernel(int n, int32_t* v) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) v[i] = i;
}

__global__ void select_out_kernel(int n, int nint, const int32_t* perm, const double* ce, const double* ca,
                                  const uint64_t* ck, uint64_t* sel, double* se, double* sn) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int nw = 2 * nint, j = perm[i];
  if (sel)
    for (int w = 0; w < nw; w++) sel[(size_t)i * nw + w] = ck[(size_t)j * nw + w];
  if (se) se[i] = ce[j];
  if (sn) sn[i] = ca[j];
}

// ---------------------------------------------------------------------------
// Context
// ---------------------------------------------------------------------------
struct Buf {
  void* p = nullptr;
  size_t n = 0;
  int grow(size_t bytes) {
    if (bytes <= n) return QP_OK;
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
    size_t want = bytes < 256 ? 256 : bytes;
    cudaError_t e = cudaMalloc(&p, want);
    if (e != cudaSuccess) {
      p = nullptr;
      return fail(e == cudaErrorMemoryAllocation ? QP_ENOMEM : QP_ECUDA,
                  std::string("cudaMalloc: ") + cudaGetErrorString(e));
    }
    n = want;
    return QP_OK;
  }
  template <typename T>
  T* as() const { return reinterpret_cast<T*>(p); }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    n = 0;
  }
};

struct qp_pt2_ctx {
  int norb, nalpha, nbeta, nint, nel, nbat;
  int64_t P;
  qp_pt2_config cfg;
  cudaStream_t st;
  int device, nsm;
  int max_cells, bps, grid;
  int ntile;  // row tiles of the opposite-spin batches (1: not split)
  int tgt_on = 0, tgt_max_exc = -1;  // target space (qp_pt2_set_target)
  uint64_t tgt_ref[4] = {0, 0, 0, 0}, tgt_core[4] = {0, 0, 0, 0}, tgt_del[4] = {0, 0, 0, 0};
  size_t smem;
  double *d_h = nullptr, *d_eri = nullptr, *d_J = nullptr, *d_K = nullptr;
  float *d_h32 = nullptr, *d_eri32 = nullptr;  // mixed precision only
  double* d_eri4 = nullptr;                      // four-index layout (eri4_index)
  float* d_eri4_32 = nullptr;                    // its FP32 copy, mixed precision only
  unsigned long long* d_hmax = nullptr;        // bits of max |h|, max |(pq|rs)|
  // workspace
  Buf in_dets, in_coefs, hkey, hkey2, hidx, hidx2, rkey, rkey2, order, rank_of, cub_tmp;
  Buf eps, s2, na, ncon, acc, res;
  Buf meta, r_words, r_coef, r_hmask, r_part, r_flag, b_ofs, e_hp, e_rec, b_dead, queues, it_sum;
  Buf tk_e, tk_a, tk_key, tk_cnt, tk_tau, sel_hist, gen_list, gen_out, st_cmax;
  Buf cand_e, cand_a, cand_key, skey, skey2, perm, perm2, cub_tmp2;
  Buf out_sel, out_e, out_num, out_eps, out_na, out_ncon, out_rank;
  Buf g_dh, g_deri, g_wF, g_wH;
  int grad_grid = 0;
  int64_t launches = 0;
  cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};  // call start, sweep start, sweep end
  cudaEvent_t ev_end = nullptr;
  bool timed = false;
};

namespace qp {
int ctx_view(const qp_pt2_ctx* x, CtxView* v) {
  if (!x || !v) return fail(QP_EINVAL, "ctx is NULL");
  v->norb = x->norb;
  v->nalpha = x->nalpha;
  v->nbeta = x->nbeta;
  v->nint = x->nint;
  v->nel = x->nel;
  v->device = x->device;
  v->h = x->d_h;
  v->eri = x->d_eri;
  v->Jm = x->d_J;
  v->Km = x->d_K;
  v->st = x->st;
  return QP_OK;
}
int report(int code, const char* msg) { return fail(code, msg); }
}  // namespace qp

// NVTX range over one phase of a call (validation, a wave of the sweep, the
// selection merge), visible on the CPU timeline of a profiler; it costs
// nothing when no tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  void next(const char* name) {  // close this phase, open the next one
    nvtxRangePop();
    nvtxRangePushA(name);
  }
  ~NvtxRange() { nvtxRangePop(); }
};

// Renormalised PT2 (Sec. "Renormalized PT2"): with sum_e_over_d = sum A^2/D^2
// = -dSigma/dE at E0, Z = 1/(1 + sum_e_over_d) and E = E0 + Z E_PT2.
static void set_rpt2(qp_pt2_result& r, double e0) {
  r.z = 1.0 / (1.0 + r.sum_e_over_d);
  r.e_rpt2 = e0 + r.z * r.e_pt2;
}

// accumulator block layout (unsigned long long words)
enum { kAccDigest0 = 0, kAccDigest1, kAccMinDen, kAccTiny, kAccTau, kAccQueue, kAccErr, kAccNcand, kAccCmax, kAccT0, kAccWords };

static bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Cells of the largest work item when the opposite-spin batches are split
// into t tiles of rows.
static int cells_for_tile(int norb, int n_alpha, int n_beta, int t) {
  const int va = norb - n_alpha, vb = norb - n_beta;
  int m = (n_alpha > 0 && n_beta > 0) ? ((va + t - 1) / t) * vb : 0;
  const int others[4] = {va, vb, va * (va - 1) / 2, vb * (vb - 1) / 2};
  for (int o : others) m = o > m ? o : m;
  return m < 1 ? 1 : m;
}

extern "C" int qp_pt2_create(qp_pt2_ctx** out, int norb, int n_alpha, int n_beta, const double* h,
                             const double* eri, const qp_pt2_config* cfg) {
  if (!out) return fail(QP_EINVAL, "out is NULL");
  *out = nullptr;
  if (norb < 1 || norb > kMaxOrb) return fail(QP_EINVAL, "norb must be in [1, 128]");
  if (n_alpha < 0 || n_beta < 0 || n_alpha > norb || n_beta > norb)
    return fail(QP_EINVAL, "electron counts out of range");
  if (n_alpha + n_beta > kMaxElec) return fail(QP_EINVAL, "more than 64 electrons");
  if (!h || !eri) return fail(QP_EINVAL, "h or eri is NULL");
  qp_pt2_config c{};
  if (cfg) c = *cfg;
  if (c.precision != QP_FP64 && c.precision != QP_MIXED) return fail(QP_EINVAL, "unknown precision");
  if (c.threads != 0 && c.threads != sweep_threads())
    return fail(QP_ENOTSUP, "threads per CTA is fixed at 256 in this library");
  const int64_t M = (int64_t)norb * (norb + 1) / 2, P = M * (M + 1) / 2;
  // symmetry of h (host copy either way)
  std::vector<double> hh((size_t)norb * norb);
  if (is_device_ptr(h)) {
    if (cudaMemcpy(hh.data(), h, sizeof(double) * norb * norb, cudaMemcpyDeviceToHost) != cudaSuccess)
      return fail(QP_ECUDA, "copy of h failed");
  } else {
    memcpy(hh.data(), h, sizeof(double) * norb * norb);
  }
  for (int p = 0; p < norb; p++)
    for (int q = 0; q < p; q++)
      if (!(fabs(hh[(size_t)p * norb + q] - hh[(size_t)q * norb + p]) <= 1e-12))
        return fail(QP_ESYM, "h is not symmetric");
  qp_pt2_ctx* x = new (std::nothrow) qp_pt2_ctx();
  if (!x) return fail(QP_ENOMEM, "host allocation failed");
  x->norb = norb;
  x->nalpha = n_alpha;
  x->nbeta = n_beta;
  x->nint = (norb - 1) / 64 + 1;
  x->nel = n_alpha + n_beta;
  x->nbat = x->nel + x->nel * (x->nel - 1) / 2;
  x->P = P;
  x->cfg = c;
  x->st = (cudaStream_t)c.stream;
  auto bail = [&](int code, const char* what) {
    qp_pt2_destroy(x);
    return fail(code, what);
  };
  if (c.shard_count < 0 || c.shard_index < 0 || (c.shard_count > 0 && c.shard_index >= c.shard_count))
    return bail(QP_EINVAL, "shard_index must lie in [0, shard_count)");
  if (c.shard_count == 0) {
    x->cfg.shard_count = 1;
    x->cfg.shard_index = 0;
  }
  if (cudaGetDevice(&x->device) != cudaSuccess) return bail(QP_ECUDA, "no CUDA device");
  for (int i = 0; i < 3; i++)
    if (cudaEventCreate(&x->ev[i]) != cudaSuccess) return bail(QP_ECUDA, "cudaEventCreate failed");
  if (cudaEventCreate(&x->ev_end) != cudaSuccess) return bail(QP_ECUDA, "cudaEventCreate failed");
  cudaDeviceGetAttribute(&x->nsm, cudaDevAttrMultiProcessorCount, x->device);
  if (cudaMalloc(&x->d_h, sizeof(double) * norb * norb) != cudaSuccess ||
      cudaMalloc(&x->d_eri, sizeof(double) * P) != cudaSuccess ||
      cudaMalloc(&x->d_J, sizeof(double) * norb * norb) != cudaSuccess ||
      cudaMalloc(&x->d_K, sizeof(double) * norb * norb) != cudaSuccess)
    return bail(QP_ENOMEM, "device allocation of the integrals failed");
  if (cudaMemcpyAsync(x->d_h, hh.data(), sizeof(double) * norb * norb, cudaMemcpyHostToDevice, x->st) !=
          cudaSuccess ||
      cudaMemcpyAsync(x->d_eri, eri, sizeof(double) * P, cudaMemcpyDefault, x->st) != cudaSuccess)
    return bail(QP_ECUDA, "copy of the integrals failed");
  jk_kernel<<<(norb * norb + 255) / 256, 256, 0, x->st>>>(norb, x->d_eri, x->d_J, x->d_K);
  if (cudaMalloc(&x->d_hmax, 2 * sizeof(unsigned long long)) != cudaSuccess)
    return bail(QP_ENOMEM, "device allocation failed");
  if (cudaMemsetAsync(x->d_hmax, 0, 2 * sizeof(unsigned long long), x->st) != cudaSuccess)
    return bail(QP_ECUDA, "cudaMemsetAsync failed");
  absmax_kernel<<<(norb * norb + 255) / 256, 256, 0, x->st>>>((int64_t)norb * norb, x->d_h, x->d_hmax);
  absmax_kernel<<<(unsigned)std::min<int64_t>((P + 255) / 256, 4096), 256, 0, x->st>>>(P, x->d_eri, x->d_hmax + 1);
  if (c.precision == QP_MIXED) {
    if (cudaMalloc(&x->d_h32, sizeof(float) * norb * norb) != cudaSuccess ||
        cudaMalloc(&x->d_eri32, sizeof(float) * P) != cudaSuccess)
      return bail(QP_ENOMEM, "device allocation of the FP32 integrals failed");
    to_f32_kernel<<<(unsigned)((norb * norb + 255) / 256), 256, 0, x->st>>>(norb * norb, x->d_h, x->d_h32);
    to_f32_kernel<<<(unsigned)((P + 255) / 256), 256, 0, x->st>>>(P, x->d_eri, x->d_eri32);
  }
  {  // the four-index layout of the numerator gathers (12 norb^4 bytes in mixed precision, 8 in FP64)
    const int64_t n4 = (int64_t)norb * norb * norb * norb;
    if (cudaMalloc(&x->d_eri4, sizeof(double) * n4) != cudaSuccess ||
        (c.precision == QP_MIXED && cudaMalloc(&x->d_eri4_32, sizeof(float) * n4) != cudaSuccess))
      return bail(QP_ENOMEM, "device allocation of the four-index integrals failed");
    eri4_kernel<<<(unsigned)((n4 + 255) / 256), 256, 0, x->st>>>(norb, x->d_eri, x->d_eri4, x->d_eri4_32);
  }
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(x->st) != cudaSuccess)
    return bail(QP_ECUDA, "integral tables failed");
  if (c.tile < 0) return bail(QP_EINVAL, "tile must be >= 0");
  if (c.work_chunk < 0) return bail(QP_EINVAL, "work_chunk must be >= 0");
  if (!(c.timeout_s >= 0.0)) return bail(QP_EINVAL, "timeout_s must be >= 0");
  // cells of the largest work item when the opposite-spin batches are split
  // into t tiles of rows
  const int va = norb - n_alpha;
  auto cells_tiled = [&](int t) { return cells_for_tile(norb, n_alpha, n_beta, t); };
  x->ntile = 1;
  if (c.tile > 0) {
    x->ntile = (n_alpha > 0 && n_beta > 0) ? std::min(c.tile, std::max(va, 1)) : 1;
  }
  x->max_cells = cells_tiled(x->ntile);
  x->smem = sweep_smem(x->max_cells);
  int bps = batch_blocks_per_sm(x->nint, c.precision == QP_MIXED, x->smem);
  if (c.tile == 0 && x->nint == 2 && bps < 2 && n_alpha > 0 && n_beta > 0 && cells_tiled(2) < x->max_cells) {
    // the opposite-spin accumulator fits only once per SM: split those
    // batches in two tiles of rows, so that two CTAs share the SM
    x->ntile = 2;
    x->max_cells = cells_tiled(2);
    x->smem = sweep_smem(x->max_cells);
    bps = batch_blocks_per_sm(x->nint, c.precision == QP_MIXED, x->smem);
  }
  if (bps < 1) return bail(QP_ENOTSUP, "the batch accumulator does not fit in shared memory");
  if (c.blocks_per_sm > 0 && c.blocks_per_sm < bps) bps = c.blocks_per_sm;
  x->bps = bps;
  x->grid = bps * x->nsm;
  *out = x;
  return QP_OK;
}

extern "C" void qp_pt2_destroy(qp_pt2_ctx* x) {
  if (!x) return;
  for (int i = 0; i < 3; i++)
    if (x->ev[i]) cudaEventDestroy(x->ev[i]);
  if (x->ev_end) cudaEventDestroy(x->ev_end);
  cudaFree(x->d_h);
  cudaFree(x->d_eri);
  cudaFree(x->d_h32);
  cudaFree(x->d_eri32);
  cudaFree(x->d_eri4);
  cudaFree(x->d_eri4_32);
  cudaFree(x->d_J);
  cudaFree(x->d_K);
  cudaFree(x->d_hmax);
  Buf* all[] = {&x->in_dets, &x->in_coefs, &x->hkey, &x->hkey2, &x->hidx, &x->hidx2, &x->rkey, &x->rkey2,
                &x->order, &x->rank_of, &x->cub_tmp, &x->eps, &x->s2, &x->na, &x->ncon, &x->acc,
                &x->res, &x->meta, &x->r_words, &x->r_coef, &x->r_hmask, &x->r_part, &x->r_flag,
                &x->b_ofs, &x->e_hp, &x->e_rec, &x->it_sum, &x->b_dead, &x->queues, &x->tk_e, &x->tk_a, &x->tk_key, &x->tk_cnt, &x->tk_tau, &x->sel_hist, &x->gen_list, &x->gen_out, &x->cand_e, &x->cand_a, &x->cand_key, &x->skey,
                &x->skey2, &x->perm, &x->perm2, &x->cub_tmp2, &x->out_sel, &x->out_e, &x->out_num,
                &x->out_eps, &x->out_na, &x->out_ncon, &x->out_rank, &x->g_dh, &x->g_deri, &x->g_wF, &x->g_wH};
  for (Buf* b : all) b->release();
  delete x;
}

extern "C" int qp_pt2_set_target(qp_pt2_ctx* x, const uint64_t* ref, int max_exc, const uint64_t* core,
                                 const uint64_t* deleted) {
  if (!x) return fail(QP_EINVAL, "ctx is NULL");
  const int nw = 2 * x->nint;
  for (const uint64_t* a : {ref, core, deleted})
    if (a && is_device_ptr(a)) return fail(QP_EINVAL, "target-space masks must be host arrays");
  if (core && deleted)
    for (int w = 0; w < nw; w++)
      if (core[w] & deleted[w]) return fail(QP_EINVAL, "a spin orbital is both core and deleted");
  x->tgt_on = (ref || core || deleted) ? 1 : 0;
  x->tgt_max_exc = ref ? max_exc : -1;
  for (int w = 0; w < 4; w++) {
    x->tgt_ref[w] = (ref && w < nw) ? ref[w] : 0;
    x->tgt_core[w] = (core && w < nw) ? core[w] : 0;
    x->tgt_del[w] = (deleted && w < nw) ? deleted[w] : 0;
  }
  return QP_OK;
}

extern "C" int64_t qp_pt2_last_launches(const qp_pt2_ctx* x) { return x ? x->launches : 0; }

extern "C" int qp_pt2_last_timings(const qp_pt2_ctx* x, double* ms) {
  if (!x || !ms) return fail(QP_EINVAL, "ctx or ms is NULL");
  if (!x->timed) return fail(QP_EINVAL, "no completed call to time");
  float a = 0.f, b = 0.f;
  if (cudaEventElapsedTime(&a, x->ev[1], x->ev[2]) != cudaSuccess ||
      cudaEventElapsedTime(&b, x->ev[0], x->ev_end) != cudaSuccess)
    return fail(QP_ECUDA, "cudaEventElapsedTime failed");
  ms[0] = a;
  ms[1] = b;
  return QP_OK;
}

extern "C" const char* qp_pt2_strerror(int code) {
  switch (code) {
    case QP_OK: return "ok";
    case QP_EINVAL: return "invalid argument";
    case QP_EDUP: return "duplicate determinant";
    case QP_ESYM: return "h is not symmetric";
    case QP_ESINGULAR: return "a denominator E0 - H_aa is below 1e-12 in magnitude";
    case QP_ENOMEM: return "device memory allocation failed";
    case QP_ECUDA: return "CUDA runtime error";
    case QP_ENOTSUP: return "not supported by the library";
    case QP_ENOTCONV: return "Davidson did not reach the residual tolerance";
    case QP_ETIMEOUT: return "the device watchdog stopped the sweep";
    default: return "unknown error";
  }
}

extern "C" const char* qp_pt2_last_error(void) { return g_last_error.c_str(); }

extern "C" int qp_pt2_merge_results(int n, const qp_pt2_result* parts, double e0, qp_pt2_result* out) {
  if (n < 1 || !parts || !out) return fail(QP_EINVAL, "n < 1 or a NULL pointer");
  qp_pt2_result m;
  memset(&m, 0, sizeof(m));
  m.min_abs_denominator = INFINITY;
  for (int i = 0; i < n; i++) {
    const qp_pt2_result& r = parts[i];
    m.e_pt2 += r.e_pt2;
    m.sum_e_over_d += r.sum_e_over_d;
    m.n_perturbers += r.n_perturbers;
    m.n_connections += r.n_connections;
    m.n_tiny += r.n_tiny;
    m.perturber_digest[0] += r.perturber_digest[0];  // modulo 2^64
    m.perturber_digest[1] ^= r.perturber_digest[1];
    if (r.min_abs_denominator < m.min_abs_denominator) m.min_abs_denominator = r.min_abs_denominator;
  }
  set_rpt2(m, e0);
  *out = m;
  return QP_OK;
}

// Stage a caller array on the device: returns the device pointer to use.
template <typename T>
static int stage_in(qp_pt2_ctx* x, Buf& b, const T* src, size_t count, const T** dst) {
  if (is_device_ptr(src)) {
    *dst = src;
    return QP_OK;
  }
  int rc = b.grow(sizeof(T) * count);
  if (rc) return rc;
  CUDA_TRY(cudaMemcpyAsync(b.p, src, sizeof(T) * count, cudaMemcpyHostToDevice, x->st));
  *dst = b.as<T>();
  return QP_OK;
}

template <typename T>
static int out_target(Buf& b, T* user, size_t count, T** dst, bool* copy_back) {
  *copy_back = false;
  *dst = nullptr;
  if (!user) return QP_OK;
  if (is_device_ptr(user)) {
    *dst = user;
    return QP_OK;
  }
  int rc = b.grow(sizeof(T) * (count ? count : 1));
  if (rc) return rc;
  *dst = b.as<T>();
  *copy_back = true;
  return QP_OK;
}

// eps, |A_I| and connections of the listed generators (by rank).
__global__ void gather_gen_kernel(int64_t n, const int32_t* ranks, const double* eps, const double* s2,
                                  const unsigned long long* na, const unsigned long long* ncon, double* out_eps,
                                  double* out_s2, int64_t* out_na, int64_t* out_ncon) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int r = ranks[i];
  out_eps[i] = eps[r];
  out_s2[i] = s2[r];
  out_na[i] = (int64_t)na[r];
  out_ncon[i] = (int64_t)ncon[r];
}

// The sweep; with gen_ranks (host array of ngen_list distinct ranks) only
// those generators are swept and their eps, |A_I| and connections are
// written to gen_eps / gen_na / gen_ncon in list order.  nst > 0 selects
// the multi-state form: coefs holds nst states ([nst][ndet]), e0s (host)
// their energies, res nst results, and sel_e receives the multi-state
// criterion; e0 is then ignored.  The generator order is that of state 0
// (no output depends on the order).
static int eval_core(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, const double* coefs, double e0,
                     int64_t k, uint64_t* sel_dets, double* sel_e, double* sel_num, double* eps_by_rank,
                     int64_t* na_by_rank, int64_t* ncon_by_rank, int32_t* rank_of_out, qp_pt2_result* res,
                     const int32_t* gen_ranks, int64_t ngen_list, double* gen_eps, int64_t* gen_na,
                     int64_t* gen_ncon, int nst = 0, const double* e0s = nullptr, double* gen_s2 = nullptr) {
  const bool ms = nst > 0;
  const int nsts = ms ? nst : 1;
  if (!x || !res) return fail(QP_EINVAL, "ctx or res is NULL");
  if (ndet < 0 || k < 0) return fail(QP_EINVAL, "ndet and k must be non-negative");
  if (ndet > 0 && (!dets || !coefs)) return fail(QP_EINVAL, "dets or coefs is NULL");
  if (ndet >= (1ll << 31)) return fail(QP_EINVAL, "ndet must be below 2^31");
  if (ms) {
    if (nst > kMaxStates) return fail(QP_EINVAL, "nstates must be in [1, 4]");
    if (!e0s) return fail(QP_EINVAL, "e0 is NULL");
    for (int s = 0; s < nst; s++)
      if (!std::isfinite(e0s[s])) return fail(QP_EINVAL, "E0 is not finite");
    if (x->cfg.precision != QP_FP64) return fail(QP_ENOTSUP, "the multi-state sweep is FP64 only");
    e0 = e0s[0];
  }
  if (!std::isfinite(e0)) return fail(QP_EINVAL, "E0 is not finite");
  for (int s = 0; s < nsts; s++) {
    memset(res + s, 0, sizeof(*res));
    res[s].min_abs_denominator = INFINITY;
  }
  x->launches = 0;
  x->timed = false;
  if (ndet == 0) return QP_OK;
  const int nint = x->nint, nw = 2 * nint;
  cudaStream_t st = x->st;
  int rc;
  const uint64_t* d_dets;
  const double* d_coefs;
  CUDA_TRY(cudaEventRecord(x->ev[0], st));
  if ((rc = stage_in(x, x->in_dets, dets, (size_t)ndet * nw, &d_dets))) return rc;
  if ((rc = stage_in(x, x->in_coefs, coefs, (size_t)ndet * nsts, &d_coefs))) return rc;

  NvtxRange nvtx_call("qp_pt2 sweep");
  // ---- validation and generator order ----
  const size_t nd = (size_t)ndet;
  NvtxRange nvtx_phase("qp_pt2 validate and rank");
  if ((rc = x->hkey.grow(8 * nd)) || (rc = x->hkey2.grow(8 * nd)) || (rc = x->hidx.grow(4 * nd)) ||
      (rc = x->hidx2.grow(4 * nd)) || (rc = x->rkey.grow(8 * nd)) || (rc = x->rkey2.grow(8 * nd)) ||
      (rc = x->order.grow(4 * nd)) || (rc = x->rank_of.grow(4 * nd)) || (rc = x->acc.grow(8 * kAccWords)))
    return rc;
  unsigned long long* acc = x->acc.as<unsigned long long>();
  {
    unsigned long long init[kAccWords] = {0};
    init[kAccMinDen] = 0x7FF0000000000000ull;  // +inf
    CUDA_TRY(cudaMemcpyAsync(acc, init, sizeof(init), cudaMemcpyHostToDevice, st));
  }
  int* d_err = reinterpret_cast<int*>(acc + kAccErr);
  const int tb = 256;
  const int nb = (int)((ndet + tb - 1) / tb);
  validate_kernel<<<nb, tb, 0, st>>>(ndet, nint, x->norb, x->nalpha, x->nbeta, d_dets, d_coefs,
                                 x->hkey.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                 x->rkey.as<unsigned long long>(), x->rank_of.as<int32_t>(), d_err,
                                      acc + kAccCmax);
  x->launches++;
  CUDA_TRY(cudaGetLastError());
  size_t tmp1 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp1, x->hkey.as<unsigned long long>(),
                                  x->hkey2.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                  x->hidx2.as<int32_t>(), (int)ndet, 0, 64, st);
  if ((rc = x->cub_tmp.grow(tmp1))) return rc;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, tmp1, x->hkey.as<unsigned long long>(),
                                           x->hkey2.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                           x->hidx2.as<int32_t>(), (int)ndet, 0, 64, st));
  dup_kernel<<<nb, tb, 0, st>>>(ndet, nint, d_dets, x->hkey2.as<unsigned long long>(), x->hidx2.as<int32_t>(),
                                d_err);
  x->launches++;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, tmp1, x->rkey.as<unsigned long long>(),
                                           x->rkey2.as<unsigned long long>(), x->rank_of.as<int32_t>(),
                                           x->order.as<int32_t>(), (int)ndet, 0, 64, st));
  rank_kernel<<<nb, tb, 0, st>>>(ndet, x->order.as<int32_t>(), x->rank_of.as<int32_t>());
  x->launches++;
  unsigned long long hcmax[kMaxStates] = {0};
  if (ms) {  // every state's coefficients: finite, and max_I |c_Is|
    if ((rc = x->st_cmax.grow(8 * (size_t)kMaxStates))) return rc;
    CUDA_TRY(cudaMemsetAsync(x->st_cmax.p, 0, 8 * (size_t)kMaxStates, st));
    const int sb = (int)std::min<int64_t>((ndet + tb - 1) / tb, 1024);
    state_scan_kernel<<<dim3(sb, nst), tb, 0, st>>>(ndet, d_coefs, x->st_cmax.as<unsigned long long>(), d_err);
    x->launches++;
    CUDA_TRY(cudaGetLastError());
    CUDA_TRY(cudaMemcpyAsync(hcmax, x->st_cmax.p, 8 * (size_t)nst, cudaMemcpyDeviceToHost, st));
  }
  int herr = 0;
  CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (herr & kErrOcc) return fail(QP_EINVAL, "a determinant has the wrong occupation or bits beyond norb");
  if (herr & kErrCoef) return fail(QP_EINVAL, "a coefficient is not finite");
  if (herr & kErrDup) return fail(QP_EDUP, "duplicate determinant in Psi0");
  for (int s = 0; s < (ms ? nst : 0); s++)
    if (hcmax[s] == 0ull) return fail(QP_EINVAL, "a state has no nonzero coefficient");

  // ---- sweep: waves of generator slots, prep + batch kernels ----
  nvtx_phase.next("qp_pt2 waves");
  size_t smem = x->smem;
  int grid = x->grid;
  if (ms) {  // nst accumulators per CTA: fewer CTAs per SM may fit
    smem = states_smem(x->max_cells, nst);
    int bps = batch_blocks_per_sm_states(nint, smem);
    if (bps < 1) return fail(QP_ENOTSUP, "the accumulators of this many states do not fit in shared memory");
    if (bps > x->bps) bps = x->bps;
    grid = bps * x->nsm;
  }
  const int64_t cap = k > 0 ? k + x->max_cells : 1;
  const int shard_count = x->cfg.shard_count, shard_index = x->cfg.shard_index;
  const int64_t ngen = gen_ranks ? ngen_list
                                 : (ndet > shard_index) ? (ndet - shard_index + shard_count - 1) / shard_count : 0;
  if (gen_ranks) {
    if ((rc = x->gen_list.grow(4 * (size_t)(ngen > 0 ? ngen : 1))) ||
        (rc = x->gen_out.grow(32 * (size_t)(ngen > 0 ? ngen : 1))))
      return rc;
    if (ngen > 0)
      CUDA_TRY(cudaMemcpyAsync(x->gen_list.p, gen_ranks, 4 * (size_t)ngen, cudaMemcpyHostToDevice, st));
  }
  const int64_t ent_per = bucket_entries_per_record(x->nel);
  const int64_t ent_cap = (int64_t)nd * ent_per;
  const size_t dwords = (size_t)(x->nbat + 31) / 32;
  const int nper = x->nbat + (x->ntile - 1) * x->nalpha * x->nbeta;
  const size_t per_slot = wave_slot_bytes(sizeof(GenMeta), x->nel, x->nbat, nw, nd, nsts, nper);
  int64_t W = (int64_t)(kWaveBudget / per_slot);
  if (W < 1) W = 1;
  if (W > ngen) W = ngen > 0 ? ngen : 1;
  const int64_t nwaves = ngen > 0 ? (ngen + W - 1) / W : 0;
  const size_t ws = (size_t)W;
  if ((rc = x->eps.grow(8 * nd * nsts)) || (rc = x->s2.grow(8 * nd * nsts)) || (rc = x->na.grow(8 * nd)) ||
      (rc = x->ncon.grow(8 * nd)) || (rc = x->meta.grow(sizeof(GenMeta) * ws)) ||
      (rc = x->r_words.grow(8 * nd * nw * ws)) || (rc = x->r_coef.grow(8 * nd * ws * nsts)) ||
      (rc = x->r_hmask.grow(8 * nd * ws)) || (rc = x->r_part.grow(8 * nd * ws)) ||
      (rc = x->r_flag.grow(4 * nd * ws)) || (rc = x->b_ofs.grow(4 * (size_t)(x->nbat + 2) * ws)) ||
      (rc = x->e_hp.grow(16 * (size_t)ent_cap * ws)) ||
      (rc = x->e_rec.grow(4 * (size_t)ent_cap * ws)) || (rc = x->it_sum.grow(16 * (size_t)nper * nsts * ws)) ||
      (rc = x->b_dead.grow(4 * dwords * ws)) || (rc = x->queues.grow(4 * (size_t)(nwaves + 1))) ||
      (rc = x->tk_e.grow(8 * (size_t)cap * grid)) || (rc = x->tk_a.grow(8 * (size_t)cap * grid)) ||
      (rc = x->tk_key.grow(8 * (size_t)cap * grid * nw)) || (rc = x->tk_cnt.grow(4 * (size_t)grid)) ||
      (rc = x->tk_tau.grow(8 * (size_t)grid)) || (rc = x->res.grow(sizeof(DevResult) * nsts)) ||
      (rc = x->sel_hist.grow(4 * (size_t)kSelBins)))
    return rc;
  CUDA_TRY(cudaMemsetAsync(x->sel_hist.p, 0, 4 * (size_t)kSelBins, st));
  CUDA_TRY(cudaMemsetAsync(x->eps.p, 0, 8 * nd * nsts, st));
  CUDA_TRY(cudaMemsetAsync(x->s2.p, 0, 8 * nd * nsts, st));
  CUDA_TRY(cudaMemsetAsync(x->na.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->ncon.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->queues.p, 0, 4 * (size_t)(nwaves + 1), st));
  CUDA_TRY(cudaMemsetAsync(x->tk_cnt.p, 0, 4 * (size_t)grid, st));
  CUDA_TRY(cudaMemsetAsync(x->tk_tau.p, 0, 8 * (size_t)grid, st));
  SweepParams p{};
  p.norb = x->norb;
  p.nalpha = x->nalpha;
  p.nbeta = x->nbeta;
  p.nel = x->nel;
  p.nbat = x->nbat;
  p.ntile = x->ntile;
  p.nper = x->nbat + (x->ntile - 1) * x->nalpha * x->nbeta;
  p.chunk = x->cfg.work_chunk > 0 ? x->cfg.work_chunk : 1;
  p.timeout_ns = (unsigned long long)(x->cfg.timeout_s * 1e9);
  p.t_start = acc + kAccT0;
  p.hmax_bits = x->d_hmax;
  p.cmax_bits = acc + kAccCmax;
  p.it_sum = x->it_sum.as<double>();
  p.it_stride = 2;
  p.e_hp = x->e_hp.as<ulonglong2>();
  p.e_rec = x->e_rec.as<uint32_t>();
  p.tgt_on = x->tgt_on;
  p.tgt_max_exc = x->tgt_max_exc;
  for (int w = 0; w < 4; w++) {
    p.tgt_ref[w] = x->tgt_ref[w];
    p.tgt_core[w] = x->tgt_core[w];
    p.tgt_del[w] = x->tgt_del[w];
  }
  p.ndet = ndet;
  p.dets = d_dets;
  p.coefs = d_coefs;
  p.order = x->order.as<int32_t>();
  p.rank_of = x->rank_of.as<int32_t>();
  p.h = x->d_h;
  p.eri = x->d_eri;
  p.h32 = x->d_h32;
  p.eri32 = x->d_eri32;
  p.eri4 = x->d_eri4;
  p.eri4_32 = x->d_eri4_32;
  p.mixed = x->cfg.precision == QP_MIXED;
  p.Jm = x->d_J;
  p.Km = x->d_K;
  p.e0 = e0;
  p.shard_index = shard_index;
  p.shard_count = shard_count;
  p.gen_list = gen_ranks ? x->gen_list.as<int32_t>() : nullptr;
  p.meta = x->meta.as<GenMeta>();
  p.r_words = x->r_words.as<uint64_t>();
  p.r_coef = x->r_coef.as<double>();
  p.r_hmask = x->r_hmask.as<uint64_t>();
  p.r_part = x->r_part.as<uint64_t>();
  p.r_flag = x->r_flag.as<uint32_t>();
  p.b_ofs = x->b_ofs.as<int>();
  p.b_dead = x->b_dead.as<uint32_t>();
  p.ent_cap = ent_cap;
  p.eps = x->eps.as<double>();
  p.s2 = x->s2.as<double>();
  p.na = x->na.as<unsigned long long>();
  p.ncon = x->ncon.as<unsigned long long>();
  p.digest = acc + kAccDigest0;
  p.min_den_bits = acc + kAccMinDen;
  p.n_tiny = acc + kAccTiny;
  p.k = k;
  p.cap = cap;
  p.tk_e = x->tk_e.as<double>();
  p.tk_a = x->tk_a.as<double>();
  p.tk_key = x->tk_key.as<uint64_t>();
  p.tk_cnt = x->tk_cnt.as<int>();
  p.tk_tau = x->tk_tau.as<unsigned long long>();
  p.tau_bits = acc + kAccTau;
  p.sel_hist = x->sel_hist.as<unsigned int>();
  p.max_cells = x->max_cells;
  p.err = d_err;
  p.it_stride = 2 * nsts;
  if (ms) {
    p.nst = nst;
    p.rc_stride = (int64_t)(nd * ws);
    for (int s = 0; s < nst; s++) p.st_e0[s] = e0s[s];
    p.st_cmax = x->st_cmax.as<unsigned long long>();
  }
  CUDA_TRY(cudaEventRecord(x->ev[1], st));
  for (int64_t w = 0; w < nwaves; w++) {
    p.wave_start = (int)(w * W);
    p.wave_slots = (int)((ngen - w * W) < W ? (ngen - w * W) : W);
    p.last_wave = (w == nwaves - 1);
    p.queue = x->queues.as<int>() + w;
    CUDA_TRY(cudaMemsetAsync(p.it_sum, 0, sizeof(double) * (size_t)p.wave_slots * p.nper * p.it_stride, st));
    CUDA_TRY(launch_prep(nint, p, p.wave_slots, st));
    if (ms) CUDA_TRY(launch_batch_states(nint, p, grid, smem, st));
    else CUDA_TRY(launch_batch(nint, p, grid, smem, st));
    CUDA_TRY(launch_reduce_items(p, st));
    x->launches += 3;
  }
  CUDA_TRY(cudaEventRecord(x->ev[2], st));
  DevResult* dres = x->res.as<DevResult>();
  for (int s = 0; s < nsts; s++) {
    finalize_kernel<<<1, 1024, 0, st>>>(ndet, p.eps + (size_t)s * nd, p.s2 + (size_t)s * nd,
                                        reinterpret_cast<const long long*>(p.na),
                                        reinterpret_cast<const long long*>(p.ncon), dres + s);
    x->launches++;
  }
  CUDA_TRY(cudaGetLastError());

  // ---- selection merge ----
  nvtx_phase.next("qp_pt2 selection merge");
  int64_t nsel = 0;
  if (k > 0) {
    const size_t maxc = (size_t)grid * (size_t)k;
    if ((rc = x->cand_e.grow(8 * maxc)) || (rc = x->cand_a.grow(8 * maxc)) ||
        (rc = x->cand_key.grow(8 * maxc * nw)) || (rc = x->skey.grow(8 * maxc)) ||
        (rc = x->skey2.grow(8 * maxc)) || (rc = x->perm.grow(4 * maxc)) || (rc = x->perm2.grow(4 * maxc)))
      return rc;
    int* d_ncand = reinterpret_cast<int*>(acc + kAccNcand);
    gather_kernel<<<grid, 256, 0, st>>>(grid, nint, cap, p.tk_cnt, p.tk_e, p.tk_a, p.tk_key, p.tau_bits,
                                        x->cand_e.as<double>(), x->cand_a.as<double>(),
                                        x->cand_key.as<uint64_t>(), d_ncand, (int64_t)maxc, d_err);
    x->launches++;
    int ncand = 0;
    CUDA_TRY(cudaMemcpyAsync(&ncand, d_ncand, sizeof(int), cudaMemcpyDeviceToHost, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    if (ncand > 0) {
      size_t tmp2 = 0;
      cub::DeviceRadixSort::SortPairs(nullptr, tmp2, x->skey.as<unsigned long long>(),
                                      x->skey2.as<unsigned long long>(), x->perm.as<int32_t>(),
                                      x->perm2.as<int32_t>(), ncand, 0, 64, st);
      if ((rc = x->cub_tmp2.grow(tmp2))) return rc;
      const int sb = (ncand + 255) / 256;
      iota_kernel<<<sb, 256, 0, st>>>(ncand, x->perm.as<int32_t>());
      x->launches++;
      // least significant first: key words from last to first, then |e|
      for (int pass = 0; pass <= nw; pass++) {
        const int word = (pass < nw) ? (nw - 1 - pass) : nw;  // nw means |e|
        sortkey_kernel<<<sb, 256, 0, st>>>(ncand, nint, word, x->cand_e.as<double>(),
                                           x->cand_key.as<uint64_t>(), x->perm.as<int32_t>(),
                                           x->skey.as<unsigned long long>());
        x->launches++;
        CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp2.p, tmp2, x->skey.as<unsigned long long>(),
                                                 x->skey2.as<unsigned long long>(), x->perm.as<int32_t>(),
                                                 x->perm2.as<int32_t>(), ncand, 0, 64, st));
        std::swap(x->perm, x->perm2);
      }
      nsel = ncand < k ? ncand : k;
      uint64_t* d_sel;
      double *d_se, *d_sn;
      bool cb1, cb2, cb3;
      if ((rc = out_target(x->out_sel, sel_dets, (size_t)k * nw, &d_sel, &cb1)) ||
          (rc = out_target(x->out_e, sel_e, (size_t)k, &d_se, &cb2)) ||
          (rc = out_target(x->out_num, sel_num, (size_t)k, &d_sn, &cb3)))
        return rc;
      select_out_kernel<<<(int)((nsel + 255) / 256), 256, 0, st>>>((int)nsel, nint, x->perm.as<int32_t>(),
                                                                 x->cand_e.as<double>(), x->cand_a.as<double>(),
                                                                 x->cand_key.as<uint64_t>(), d_sel, d_se, d_sn);
      x->launches++;
      CUDA_TRY(cudaGetLastError());
      if (cb1) CUDA_TRY(cudaMemcpyAsync(sel_dets, d_sel, 8 * nsel * nw, cudaMemcpyDeviceToHost, st));
      if (cb2) CUDA_TRY(cudaMemcpyAsync(sel_e, d_se, 8 * nsel, cudaMemcpyDeviceToHost, st));
      if (cb3) CUDA_TRY(cudaMemcpyAsync(sel_num, d_sn, 8 * nsel, cudaMemcpyDeviceToHost, st));
    }
  }

  // ---- per-generator outputs ----
  auto copy_out = [&](void* user, const void* dev, size_t bytes) -> int {
    if (!user) return QP_OK;
    CUDA_TRY(cudaMemcpyAsync(user, dev, bytes, cudaMemcpyDefault, st));
    return QP_OK;
  };
  if ((rc = copy_out(eps_by_rank, p.eps, 8 * nd)) || (rc = copy_out(na_by_rank, p.na, 8 * nd)) ||
      (rc = copy_out(ncon_by_rank, p.ncon, 8 * nd)) || (rc = copy_out(rank_of_out, p.rank_of, 4 * nd)))
    return rc;
  if (gen_ranks && ngen > 0) {
    double* ge = x->gen_out.as<double>();
    double* gs = ge + ngen;
    int64_t* gn = reinterpret_cast<int64_t*>(gs + ngen);
    int64_t* gc = gn + ngen;
    gather_gen_kernel<<<(unsigned)((ngen + 255) / 256), 256, 0, st>>>(ngen, x->gen_list.as<int32_t>(), p.eps, p.s2,
                                                                       p.na, p.ncon, ge, gs, gn, gc);
    x->launches++;
    CUDA_TRY(cudaGetLastError());
    if ((rc = copy_out(gen_eps, ge, 8 * (size_t)ngen)) || (rc = copy_out(gen_na, gn, 8 * (size_t)ngen)) ||
        (rc = copy_out(gen_ncon, gc, 8 * (size_t)ngen)) || (rc = copy_out(gen_s2, gs, 8 * (size_t)ngen)))
      return rc;
  }

  DevResult hres[kMaxStates];
  unsigned long long hacc[kAccWords];
  CUDA_TRY(cudaMemcpyAsync(hres, dres, sizeof(DevResult) * nsts, cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaEventRecord(x->ev_end, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  x->timed = true;
  if (herr & kErrBucket) return fail(QP_ECUDA, "internal error: bucket capacity exceeded");
  if (herr & kErrRange)
    return fail(QP_ENOTSUP, "coefficients times integrals beyond 2^93: outside the exact accumulator's range");
  double md;
  memcpy(&md, &hacc[kAccMinDen], sizeof(md));
  for (int s = 0; s < nsts; s++) {
    res[s].e_pt2 = hres[s].e_pt2;
    res[s].sum_e_over_d = hres[s].s2;
    res[s].n_perturbers = hres[s].na;
    res[s].n_connections = hres[s].ncon;
    res[s].n_selected = nsel;
    res[s].n_tiny = (int64_t)hacc[kAccTiny];
    res[s].perturber_digest[0] = hacc[kAccDigest0];
    res[s].perturber_digest[1] = hacc[kAccDigest1];
    res[s].min_abs_denominator = md;
    set_rpt2(res[s], ms ? e0s[s] : e0);
  }
  if (herr & kErrTimeout) return fail(QP_ETIMEOUT, "the device watchdog stopped the sweep (timeout_s)");
  if (hres[0].na > 0 && md < 1e-12) return fail(QP_ESINGULAR, "a denominator E0 - H_aa is below 1e-12");
  return QP_OK;
}

extern "C" int qp_pt2_reduce_ranks(qp_pt2_ctx* x, int64_t n, const double* eps, const double* s2, const int64_t* na,
                                   const int64_t* ncon, double e0, qp_pt2_result* res) {
  if (!x || !res || !eps || !s2 || !na || !ncon) return fail(QP_EINVAL, "a NULL argument");
  if (n < 1 || n >= (1ll << 31)) return fail(QP_EINVAL, "n must lie in [1, 2^31)");
  memset(res, 0, sizeof(*res));
  res->min_abs_denominator = INFINITY;
  cudaStream_t st = x->st;
  int rc;
  const double *d_eps, *d_s2;
  const int64_t *d_na, *d_nc;
  if ((rc = stage_in(x, x->eps, eps, (size_t)n, &d_eps)) || (rc = stage_in(x, x->s2, s2, (size_t)n, &d_s2)) ||
      (rc = stage_in(x, x->na, na, (size_t)n, &d_na)) || (rc = stage_in(x, x->ncon, ncon, (size_t)n, &d_nc)) ||
      (rc = x->res.grow(sizeof(DevResult))))
    return rc;
  finalize_kernel<<<1, 1024, 0, st>>>(n, d_eps, d_s2, reinterpret_cast<const long long*>(d_na),
                                      reinterpret_cast<const long long*>(d_nc), x->res.as<DevResult>());
  CUDA_TRY(cudaGetLastError());
  DevResult h;
  CUDA_TRY(cudaMemcpyAsync(&h, x->res.p, sizeof(h), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  res->e_pt2 = h.e_pt2;
  res->sum_e_over_d = h.s2;
  res->n_perturbers = h.na;
  res->n_connections = h.ncon;
  set_rpt2(*res, e0);
  return QP_OK;
}

extern "C" int qp_pt2_eval_ex(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, const double* coefs,
                              double e0, int64_t k, uint64_t* sel_dets, double* sel_e, double* sel_num,
                              double* eps_by_rank, int64_t* na_by_rank, int64_t* ncon_by_rank,
                              int32_t* rank_of_out, qp_pt2_result* res) {
  return eval_core(x, ndet, dets, coefs, e0, k, sel_dets, sel_e, sel_num, eps_by_rank, na_by_rank, ncon_by_rank,
                   rank_of_out, res, nullptr, 0, nullptr, nullptr, nullptr);
}

extern "C" int qp_pt2_eval_gens(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, const double* coefs,
                                double e0, int64_t ngen, const int32_t* ranks, int64_t k, uint64_t* sel_dets,
                                double* sel_e, double* gen_eps, double* gen_s2, int64_t* gen_na, int64_t* gen_ncon,
                                qp_pt2_result* res) {
  if (!x || !res) return fail(QP_EINVAL, "ctx or res is NULL");
  if (ngen < 0 || (ngen > 0 && !ranks)) return fail(QP_EINVAL, "ngen is negative or ranks is NULL");
  if (ngen > ndet) return fail(QP_EINVAL, "more generators than determinants");
  if (ngen > 0 && is_device_ptr(ranks)) return fail(QP_EINVAL, "ranks must be a host array");
  {
    std::vector<int32_t> srt(ranks, ranks + ngen);
    std::sort(srt.begin(), srt.end());
    for (int64_t i = 0; i < ngen; i++) {
      if (srt[i] < 0 || srt[i] >= ndet) return fail(QP_EINVAL, "a generator rank is outside [0, ndet)");
      if (i > 0 && srt[i] == srt[i - 1]) return fail(QP_EINVAL, "a generator rank is listed twice");
    }
  }
  return eval_core(x, ndet, dets, coefs, e0, k, sel_dets, sel_e, nullptr, nullptr, nullptr, nullptr, nullptr, res,
                   ranks, ngen, gen_eps, gen_na, gen_ncon, 0, nullptr, gen_s2);
}

extern "C" int qp_pt2_eval_states(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, int nstates,
                                  const double* coefs, const double* e0, int64_t k, uint64_t* sel_dets,
                                  double* sel_crit, double* sel_num, qp_pt2_result* res) {
  if (nstates < 1) return fail(QP_EINVAL, "nstates must be in [1, 4]");
  return eval_core(x, ndet, dets, coefs, 0.0, k, sel_dets, sel_crit, sel_num, nullptr, nullptr, nullptr, nullptr,
                   res, nullptr, 0, nullptr, nullptr, nullptr, nstates, e0);
}

extern "C" int qp_pt2_eval(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, const double* coefs, double e0,
                           int64_t k, uint64_t* sel_dets, double* sel_e, qp_pt2_result* res) {
  return qp_pt2_eval_ex(x, ndet, dets, coefs, e0, k, sel_dets, sel_e, nullptr, nullptr, nullptr, nullptr,
                        nullptr, res);
}

// ---------------------------------------------------------------------------
// Gradient of E_PT2 with respect to h and the packed integrals (Psi0 and E0
// held fixed): the sweep is repeated in gradient mode, which rebuilds every
// accumulator A_alpha and scatters (2 A/D) c_J d<J|H|alpha> and
// (A/D)^2 d<alpha|H|alpha>; dE/dE0 = -sum A^2/D^2.
// ---------------------------------------------------------------------------
extern "C" int qp_pt2_grad(qp_pt2_ctx* x, int64_t ndet, const uint64_t* dets, const double* coefs, double e0,
                           double* dh, double* deri, double* de0, qp_pt2_result* res) {
  if (!x || !dh || !deri || !de0) return fail(QP_EINVAL, "ctx, dh, deri or de0 is NULL");
  if (ndet < 0) return fail(QP_EINVAL, "ndet must be non-negative");
  if (ndet > 0 && (!dets || !coefs)) return fail(QP_EINVAL, "dets or coefs is NULL");
  if (ndet >= (1ll << 31)) return fail(QP_EINVAL, "ndet must be below 2^31");
  if (!std::isfinite(e0)) return fail(QP_EINVAL, "E0 is not finite");
  if (x->cfg.precision != QP_FP64) return fail(QP_ENOTSUP, "the gradient is computed in FP64 contexts only");
  qp_pt2_result local;
  if (!res) res = &local;
  memset(res, 0, sizeof(*res));
  res->min_abs_denominator = INFINITY;
  x->launches = 0;
  x->timed = false;
  const int norb = x->norb, nint = x->nint, nw = 2 * nint;
  const size_t nh = (size_t)norb * norb, P = (size_t)x->P;
  cudaStream_t st = x->st;
  int rc;
  double* d_dh;
  double* d_deri;
  bool cb_dh, cb_eri;
  if ((rc = x->g_dh.grow(8 * nh)) || (rc = x->g_deri.grow(8 * P))) return rc;
  // gradients accumulate in library buffers, then go to the caller's
  (void)cb_dh;
  (void)cb_eri;
  d_dh = x->g_dh.as<double>();
  d_deri = x->g_deri.as<double>();
  CUDA_TRY(cudaMemsetAsync(d_dh, 0, 8 * nh, st));
  CUDA_TRY(cudaMemsetAsync(d_deri, 0, 8 * P, st));
  if (ndet == 0) {
    CUDA_TRY(cudaMemcpyAsync(dh, d_dh, 8 * nh, cudaMemcpyDefault, st));
    CUDA_TRY(cudaMemcpyAsync(deri, d_deri, 8 * P, cudaMemcpyDefault, st));
    CUDA_TRY(cudaStreamSynchronize(st));
    *de0 = 0.0;
    return QP_OK;
  }
  CUDA_TRY(cudaEventRecord(x->ev[0], st));
  const uint64_t* d_dets;
  const double* d_coefs;
  if ((rc = stage_in(x, x->in_dets, dets, (size_t)ndet * nw, &d_dets))) return rc;
  if ((rc = stage_in(x, x->in_coefs, coefs, (size_t)ndet, &d_coefs))) return rc;
  const size_t nd = (size_t)ndet;
  if ((rc = x->hkey.grow(8 * nd)) || (rc = x->hkey2.grow(8 * nd)) || (rc = x->hidx.grow(4 * nd)) ||
      (rc = x->hidx2.grow(4 * nd)) || (rc = x->rkey.grow(8 * nd)) || (rc = x->rkey2.grow(8 * nd)) ||
      (rc = x->order.grow(4 * nd)) || (rc = x->rank_of.grow(4 * nd)) || (rc = x->acc.grow(8 * kAccWords)))
    return rc;
  unsigned long long* acc = x->acc.as<unsigned long long>();
  {
    unsigned long long init[kAccWords] = {0};
    init[kAccMinDen] = 0x7FF0000000000000ull;
    CUDA_TRY(cudaMemcpyAsync(acc, init, sizeof(init), cudaMemcpyHostToDevice, st));
  }
  int* d_err = reinterpret_cast<int*>(acc + kAccErr);
  const int nb = (int)((ndet + 255) / 256);
  validate_kernel<<<nb, 256, 0, st>>>(ndet, nint, norb, x->nalpha, x->nbeta, d_dets, d_coefs,
                                      x->hkey.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                      x->rkey.as<unsigned long long>(), x->rank_of.as<int32_t>(), d_err,
                                      acc + kAccCmax);
  x->launches++;
  CUDA_TRY(cudaGetLastError());
  size_t tmp1 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp1, x->hkey.as<unsigned long long>(),
                                  x->hkey2.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                  x->hidx2.as<int32_t>(), (int)ndet, 0, 64, st);
  if ((rc = x->cub_tmp.grow(tmp1))) return rc;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, tmp1, x->hkey.as<unsigned long long>(),
                                           x->hkey2.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                           x->hidx2.as<int32_t>(), (int)ndet, 0, 64, st));
  dup_kernel<<<nb, 256, 0, st>>>(ndet, nint, d_dets, x->hkey2.as<unsigned long long>(), x->hidx2.as<int32_t>(), d_err);
  x->launches++;
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, tmp1, x->rkey.as<unsigned long long>(),
                                           x->rkey2.as<unsigned long long>(), x->rank_of.as<int32_t>(),
                                           x->order.as<int32_t>(), (int)ndet, 0, 64, st));
  rank_kernel<<<nb, 256, 0, st>>>(ndet, x->order.as<int32_t>(), x->rank_of.as<int32_t>());
  x->launches++;
  int herr = 0;
  CUDA_TRY(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  if (herr & kErrOcc) return fail(QP_EINVAL, "a determinant has the wrong occupation or bits beyond norb");
  if (herr & kErrCoef) return fail(QP_EINVAL, "a coefficient is not finite");
  if (herr & kErrDup) return fail(QP_EDUP, "duplicate determinant in Psi0");

  // waves (same layout as the sweep, no selection)
  const int grid = x->grid;
  const int shard_count = x->cfg.shard_count, shard_index = x->cfg.shard_index;
  const int64_t ngen = (ndet > shard_index) ? (ndet - shard_index + shard_count - 1) / shard_count : 0;
  const int64_t ent_per = bucket_entries_per_record(x->nel);
  const int64_t ent_cap = (int64_t)nd * ent_per;
  const size_t dwords = (size_t)(x->nbat + 31) / 32;
  const int nper = x->nbat + (x->ntile - 1) * x->nalpha * x->nbeta;
  const size_t per_slot = wave_slot_bytes(sizeof(GenMeta), x->nel, x->nbat, nw, nd, 1, nper);
  int64_t W = (int64_t)(kWaveBudget / per_slot);
  if (W < 1) W = 1;
  if (W > ngen) W = ngen > 0 ? ngen : 1;
  const int64_t nwaves = ngen > 0 ? (ngen + W - 1) / W : 0;
  const size_t wsl = (size_t)W;
  if ((rc = x->eps.grow(8 * nd)) || (rc = x->s2.grow(8 * nd)) || (rc = x->na.grow(8 * nd)) ||
      (rc = x->ncon.grow(8 * nd)) || (rc = x->meta.grow(sizeof(GenMeta) * wsl)) ||
      (rc = x->r_words.grow(8 * nd * nw * wsl)) || (rc = x->r_coef.grow(8 * nd * wsl)) ||
      (rc = x->r_hmask.grow(8 * nd * wsl)) || (rc = x->r_part.grow(8 * nd * wsl)) ||
      (rc = x->r_flag.grow(4 * nd * wsl)) || (rc = x->b_ofs.grow(4 * (size_t)(x->nbat + 2) * wsl)) ||
      (rc = x->e_hp.grow(16 * (size_t)ent_cap * wsl)) ||
      (rc = x->e_rec.grow(4 * (size_t)ent_cap * wsl)) || (rc = x->it_sum.grow(16 * (size_t)nper * wsl)) ||
      (rc = x->b_dead.grow(4 * dwords * wsl)) ||
      (rc = x->queues.grow(4 * (size_t)(nwaves + 1))) || (rc = x->tk_cnt.grow(4 * (size_t)grid)) ||
      (rc = x->tk_tau.grow(8 * (size_t)grid)) || (rc = x->res.grow(sizeof(DevResult))) ||
      (rc = x->g_wF.grow(8 * nd * 2 * norb)) || (rc = x->g_wH.grow(8 * nd)))
    return rc;
  CUDA_TRY(cudaMemsetAsync(x->eps.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->s2.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->na.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->ncon.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->queues.p, 0, 4 * (size_t)(nwaves + 1), st));
  CUDA_TRY(cudaMemsetAsync(x->tk_cnt.p, 0, 4 * (size_t)grid, st));
  CUDA_TRY(cudaMemsetAsync(x->tk_tau.p, 0, 8 * (size_t)grid, st));
  CUDA_TRY(cudaMemsetAsync(x->g_wF.p, 0, 8 * nd * 2 * norb, st));
  CUDA_TRY(cudaMemsetAsync(x->g_wH.p, 0, 8 * nd, st));
  SweepParams p{};
  p.norb = norb;
  p.nalpha = x->nalpha;
  p.nbeta = x->nbeta;
  p.nel = x->nel;
  p.nbat = x->nbat;
  p.ntile = x->ntile;
  p.nper = x->nbat + (x->ntile - 1) * x->nalpha * x->nbeta;
  p.chunk = x->cfg.work_chunk > 0 ? x->cfg.work_chunk : 1;
  p.timeout_ns = (unsigned long long)(x->cfg.timeout_s * 1e9);
  p.t_start = acc + kAccT0;
  p.hmax_bits = x->d_hmax;
  p.cmax_bits = acc + kAccCmax;
  p.it_sum = x->it_sum.as<double>();
  p.it_stride = 2;
  p.e_hp = x->e_hp.as<ulonglong2>();
  p.e_rec = x->e_rec.as<uint32_t>();
  p.tgt_on = x->tgt_on;
  p.tgt_max_exc = x->tgt_max_exc;
  for (int w = 0; w < 4; w++) {
    p.tgt_ref[w] = x->tgt_ref[w];
    p.tgt_core[w] = x->tgt_core[w];
    p.tgt_del[w] = x->tgt_del[w];
  }
  p.ndet = ndet;
  p.dets = d_dets;
  p.coefs = d_coefs;
  p.order = x->order.as<int32_t>();
  p.rank_of = x->rank_of.as<int32_t>();
  p.h = x->d_h;
  p.eri = x->d_eri;
  p.eri4 = x->d_eri4;
  p.Jm = x->d_J;
  p.Km = x->d_K;
  p.e0 = e0;
  p.shard_index = shard_index;
  p.shard_count = shard_count;
  p.meta = x->meta.as<GenMeta>();
  p.r_words = x->r_words.as<uint64_t>();
  p.r_coef = x->r_coef.as<double>();
  p.r_hmask = x->r_hmask.as<uint64_t>();
  p.r_part = x->r_part.as<uint64_t>();
  p.r_flag = x->r_flag.as<uint32_t>();
  p.b_ofs = x->b_ofs.as<int>();
  p.b_dead = x->b_dead.as<uint32_t>();
  p.ent_cap = ent_cap;
  p.eps = x->eps.as<double>();
  p.s2 = x->s2.as<double>();
  p.na = x->na.as<unsigned long long>();
  p.ncon = x->ncon.as<unsigned long long>();
  p.digest = acc + kAccDigest0;
  p.min_den_bits = acc + kAccMinDen;
  p.n_tiny = acc + kAccTiny;
  p.k = 0;
  p.cap = 1;
  p.tk_cnt = x->tk_cnt.as<int>();
  p.tk_tau = x->tk_tau.as<unsigned long long>();
  p.tau_bits = acc + kAccTau;
  p.sel_hist = x->sel_hist.as<unsigned int>();
  p.max_cells = x->max_cells;
  p.err = d_err;
  p.g_dh = d_dh;
  p.g_deri = d_deri;
  p.g_wF = x->g_wF.as<double>();
  p.g_wH = x->g_wH.as<double>();
  CUDA_TRY(cudaEventRecord(x->ev[1], st));
  for (int64_t w = 0; w < nwaves; w++) {
    p.wave_start = (int)(w * W);
    p.wave_slots = (int)((ngen - w * W) < W ? (ngen - w * W) : W);
    p.last_wave = (w == nwaves - 1);
    p.queue = x->queues.as<int>() + w;
    CUDA_TRY(cudaMemsetAsync(p.it_sum, 0, sizeof(double) * (size_t)p.wave_slots * p.nper * p.it_stride, st));
    CUDA_TRY(launch_prep(nint, p, p.wave_slots, st));
    CUDA_TRY(launch_batch_grad(nint, p, grid, x->smem, st));
    CUDA_TRY(launch_reduce_items(p, st));
    x->launches += 3;
  }
  CUDA_TRY(launch_grad_gen(nint, p, (int)ndet, st));
  x->launches++;
  CUDA_TRY(cudaEventRecord(x->ev[2], st));
  DevResult* dres = x->res.as<DevResult>();
  finalize_kernel<<<1, 1024, 0, st>>>(ndet, p.eps, p.s2, reinterpret_cast<const long long*>(p.na),
                                      reinterpret_cast<const long long*>(p.ncon), dres);
  x->launches++;
  CUDA_TRY(cudaGetLastError());
  CUDA_TRY(cudaMemcpyAsync(dh, d_dh, 8 * nh, cudaMemcpyDefault, st));
  CUDA_TRY(cudaMemcpyAsync(deri, d_deri, 8 * P, cudaMemcpyDefault, st));
  DevResult hres;
  unsigned long long hacc[kAccWords];
  CUDA_TRY(cudaMemcpyAsync(&hres, dres, sizeof(hres), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st));
  CUDA_TRY(cudaEventRecord(x->ev_end, st));
  CUDA_TRY(cudaStreamSynchronize(st));
  x->timed = true;
  res->e_pt2 = hres.e_pt2;
  res->sum_e_over_d = hres.s2;
  res->n_perturbers = hres.na;
  res->n_connections = hres.ncon;
  res->n_tiny = (int64_t)hacc[kAccTiny];
  res->perturber_digest[0] = hacc[kAccDigest0];
  res->perturber_digest[1] = hacc[kAccDigest1];
  double md;
  memcpy(&md, &hacc[kAccMinDen], sizeof(md));
  res->min_abs_denominator = md;
  *de0 = -hres.s2;
  set_rpt2(*res, e0);
  if (((int)(hacc[kAccErr] & 0xffffffffull)) & kErrRange)
    return fail(QP_ENOTSUP, "coefficients times integrals beyond 2^93: outside the exact accumulator's range");
  if (((int)(hacc[kAccErr] & 0xffffffffull)) & kErrTimeout)
    return fail(QP_ETIMEOUT, "the device watchdog stopped the sweep (timeout_s)");
  if (hres.na > 0 && md < 1e-12) return fail(QP_ESINGULAR, "a denominator E0 - H_aa is below 1e-12");
  return QP_OK;
}

// ---------------------------------------------------------------------------
// Batched sweeps.  Many contexts' sweeps (each its own Hamiltonian and Psi0)
// are planned once (workspaces allocated outside any capture) and enqueued
// without host synchronisation on forked streams inside one stream capture;
// the resulting CUDA graph runs all of them concurrently per launch.  Input
// checks that the ordinary sweep does on the host are made on the device and
// reported after the run; the final sort uses a segmented radix sort whose
// segment end (the candidate count) lives on the device.
// ---------------------------------------------------------------------------
__global__ void init_acc_kernel(unsigned long long* acc) {
  const int t = threadIdx.x;
  if (t < kAccWords) acc[t] = (t == kAccMinDen) ? 0x7FF0000000000000ull : 0ull;
}

__global__ void seg_bounds_kernel(const int* ncand, int* be) {
  be[0] = 0;
  be[1] = *ncand;
}

__global__ void sortkey_dev_kernel(int cap, const int* ncand, int nint, int w, const double* ce, const uint64_t* ck,
                                   const int32_t* perm, unsigned long long* keys) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cap || i >= *ncand) return;
  const int nw = 2 * nint, j = perm[i];
  keys[i] = (w < nw) ? ck[(size_t)j * nw + w] : ~(unsigned long long)__double_as_longlong(fabs(ce[j]));
}

__global__ void select_out_dev_kernel(int64_t k, const int* ncand, int nint, const int32_t* perm, const double* ce,
                                      const uint64_t* ck, uint64_t* sel, double* se, unsigned long long* nsel) {
  const int64_t n = (int64_t)(*ncand) < k ? (int64_t)(*ncand) : k;
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i == 0) *nsel = (unsigned long long)n;
  if (i >= n) return;
  const int nw = 2 * nint, j = perm[i];
  for (int w = 0; w < nw; w++) sel[(size_t)i * nw + w] = ck[(size_t)j * nw + w];
  se[i] = ce[j];
}

struct BatchInst {
  qp_pt2_ctx* x;
  int64_t ndet, k;
  const uint64_t* dets;
  const double* coefs;
  double e0;
  uint64_t* sel;
  double* se;
  int grid;
  int ntile, nper, max_cells;  // launch shape of this instance's work items
  size_t smem;
  int64_t W, nwaves, ngen, ent_cap, cap;
  size_t maxc, tmp1, tmp2;
  double work;
  int group;        // fused form: the instance's group
  SweepParams p;    // the sweep's parameters (the wave fields are set per wave)
};

// Fused form: the instances of one word count and precision, swept by one
// persistent launch per wave.
struct FusedGroup {
  int nint = 1, mixed = 0;
  std::vector<int> members;  // instance indices, largest work items first
  int grid = 0, nwaves = 0, chunk = 1;
  int npw = 0;  // the most pieces in a wave (row length of the tables)
  size_t smem = 0;
  unsigned long long timeout_ns = 0;
  std::vector<int> nact, slots, max_slots;  // per wave: pieces, slots, most slots of a piece
  void* pool = nullptr;           // the waves' records and buckets, laid out per wave
  std::vector<SweepParams> hps;   // host copy of the wave rows of d_ps
  std::vector<long long> hitem;   // host copy of d_item_ofs
  SweepParams* d_ps = nullptr;    // [nwaves + 1][nm]: the wave's pieces; row nwaves: all members
  int* d_slot_ofs = nullptr;      // [nwaves][nm + 1]
  long long* d_item_ofs = nullptr;  // [nwaves][nm + 1]
  unsigned long long* d_words = nullptr;  // [nwaves][npw] pieces' item counters, then the watchdog's start time
  int* d_err = nullptr;
  cudaStream_t st = nullptr;
  cudaEvent_t done = nullptr;
};

struct qp_pt2_batch {
  std::vector<BatchInst> inst;
  std::vector<FusedGroup> groups;
  bool fused = false;
  cudaStream_t main = nullptr;
  bool own_main = false;
  std::vector<cudaStream_t> br;
  std::vector<cudaEvent_t> ev;
  cudaEvent_t fork = nullptr, t0 = nullptr, t1 = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
};

// Device bytes of one generator slot of instance b's waves.
static size_t inst_slot_bytes(const BatchInst& b) {
  const qp_pt2_ctx* x = b.x;
  return wave_slot_bytes(sizeof(GenMeta), x->nel, x->nbat, 2 * x->nint, (size_t)b.ndet, 1, b.nper);
}

// Workspaces of instance b: W slots per wave (W_fixed > 0) or as many as
// wave_budget bytes hold.
static int plan_instance(BatchInst& b, size_t wave_budget, int64_t W_fixed, bool pooled = false) {
  qp_pt2_ctx* x = b.x;
  const int nint = x->nint, nw = 2 * nint;
  const size_t nd = (size_t)b.ndet;
  int rc;
  if (b.grid <= 0) b.grid = x->grid;
  const int grid = b.grid;
  b.cap = b.k > 0 ? b.k + b.max_cells : 1;
  // every CTA may hold up to k candidates when no CTA has filled its buffer
  b.maxc = (size_t)grid * (size_t)(b.k > 0 ? b.k : 1);
  b.ngen = b.ndet;
  const int64_t ent_per = bucket_entries_per_record(x->nel);
  b.ent_cap = (int64_t)nd * ent_per;
  const size_t dwords = (size_t)(x->nbat + 31) / 32;
  const int nper = b.nper;
  b.W = W_fixed > 0 ? W_fixed : (int64_t)(wave_budget / inst_slot_bytes(b));
  if (b.W < 1) b.W = 1;
  if (b.W > b.ngen) b.W = b.ngen;
  b.nwaves = (b.ngen + b.W - 1) / b.W;
  const size_t ws = (size_t)b.W;
  b.tmp1 = 0;
  b.tmp2 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, b.tmp1, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                  (int32_t*)nullptr, (int32_t*)nullptr, (int)b.ndet, 0, 64, x->st);
  cub::DeviceSegmentedRadixSort::SortPairs(nullptr, b.tmp2, (unsigned long long*)nullptr,
                                           (unsigned long long*)nullptr, (int32_t*)nullptr, (int32_t*)nullptr,
                                           (int)b.maxc, 1, (int*)nullptr, (int*)nullptr, 0, 64, x->st);
  if ((rc = x->hkey.grow(8 * nd)) || (rc = x->hkey2.grow(8 * nd)) || (rc = x->hidx.grow(4 * nd)) ||
      (rc = x->hidx2.grow(4 * nd)) || (rc = x->rkey.grow(8 * nd)) || (rc = x->rkey2.grow(8 * nd)) ||
      (rc = x->order.grow(4 * nd)) || (rc = x->rank_of.grow(4 * nd)) || (rc = x->acc.grow(8 * kAccWords)) ||
      (rc = x->cub_tmp.grow(b.tmp1)) || (rc = x->cub_tmp2.grow(b.tmp2 + 256)) || (rc = x->eps.grow(8 * nd)) ||
      (rc = x->s2.grow(8 * nd)) || (rc = x->na.grow(8 * nd)) || (rc = x->ncon.grow(8 * nd)))
    return rc;
  // the wave's per-slot records and buckets: the instance's own (pooled: in
  // the batch's pool, laid out per wave)
  if (!pooled &&
      ((rc = x->meta.grow(sizeof(GenMeta) * ws)) || (rc = x->r_words.grow(8 * nd * nw * ws)) ||
      (rc = x->r_coef.grow(8 * nd * ws)) || (rc = x->r_hmask.grow(8 * nd * ws)) ||
      (rc = x->r_part.grow(8 * nd * ws)) || (rc = x->r_flag.grow(4 * nd * ws)) ||
      (rc = x->b_ofs.grow(4 * (size_t)(x->nbat + 2) * ws)) || (rc = x->e_hp.grow(16 * (size_t)b.ent_cap * ws)) ||
      (rc = x->e_rec.grow(4 * (size_t)b.ent_cap * ws)) ||
      (rc = x->it_sum.grow(16 * (size_t)nper * ws)) || (rc = x->b_dead.grow(4 * dwords * ws))))
    return rc;
  if ((rc = x->queues.grow(4 * (size_t)(b.nwaves + 1))) ||
      (rc = x->tk_e.grow(8 * (size_t)b.cap * grid)) || (rc = x->tk_a.grow(8 * (size_t)b.cap * grid)) ||
      (rc = x->tk_key.grow(8 * (size_t)b.cap * grid * nw)) || (rc = x->tk_cnt.grow(4 * (size_t)grid)) ||
      (rc = x->tk_tau.grow(8 * (size_t)grid)) || (rc = x->res.grow(sizeof(DevResult))) ||
      (rc = x->sel_hist.grow(4 * (size_t)kSelBins)) || (rc = x->cand_e.grow(8 * b.maxc)) || (rc = x->cand_a.grow(8 * b.maxc)) ||
      (rc = x->cand_key.grow(8 * b.maxc * nw)) || (rc = x->skey.grow(8 * b.maxc)) ||
      (rc = x->skey2.grow(8 * b.maxc)) || (rc = x->perm.grow(4 * b.maxc)) || (rc = x->perm2.grow(4 * b.maxc)))
    return rc;
  b.work = (double)b.ndet * (double)(x->nel + x->nel * (x->nel - 1) / 2) * (double)b.max_cells;
  return QP_OK;
}

// The sweep's parameters of instance b (after plan_instance).
static void make_params(BatchInst& b) {
  qp_pt2_ctx* x = b.x;
  unsigned long long* acc = x->acc.as<unsigned long long>();
  SweepParams p{};
  p.norb = x->norb;
  p.nalpha = x->nalpha;
  p.nbeta = x->nbeta;
  p.nel = x->nel;
  p.nbat = x->nbat;
  p.ntile = b.ntile;
  p.nper = b.nper;
  p.chunk = x->cfg.work_chunk > 0 ? x->cfg.work_chunk : 1;
  p.timeout_ns = (unsigned long long)(x->cfg.timeout_s * 1e9);
  p.t_start = acc + kAccT0;
  p.hmax_bits = x->d_hmax;
  p.cmax_bits = acc + kAccCmax;
  p.it_sum = x->it_sum.as<double>();
  p.it_stride = 2;
  p.e_hp = x->e_hp.as<ulonglong2>();
  p.e_rec = x->e_rec.as<uint32_t>();
  p.tgt_on = x->tgt_on;
  p.tgt_max_exc = x->tgt_max_exc;
  for (int w = 0; w < 4; w++) {
    p.tgt_ref[w] = x->tgt_ref[w];
    p.tgt_core[w] = x->tgt_core[w];
    p.tgt_del[w] = x->tgt_del[w];
  }
  p.ndet = b.ndet;
  p.dets = b.dets;
  p.coefs = b.coefs;
  p.order = x->order.as<int32_t>();
  p.rank_of = x->rank_of.as<int32_t>();
  p.h = x->d_h;
  p.eri = x->d_eri;
  p.h32 = x->d_h32;
  p.eri32 = x->d_eri32;
  p.eri4 = x->d_eri4;
  p.eri4_32 = x->d_eri4_32;
  p.mixed = x->cfg.precision == QP_MIXED;
  p.Jm = x->d_J;
  p.Km = x->d_K;
  p.e0 = b.e0;
  p.shard_index = 0;
  p.shard_count = 1;
  p.meta = x->meta.as<GenMeta>();
  p.r_words = x->r_words.as<uint64_t>();
  p.r_coef = x->r_coef.as<double>();
  p.r_hmask = x->r_hmask.as<uint64_t>();
  p.r_part = x->r_part.as<uint64_t>();
  p.r_flag = x->r_flag.as<uint32_t>();
  p.b_ofs = x->b_ofs.as<int>();
  p.b_dead = x->b_dead.as<uint32_t>();
  p.ent_cap = b.ent_cap;
  p.eps = x->eps.as<double>();
  p.s2 = x->s2.as<double>();
  p.na = x->na.as<unsigned long long>();
  p.ncon = x->ncon.as<unsigned long long>();
  p.digest = acc + kAccDigest0;
  p.min_den_bits = acc + kAccMinDen;
  p.n_tiny = acc + kAccTiny;
  p.k = b.k;
  p.cap = b.cap;
  p.tk_e = x->tk_e.as<double>();
  p.tk_a = x->tk_a.as<double>();
  p.tk_key = x->tk_key.as<uint64_t>();
  p.tk_cnt = x->tk_cnt.as<int>();
  p.tk_tau = x->tk_tau.as<unsigned long long>();
  p.tau_bits = acc + kAccTau;
  p.sel_hist = x->sel_hist.as<unsigned int>();
  p.max_cells = b.max_cells;
  p.err = reinterpret_cast<int*>(acc + kAccErr);
  b.p = p;
}

// Validation, ranking and the zeroing of the sums, on stream st.
static int enqueue_pre(BatchInst& b, cudaStream_t st) {
  qp_pt2_ctx* x = b.x;
  const int nint = x->nint;
  const int64_t ndet = b.ndet;
  const size_t nd = (size_t)ndet;
  unsigned long long* acc = x->acc.as<unsigned long long>();
  int* d_err = reinterpret_cast<int*>(acc + kAccErr);
  init_acc_kernel<<<1, 32, 0, st>>>(acc);
  CUDA_TRY(cudaMemsetAsync(x->sel_hist.p, 0, 4 * (size_t)kSelBins, st));
  const int nb = (int)((ndet + 255) / 256);
  validate_kernel<<<nb, 256, 0, st>>>(ndet, nint, x->norb, x->nalpha, x->nbeta, b.dets, b.coefs,
                                      x->hkey.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                      x->rkey.as<unsigned long long>(), x->rank_of.as<int32_t>(), d_err,
                                      acc + kAccCmax);
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, b.tmp1, x->hkey.as<unsigned long long>(),
                                           x->hkey2.as<unsigned long long>(), x->hidx.as<int32_t>(),
                                           x->hidx2.as<int32_t>(), (int)ndet, 0, 64, st));
  dup_kernel<<<nb, 256, 0, st>>>(ndet, nint, b.dets, x->hkey2.as<unsigned long long>(), x->hidx2.as<int32_t>(), d_err);
  CUDA_TRY(cub::DeviceRadixSort::SortPairs(x->cub_tmp.p, b.tmp1, x->rkey.as<unsigned long long>(),
                                           x->rkey2.as<unsigned long long>(), x->rank_of.as<int32_t>(),
                                           x->order.as<int32_t>(), (int)ndet, 0, 64, st));
  rank_kernel<<<nb, 256, 0, st>>>(ndet, x->order.as<int32_t>(), x->rank_of.as<int32_t>());
  CUDA_TRY(cudaMemsetAsync(x->eps.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->s2.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->na.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->ncon.p, 0, 8 * nd, st));
  CUDA_TRY(cudaMemsetAsync(x->queues.p, 0, 4 * (size_t)(b.nwaves + 1), st));
  CUDA_TRY(cudaMemsetAsync(x->tk_cnt.p, 0, 4 * (size_t)b.grid, st));
  CUDA_TRY(cudaMemsetAsync(x->tk_tau.p, 0, 8 * (size_t)b.grid, st));
  return QP_OK;
}

// The waves of instance b's own sweep, on stream st.
static int enqueue_waves(BatchInst& b, cudaStream_t st) {
  qp_pt2_ctx* x = b.x;
  SweepParams p = b.p;
  for (int64_t w = 0; w < b.nwaves; w++) {
    p.wave_start = (int)(w * b.W);
    p.wave_slots = (int)((b.ngen - w * b.W) < b.W ? (b.ngen - w * b.W) : b.W);
    p.last_wave = (w == b.nwaves - 1);
    p.queue = x->queues.as<int>() + w;
    CUDA_TRY(launch_prep(x->nint, p, p.wave_slots, st));  // it zeroes the wave's per-item sums
    CUDA_TRY(launch_batch(x->nint, p, b.grid, b.smem, st));
    CUDA_TRY(launch_reduce_items(p, st));
  }
  return QP_OK;
}

// The totals and the merge of the CTAs' selection buffers, on stream st.
static int enqueue_post(BatchInst& b, cudaStream_t st) {
  qp_pt2_ctx* x = b.x;
  const int nint = x->nint, nw = 2 * nint;
  const int grid = b.grid;
  const SweepParams& p = b.p;
  unsigned long long* acc = x->acc.as<unsigned long long>();
  int* d_err = reinterpret_cast<int*>(acc + kAccErr);
  int* d_ncand = reinterpret_cast<int*>(acc + kAccNcand);
  finalize_kernel<<<1, 1024, 0, st>>>(b.ndet, p.eps, p.s2, reinterpret_cast<const long long*>(p.na),
                                      reinterpret_cast<const long long*>(p.ncon), x->res.as<DevResult>());
  if (b.k > 0) {
    gather_kernel<<<grid, 256, 0, st>>>(grid, nint, b.cap, p.tk_cnt, p.tk_e, p.tk_a, p.tk_key, p.tau_bits,
                                        x->cand_e.as<double>(), x->cand_a.as<double>(), x->cand_key.as<uint64_t>(),
                                        d_ncand, (int64_t)b.maxc, d_err);
    // the segment bounds: two ints after the sort's scratch space
    int* be = reinterpret_cast<int*>(x->cub_tmp2.as<unsigned char>() + ((b.tmp2 + 15) & ~(size_t)15));
    seg_bounds_kernel<<<1, 1, 0, st>>>(d_ncand, be);
    const int cap = (int)b.maxc;
    const int sb = (cap + 255) / 256;
    iota_kernel<<<sb, 256, 0, st>>>(cap, x->perm.as<int32_t>());
    int32_t *pa = x->perm.as<int32_t>(), *pb = x->perm2.as<int32_t>();
    for (int pass = 0; pass <= nw; pass++) {
      const int word = (pass < nw) ? (nw - 1 - pass) : nw;
      sortkey_dev_kernel<<<sb, 256, 0, st>>>(cap, d_ncand, nint, word, x->cand_e.as<double>(),
                                             x->cand_key.as<uint64_t>(), pa, x->skey.as<unsigned long long>());
      CUDA_TRY(cub::DeviceSegmentedRadixSort::SortPairs(x->cub_tmp2.p, b.tmp2, x->skey.as<unsigned long long>(),
                                                        x->skey2.as<unsigned long long>(), pa, pb, cap, 1, be,
                                                        be + 1, 0, 64, st));
      std::swap(pa, pb);
    }
    select_out_dev_kernel<<<(int)((b.k + 255) / 256), 256, 0, st>>>(b.k, d_ncand, nint, pa, x->cand_e.as<double>(),
                                                                   x->cand_key.as<uint64_t>(), b.sel, b.se,
                                                                   acc + kAccQueue);
  }
  CUDA_TRY(cudaGetLastError());
  return QP_OK;
}

// Fused form: group the instances by word count and precision.  A group's
// waves are filled with pieces (instance, run of generator slots) taken
// instance after instance, each wave holding at most its share of
// wave_budget bytes of records and buckets, so that a wave holds one or a few
// instances (their integrals stay in L2 while the wave runs).  The pieces'
// records and buckets live in one pool per group, laid out per wave; each
// group's per-wave tables of parameters and slot / item offsets are written
// to the device.
static int plan_fused(qp_pt2_batch* B, const qp_pt2_batch_options& o, size_t wave_budget) {
  const int n = (int)B->inst.size();
  for (int i = 0; i < n; i++) {
    BatchInst& b = B->inst[i];
    const int mixed = b.x->cfg.precision == QP_MIXED;
    int g = -1;
    for (size_t j = 0; j < B->groups.size(); j++)
      if (B->groups[j].nint == b.x->nint && B->groups[j].mixed == mixed) g = (int)j;
    if (g < 0) {
      B->groups.emplace_back();
      g = (int)B->groups.size() - 1;
      B->groups[g].nint = b.x->nint;
      B->groups[g].mixed = mixed;
    }
    b.group = g;
    B->groups[g].members.push_back(i);
  }
  double total = 0.0;
  for (auto& b : B->inst) total += (double)inst_slot_bytes(b) * (double)b.ngen;
  auto al = [](size_t x) { return (x + 255) & ~(size_t)255; };
  for (auto& G : B->groups) {
    qp_pt2_ctx* x0 = B->inst[G.members[0]].x;
    G.smem = 0;
    for (int i : G.members) G.smem = std::max(G.smem, B->inst[i].smem);
    int bps = batch_multi_blocks_per_sm(G.nint, G.mixed, G.smem);
    if (bps < 1) return fail(QP_ENOTSUP, "the batch accumulator does not fit in shared memory");
    if (o.blocks_per_sm > 0 && o.blocks_per_sm < bps) bps = o.blocks_per_sm;
    G.grid = bps * x0->nsm;
    G.chunk = o.work_chunk > 0 ? o.work_chunk : 1;
    // the instance with the largest work items first: a wave's queue ends
    // with the smallest items
    std::stable_sort(G.members.begin(), G.members.end(), [&](int a, int c) {
      const BatchInst &ba = B->inst[a], &bc = B->inst[c];
      return ba.max_cells != bc.max_cells ? ba.max_cells > bc.max_cells : ba.ndet > bc.ndet;
    });
    double gtot = 0.0;
    for (int i : G.members) gtot += (double)inst_slot_bytes(B->inst[i]) * (double)B->inst[i].ngen;
    const size_t budget = (size_t)((double)wave_budget * gtot / total);  // this group's share
    // pieces: (wave, instance, first slot, slots, pool offset)
    struct Piece {
      int wave, inst;
      int64_t start, slots;
      size_t off;
    };
    std::vector<Piece> pieces;
    G.timeout_ns = 0;
    int wave = 0, inwave = 0;
    size_t used = 0, pool_bytes = 0;
    for (int i : G.members) {
      BatchInst& b = B->inst[i];
      b.grid = G.grid;
      const size_t per = inst_slot_bytes(b) + 12 * 256;  // a slot and the alignment of its arrays
      int64_t start = 0;
      while (start < b.ngen) {
        int64_t fit = (int64_t)((budget > used ? budget - used : 0) / per);
        if ((fit < 1 && used > 0) || inwave == kMaxPieces) {  // the wave is full: start the next one
          wave++;
          used = 0;
          inwave = 0;
          continue;
        }
        if (fit < 1) fit = 1;
        const int64_t take = std::min(fit, b.ngen - start);
        pieces.push_back({wave, i, start, take, used});
        used += al(per * (size_t)take);
        pool_bytes = std::max(pool_bytes, used);
        start += take;
        inwave++;
      }
      int64_t wmax = 1;  // the instance's largest piece
      for (const Piece& q : pieces)
        if (q.inst == i) wmax = std::max(wmax, q.slots);
      int rc = plan_instance(b, 0, wmax, true);
      if (rc) return rc;
      make_params(b);
      const unsigned long long t = b.p.timeout_ns;
      if (t && (G.timeout_ns == 0 || t < G.timeout_ns)) G.timeout_ns = t;
    }
    G.nwaves = wave + 1;
    if (cudaMalloc(&G.pool, pool_bytes) != cudaSuccess)
      return fail(QP_ENOMEM, "device allocation of the batch's wave pool failed");
    const int nm = (int)G.members.size();
    int maxp = 0;  // the most pieces in a wave
    {
      std::vector<int> cnt(G.nwaves, 0);
      for (const Piece& q : pieces) maxp = std::max(maxp, ++cnt[q.wave]);
    }
    G.npw = maxp;
    std::vector<SweepParams> hp((size_t)G.nwaves * maxp + nm);
    std::vector<int> hs((size_t)G.nwaves * (maxp + 1), 0);
    std::vector<long long> hi((size_t)G.nwaves * (maxp + 1), 0);
    G.nact.assign(G.nwaves, 0);
    G.slots.assign(G.nwaves, 0);
    G.max_slots.assign(G.nwaves, 0);
    unsigned char* base = static_cast<unsigned char*>(G.pool);
    for (const Piece& q : pieces) {
      const BatchInst& b = B->inst[q.inst];
      const qp_pt2_ctx* x = b.x;
      const size_t nd = (size_t)b.ndet, ws = (size_t)q.slots, nw = 2 * (size_t)x->nint;
      SweepParams p = b.p;
      unsigned char* c = base + q.off;
      auto take = [&](size_t bytes) {
        unsigned char* r = c;
        c += al(bytes);
        return r;
      };
      p.meta = reinterpret_cast<GenMeta*>(take(sizeof(GenMeta) * ws));
      p.r_words = reinterpret_cast<uint64_t*>(take(8 * nd * nw * ws));
      p.r_coef = reinterpret_cast<double*>(take(8 * nd * ws));
      p.r_hmask = reinterpret_cast<uint64_t*>(take(8 * nd * ws));
      p.r_part = reinterpret_cast<uint64_t*>(take(8 * nd * ws));
      p.r_flag = reinterpret_cast<uint32_t*>(take(4 * nd * ws));
      p.b_ofs = reinterpret_cast<int*>(take(4 * (size_t)(x->nbat + 2) * ws));
      p.e_hp = reinterpret_cast<ulonglong2*>(take(16 * (size_t)b.ent_cap * ws));
      p.e_rec = reinterpret_cast<uint32_t*>(take(4 * (size_t)b.ent_cap * ws));
      p.b_dead = reinterpret_cast<uint32_t*>(take(4 * (size_t)((x->nbat + 31) / 32) * ws));
      p.it_sum = reinterpret_cast<double*>(take(16 * (size_t)b.nper * ws));
      p.wave_start = (int)q.start;
      p.wave_slots = (int)q.slots;
      p.last_wave = 0;  // compact_multi_kernel keeps the k best after the last wave
      p.queue = nullptr;
      const int r = q.wave, a = G.nact[r]++;
      hp[(size_t)r * maxp + a] = p;
      int* so = hs.data() + (size_t)r * (maxp + 1);
      long long* io = hi.data() + (size_t)r * (maxp + 1);
      so[a + 1] = so[a] + p.wave_slots;
      io[a + 1] = io[a] + (long long)p.wave_slots * p.nper;
      G.slots[r] = so[a + 1];
      G.max_slots[r] = std::max(G.max_slots[r], p.wave_slots);
    }
    for (int m = 0; m < nm; m++) hp[(size_t)G.nwaves * maxp + m] = B->inst[G.members[m]].p;
    G.hps = hp;
    G.hitem = hi;
    if (cudaMalloc(&G.d_ps, sizeof(SweepParams) * hp.size()) != cudaSuccess ||
        cudaMalloc(&G.d_slot_ofs, sizeof(int) * hs.size()) != cudaSuccess ||
        cudaMalloc(&G.d_item_ofs, sizeof(long long) * hi.size()) != cudaSuccess ||
        cudaMalloc(&G.d_words, sizeof(unsigned long long) * ((size_t)G.nwaves * maxp + 1)) != cudaSuccess ||
        cudaMalloc(&G.d_err, sizeof(int)) != cudaSuccess)
      return fail(QP_ENOMEM, "device allocation of the batch tables failed");
    if (cudaMemcpy(G.d_ps, hp.data(), sizeof(SweepParams) * hp.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.d_slot_ofs, hs.data(), sizeof(int) * hs.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemcpy(G.d_item_ofs, hi.data(), sizeof(long long) * hi.size(), cudaMemcpyHostToDevice) != cudaSuccess ||
        cudaMemset(G.d_err, 0, sizeof(int)) != cudaSuccess)
      return fail(QP_ECUDA, "copy of the batch tables failed");
    if (cudaStreamCreateWithFlags(&G.st, cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&G.done, cudaEventDisableTiming) != cudaSuccess)
      return fail(QP_ECUDA, "stream creation failed");
  }
  return QP_OK;
}

// One group's waves on its stream: per wave the prep and batch launches over
// all active instances and the per-generator reduction; then the compaction
// of the candidate buffers.
static int enqueue_group(FusedGroup& G) {
  const int nm = (int)G.members.size(), np = G.npw;
  CUDA_TRY(cudaMemsetAsync(G.d_words, 0, sizeof(unsigned long long) * ((size_t)G.nwaves * np + 1), G.st));
  CUDA_TRY(cudaMemsetAsync(G.d_err, 0, sizeof(int), G.st));
  for (int r = 0; r < G.nwaves; r++) {
    MultiWave m{};
    m.ps = G.d_ps + (size_t)r * np;
    m.slot_ofs = G.d_slot_ofs + (size_t)r * (np + 1);
    m.item_ofs = G.d_item_ofs + (size_t)r * (np + 1);
    m.n = G.nact[r];
    m.chunk = G.chunk;
    m.queue = G.d_words + (size_t)r * np;  // one item counter per piece
    m.timeout_ns = G.timeout_ns;
    m.t_start = G.d_words + (size_t)G.nwaves * np;
    m.err = G.d_err;
    MultiWaveInline mi{};
    for (int a = 0; a < G.nact[r]; a++) mi.ps[a] = G.hps[(size_t)r * np + a];
    for (int a = 0; a <= G.nact[r]; a++) mi.item_ofs[a] = G.hitem[(size_t)r * (np + 1) + a];
    mi.n = m.n;
    mi.chunk = m.chunk;
    mi.queue = m.queue;
    mi.timeout_ns = m.timeout_ns;
    mi.t_start = m.t_start;
    mi.err = m.err;
    CUDA_TRY(launch_wave_multi(G.nint, G.mixed, m, mi, G.slots[r], G.grid, G.smem, G.st));
    CUDA_TRY(launch_reduce_items_multi(m.ps, G.nact[r], G.max_slots[r], G.st));
  }
  CUDA_TRY(launch_compact_multi(G.nint, G.mixed, G.d_ps + (size_t)G.nwaves * np, nm, G.grid, G.st));
  return QP_OK;
}

extern "C" int qp_pt2_batch_create(qp_pt2_batch** out, int n, qp_pt2_ctx* const* ctxs, const int64_t* ndet,
                                   const uint64_t* const* dets, const double* const* coefs, const double* e0,
                                   const int64_t* k, uint64_t* const* sel_dets, double* const* sel_e,
                                   const int* grid, int max_streams, void* stream) {
  qp_pt2_batch_options o{};
  o.fused = 0;
  o.max_streams = max_streams;
  return qp_pt2_batch_create_ex(out, n, ctxs, ndet, dets, coefs, e0, k, sel_dets, sel_e, grid, &o, stream);
}

extern "C" int qp_pt2_batch_create_ex(qp_pt2_batch** out, int n, qp_pt2_ctx* const* ctxs, const int64_t* ndet,
                                      const uint64_t* const* dets, const double* const* coefs, const double* e0,
                                      const int64_t* k, uint64_t* const* sel_dets, double* const* sel_e,
                                      const int* grid, const qp_pt2_batch_options* opt, void* stream) {
  if (!out || n < 1 || !ctxs || !ndet || !dets || !coefs || !e0 || !k) return fail(QP_EINVAL, "bad batch arguments");
  *out = nullptr;
  qp_pt2_batch_options o{};
  o.fused = 1;
  if (opt) o = *opt;
  if (o.work_chunk < 0 || o.tile < 0 || o.blocks_per_sm < 0 || !(o.wave_gb >= 0.0))
    return fail(QP_EINVAL, "bad batch options");
  qp_pt2_batch* B = new (std::nothrow) qp_pt2_batch();
  if (!B) return fail(QP_ENOMEM, "host allocation failed");
  auto bail = [&](int code, const std::string& m) {
    qp_pt2_batch_destroy(B);
    return fail(code, m);
  };
  B->main = (cudaStream_t)stream;
  B->fused = o.fused != 0;
  for (int i = 0; i < n; i++) {
    BatchInst b{};
    b.x = ctxs[i];
    b.ndet = ndet[i];
    b.k = k[i];
    b.dets = dets[i];
    b.coefs = coefs[i];
    b.e0 = e0[i];
    b.sel = sel_dets ? sel_dets[i] : nullptr;
    b.se = sel_e ? sel_e[i] : nullptr;
    b.grid = (grid && !B->fused) ? grid[i] : 0;
    if (!b.x || b.ndet < 1 || b.k < 0 || b.ndet >= (1ll << 31) || !std::isfinite(b.e0))
      return bail(QP_EINVAL, "bad instance " + std::to_string(i));
    if (b.x->cfg.shard_count > 1) return bail(QP_EINVAL, "sharded contexts cannot be batched");
    if (!is_device_ptr(b.dets) || !is_device_ptr(b.coefs) || (b.k > 0 && (!is_device_ptr(b.sel) || !is_device_ptr(b.se))))
      return bail(QP_EINVAL, "batched inputs and outputs must be device memory (instance " + std::to_string(i) + ")");
    for (int j = 0; j < i; j++)
      if (B->inst[j].x == b.x) return bail(QP_EINVAL, "each instance needs its own context");
    qp_pt2_ctx* x = b.x;
    b.ntile = x->ntile;
    b.max_cells = x->max_cells;
    b.smem = x->smem;
    if (B->fused && o.tile > 0) {
      const int va = x->norb - x->nalpha;
      b.ntile = (x->nalpha > 0 && x->nbeta > 0) ? std::min(o.tile, std::max(va, 1)) : 1;
      b.max_cells = cells_for_tile(x->norb, x->nalpha, x->nbeta, b.ntile);
      b.smem = sweep_smem(b.max_cells);
    }
    b.nper = x->nbat + (b.ntile - 1) * x->nalpha * x->nbeta;
    b.ngen = b.ndet;
    if (!B->fused) {
      // all instances' workspaces stay allocated together: share the wave budget
      size_t budget = (size_t)(16ull << 30) / (size_t)n;
      if (budget > kWaveBudget) budget = kWaveBudget;
      if (budget < ((size_t)64 << 20)) budget = (size_t)64 << 20;
      int rc = plan_instance(b, budget, 0);
      if (rc) return bail(rc, "planning instance " + std::to_string(i) + ": " + g_last_error);
      make_params(b);
    }
    B->inst.push_back(b);
  }
  if (B->fused) {
    const double gb = o.wave_gb > 0.0 ? o.wave_gb : 24.0;
    int rc = plan_fused(B, o, (size_t)(gb * (double)(1ull << 30)));
    if (rc) return bail(rc, "planning the batch: " + g_last_error);
  }
  int ns = o.max_streams > 0 ? o.max_streams : 16;
  if (ns > n) ns = n;
  B->br.resize(ns);
  B->ev.resize(ns);
  for (int i = 0; i < ns; i++) {
    if (cudaStreamCreateWithFlags(&B->br[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&B->ev[i], cudaEventDisableTiming) != cudaSuccess)
      return bail(QP_ECUDA, "stream creation failed");
  }
  if (cudaEventCreateWithFlags(&B->fork, cudaEventDisableTiming) != cudaSuccess ||
      cudaEventCreate(&B->t0) != cudaSuccess || cudaEventCreate(&B->t1) != cudaSuccess)
    return bail(QP_ECUDA, "event creation failed");
  if (cudaStreamSynchronize(B->main) != cudaSuccess) return bail(QP_ECUDA, "stream synchronisation failed");
  // largest work first, each on the least loaded branch
  std::vector<int> order(n);
  for (int i = 0; i < n; i++) order[i] = i;
  std::sort(order.begin(), order.end(), [&](int a, int b) { return B->inst[a].work > B->inst[b].work; });
  std::vector<double> load(ns, 0.0);
  std::vector<int> branch(n);
  for (int i : order) {
    int s = (int)(std::min_element(load.begin(), load.end()) - load.begin());
    branch[i] = s;
    load[s] += B->inst[i].work;
  }
  // capture: fork from the main stream, one branch per stream, join
  cudaStream_t cap = B->main;
  if (!cap) {  // the legacy stream cannot be captured: use a stream of our own
    if (cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking) != cudaSuccess) return bail(QP_ECUDA, "stream");
    B->own_main = true;
    B->main = cap;
  }
  if (cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess)
    return bail(QP_ECUDA, "cudaStreamBeginCapture failed");
  cudaEventRecord(B->fork, cap);
  for (int s = 0; s < ns; s++) cudaStreamWaitEvent(B->br[s], B->fork, 0);
  int erc = QP_OK;
  if (!B->fused) {
    for (int i : order) {
      BatchInst& b = B->inst[i];
      cudaStream_t st = B->br[branch[i]];
      if ((erc = enqueue_pre(b, st)) || (erc = enqueue_waves(b, st)) || (erc = enqueue_post(b, st))) break;
    }
  } else {
    for (int i : order)
      if ((erc = enqueue_pre(B->inst[i], B->br[branch[i]]))) break;
    // every group's waves start when all instances are validated and ranked
    for (int s = 0; s < ns && !erc; s++) cudaEventRecord(B->ev[s], B->br[s]);
    for (auto& G : B->groups) {
      if (erc) break;
      for (int s = 0; s < ns; s++) cudaStreamWaitEvent(G.st, B->ev[s], 0);
      erc = enqueue_group(G);
      cudaEventRecord(G.done, G.st);
    }
    for (int s = 0; s < ns && !erc; s++)
      for (auto& G : B->groups) cudaStreamWaitEvent(B->br[s], G.done, 0);
    for (int i : order) {
      if (erc) break;
      erc = enqueue_post(B->inst[i], B->br[branch[i]]);
    }
  }
  for (int s = 0; s < ns; s++) {
    cudaEventRecord(B->ev[s], B->br[s]);
    cudaStreamWaitEvent(cap, B->ev[s], 0);
  }
  cudaGraph_t g = nullptr;
  const cudaError_t ce = cudaStreamEndCapture(cap, &g);
  if (erc) {
    if (g) cudaGraphDestroy(g);
    return bail(erc, "enqueue failed: " + g_last_error);
  }
  if (ce != cudaSuccess || !g) return bail(QP_ECUDA, std::string("stream capture failed: ") + cudaGetErrorString(ce));
  B->graph = g;
  if (cudaGraphInstantiate(&B->exec, g, 0) != cudaSuccess) return bail(QP_ECUDA, "cudaGraphInstantiate failed");
  *out = B;
  return QP_OK;
}

extern "C" int qp_pt2_batch_run(qp_pt2_batch* B, qp_pt2_result* res, double* ms) {
  if (!B || !B->exec) return fail(QP_EINVAL, "batch not created");
  CUDA_TRY(cudaEventRecord(B->t0, B->main));
  CUDA_TRY(cudaGraphLaunch(B->exec, B->main));
  CUDA_TRY(cudaEventRecord(B->t1, B->main));
  CUDA_TRY(cudaStreamSynchronize(B->main));
  if (ms) {
    float f = 0.f;
    CUDA_TRY(cudaEventElapsedTime(&f, B->t0, B->t1));
    *ms = f;
  }
  int worst = QP_OK;
  for (size_t i = 0; i < B->inst.size(); i++) {
    BatchInst& b = B->inst[i];
    DevResult hres;
    unsigned long long hacc[kAccWords];
    CUDA_TRY(cudaMemcpy(&hres, b.x->res.p, sizeof(hres), cudaMemcpyDeviceToHost));
    CUDA_TRY(cudaMemcpy(hacc, b.x->acc.p, sizeof(hacc), cudaMemcpyDeviceToHost));
    qp_pt2_result r;
    memset(&r, 0, sizeof(r));
    const int herr = (int)(hacc[kAccErr] & 0xffffffffull);
    int code = QP_OK;
    if (herr & kErrOcc) code = QP_EINVAL;
    else if (herr & kErrCoef) code = QP_EINVAL;
    else if (herr & kErrDup) code = QP_EDUP;
    else if (herr & kErrBucket) code = QP_ECUDA;
    else if (herr & kErrRange) code = QP_ENOTSUP;
    else if (herr & kErrTimeout) code = QP_ETIMEOUT;
    else if (herr & 32) code = QP_ENOMEM;
    if (code == QP_OK && B->fused) {  // the group's launch stopped by its watchdog
      int gerr = 0;
      CUDA_TRY(cudaMemcpy(&gerr, B->groups[b.group].d_err, sizeof(int), cudaMemcpyDeviceToHost));
      if (gerr & kErrTimeout) code = QP_ETIMEOUT;
    }
    r.e_pt2 = hres.e_pt2;
    r.sum_e_over_d = hres.s2;
    r.n_perturbers = hres.na;
    r.n_connections = hres.ncon;
    r.n_selected = b.k > 0 ? (int64_t)hacc[kAccQueue] : 0;
    r.n_tiny = (int64_t)hacc[kAccTiny];
    r.perturber_digest[0] = hacc[kAccDigest0];
    r.perturber_digest[1] = hacc[kAccDigest1];
    double md;
    memcpy(&md, &hacc[kAccMinDen], sizeof(md));
    r.min_abs_denominator = md;
    set_rpt2(r, b.e0);
    if (code == QP_OK && hres.na > 0 && md < 1e-12) code = QP_ESINGULAR;
    if (res) res[i] = r;
    if (code != QP_OK && worst == QP_OK) {
      worst = code;
      g_last_error = "batch instance " + std::to_string(i) + ": " + qp_pt2_strerror(code);
    }
  }
  return worst;
}

extern "C" void qp_pt2_batch_destroy(qp_pt2_batch* B) {
  if (!B) return;
  if (B->exec) cudaGraphExecDestroy(B->exec);
  if (B->graph) cudaGraphDestroy(B->graph);
  for (auto& G : B->groups) {
    if (G.pool) cudaFree(G.pool);
    if (G.d_ps) cudaFree(G.d_ps);
    if (G.d_slot_ofs) cudaFree(G.d_slot_ofs);
    if (G.d_item_ofs) cudaFree(G.d_item_ofs);
    if (G.d_words) cudaFree(G.d_words);
    if (G.d_err) cudaFree(G.d_err);
    if (G.st) cudaStreamDestroy(G.st);
    if (G.done) cudaEventDestroy(G.done);
  }
  for (auto s : B->br) if (s) cudaStreamDestroy(s);
  for (auto e : B->ev) if (e) cudaEventDestroy(e);
  if (B->fork) cudaEventDestroy(B->fork);
  if (B->t0) cudaEventDestroy(B->t0);
  if (B->t1) cudaEventDestroy(B->t1);
  if (B->own_main && B->main) cudaStreamDestroy(B->main);
  delete B;
}
