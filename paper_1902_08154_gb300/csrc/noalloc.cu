// noalloc.cu -- qp_pt2_eval_noalloc: the whole EN-PT2 + selection sweep with
// no device memory allocation at all.
//
// Who needs it: a host program that reserves the GPU's memory up front and
// hands its plugins no allocator, or a deployment whose device-memory
// footprint is fixed and audited, cannot let a library call cudaMalloc or
// cudaFree.  Such a caller gives device pointers for every input and output;
// everything else the sweep needs (integral tables, generator order, per-
// generator records and buckets, selection buffers, sort space) lives in one
// file-scope device array of fixed size, loaded with the library on every
// GPU that loads it and held until the process exits.
//
// The array's host-side name is only a stand-in: host code obtains its device
// address with cudaGetSymbolAddress, once per device, on the first call made
// on that device (that first call should therefore come before any stream
// capture).  Every call reuses the same array and leaves its contents behind,
// so each call clears what must start at zero; two calls whose work overlaps
// on the GPU (on different streams, or from different threads) race on it.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cmath>
#include <cstring>
#include <mutex>
#include <string>

#include "../../include/qp_pt2.h"
#include "common.cuh"

// kernels defined with the main entry points (qp_pt2.cu) and the sweep
// (sweep.cu); this file launches them unchanged
struct DevResult {
  double e_pt2, s2;
  long long na, ncon;
};
__global__ void jk_kernel(int norb, const double* eri, double* Jm, double* Km);
__global__ void validate_kernel(int64_t ndet, int nint, int norb, int na, int nb, const uint64_t* dets,
                            const double* coefs, unsigned long long* hkey, int32_t* hidx,
                            unsigned long long* rkey, int32_t* ridx, int* err, unsigned long long* cmax);
__global__ void absmax_kernel(int64_t n, const double* x, unsigned long long* out);
__global__ void dup_kernel(int64_t ndet, int nint, const uint64_t* dets, const unsigned long long* hs,
                           const int32_t* hi, int* err);
__global__ void rank_kernel(int64_t ndet, const int32_t* order, int32_t* rank_of);
__global__ void finalize_kernel(int64_t ndet, const double* eps, const double* s2, const long long* na,
                                const long long* nc, DevResult* out);
__global__ void gather_kernel(int grid, int nint, int64_t cap, const int* tk_cnt, const double* tk_e,
                              const double* tk_a, const uint64_t* tk_key, const unsigned long long* tau,
                              double* ce, double* ca, uint64_t* ck, int* ncand, int64_t cand_cap, int* err);
__global__ void sortkey_kernel(int n, int nint, int w, const double* ce, const uint64_t* ck,
                               const int32_t* perm, unsigned long long* keys);
__global__ void iota_kernel(int n, int32_t* v);
__global__ void select_out_kernel(int n, int nint, const int32_t* perm, const double* ce, const double* ca,
                                  const uint64_t* ck, uint64_t* sel, double* se, double* sn);
namespace qp {
cudaError_t launch_prep(int nint, const SweepParams& p, int slots, cudaStream_t st);
cudaError_t launch_batch_packed(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st);
cudaError_t launch_reduce_items(const SweepParams& p, cudaStream_t st);
int batch_blocks_per_sm_packed(int nint, size_t smem);
int report(int code, const char* msg);
}  // namespace qp

using namespace qp;

namespace {

constexpr size_t kScratchBytes = (size_t)64 << 20;  // 64 MiB per device
constexpr int kMaxDevices = 64;

std::mutex g_mu;
unsigned char* g_base[kMaxDevices] = {nullptr};

// Failures are reported through the library's error channel, so that
// qp_pt2_last_error() names them.
int nfail(int code, const std::string& m) { return qp::report(code, m.c_str()); }

// Symmetry of h, checked on the device (no host copy of h).
__global__ void sym_kernel(int norb, const double* h, int* err) {
  int x = blockIdx.x * blockDim.x + threadIdx.x;
  if (x >= norb * norb) return;
  int p = x / norb, q = x % norb;
  if (q < p && !(fabs(h[p * norb + q] - h[q * norb + p]) <= 1e-12)) atomicOr(err, 16);
}

// Bump allocation inside the static array.
struct Carve {
  unsigned char* base;
  size_t off = 0;
  bool ok = true;
  template <typename T>
  T* take(size_t count) {
    off = (off + 255) & ~(size_t)255;
    const size_t bytes = sizeof(T) * (count ? count : 1);
    if (off + bytes > kScratchBytes) {
      ok = false;
      return nullptr;
    }
    T* p = reinterpret_cast<T*>(base + off);
    off += bytes;
    return p;
  }
};

// Device (or managed) memory that belongs to device dev: memory of another
// GPU would be reached by peer access, or fault.
bool on_device(const void* p, int dev) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (a.type == cudaMemoryTypeManaged) return true;
  return a.type == cudaMemoryTypeDevice && a.device == dev;
}

int cells_max(int norb, int na, int nb) {
  const int va = norb - na, vb = norb - nb;
  int m = va > vb ? va : vb;
  int t = va * (va - 1) / 2;
  m = t > m ? t : m;
  t = vb * (vb - 1) / 2;
  m = t > m ? t : m;
  t = va * vb;
  m = t > m ? t : m;
  return m < 1 ? 1 : m;
}

}  // namespace

// The fixed device array all calls share (see the file header).
static __device__ __align__(256) unsigned char qp_noalloc_scratch[kScratchBytes];

#define NTRY(expr)                                                                     \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) return nfail(QP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_)); \
  } while (0)

// After the first kernel of a call is queued: on a failure, wait for the
// work already queued, so that no kernel of this call still writes the
// shared array when the call returns.
#define NTRY_Q(expr)                                                                   \
  do {                                                                                 \
    cudaError_t e_ = (expr);                                                           \
    if (e_ != cudaSuccess) {                                                           \
      cudaStreamSynchronize(st);                                                       \
      return nfail(QP_ECUDA, std::string(#expr) + ": " + cudaGetErrorString(e_));      \
    }                                                                                  \
  } while (0)

extern "C" int qp_pt2_eval_noalloc(int norb, int n_alpha, int n_beta, const double* h, const double* eri,
                                   int64_t ndet, const uint64_t* dets, const double* coefs, double e0,
                                   int64_t k, uint64_t* sel_dets, double* sel_e, qp_pt2_result* res,
                                   void* stream) {
  if (!res) return nfail(QP_EINVAL, "res is NULL");
  memset(res, 0, sizeof(*res));
  res->min_abs_denominator = INFINITY;
  if (norb < 1 || norb > kMaxOrb) return nfail(QP_EINVAL, "norb must be in [1, 128]");
  if (n_alpha < 0 || n_beta < 0 || n_alpha > norb || n_beta > norb || n_alpha + n_beta > kMaxElec)
    return nfail(QP_EINVAL, "electron counts out of range");
  if (ndet < 0 || k < 0) return nfail(QP_EINVAL, "ndet and k must be non-negative");
  if (ndet >= (1ll << 31)) return nfail(QP_EINVAL, "ndet must be below 2^31");
  if (!std::isfinite(e0)) return nfail(QP_EINVAL, "E0 is not finite");
  if (ndet == 0) return QP_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int dev = 0;
  NTRY(cudaGetDevice(&dev));
  if (!on_device(h, dev) || !on_device(eri, dev) || !on_device(dets, dev) || !on_device(coefs, dev) ||
      (k > 0 && (!on_device(sel_dets, dev) || !on_device(sel_e, dev))))
    return nfail(QP_EINVAL, "every array must be device memory of the current device");

  // ---- the static array of this device ----
  if (dev < 0 || dev >= kMaxDevices) return nfail(QP_ENOTSUP, "device index too large");
  unsigned char* base;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_base[dev]) {
      void* ptr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&ptr, qp_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return nfail(QP_ECUDA, std::string("cudaGetSymbolAddress: ") + cudaGetErrorString(e));
      g_base[dev] = static_cast<unsigned char*>(ptr);
    }
    base = g_base[dev];
  }

  // ---- sizes and layout ----
  const int nint = (norb - 1) / 64 + 1, nw = 2 * nint, nel = n_alpha + n_beta;
  const int nbat = nel + nel * (nel - 1) / 2;
  const int max_cells = cells_max(norb, n_alpha, n_beta);
  const size_t smem = sweep_smem(max_cells);
  if (batch_blocks_per_sm_packed(nint, smem) < 1) return nfail(QP_ENOTSUP, "batch accumulator exceeds shared memory");
  int nsm = 0;
  NTRY(cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev));
  const int grid = nsm;  // one CTA per SM keeps the selection buffers small
  const size_t nd = (size_t)ndet;
  const int64_t cap = k > 0 ? k + max_cells : 1;
  const size_t maxc = (size_t)grid * (size_t)(k > 0 ? k : 1);
  size_t tmp1 = 0, tmp2 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp1, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                  (int32_t*)nullptr, (int32_t*)nullptr, (int)ndet, 0, 64, st);
  cub::DeviceRadixSort::SortPairs(nullptr, tmp2, (unsigned long long*)nullptr, (unsigned long long*)nullptr,
                                  (int32_t*)nullptr, (int32_t*)nullptr, (int)maxc, 0, 64, st);
  Carve cv{base};
  double* d_J = cv.take<double>((size_t)norb * norb);
  double* d_K = cv.take<double>((size_t)norb * norb);
  unsigned long long* hkey = cv.take<unsigned long long>(nd);
  unsigned long long* hkey2 = cv.take<unsigned long long>(nd);
  unsigned long long* rkey = cv.take<unsigned long long>(nd);
  unsigned long long* rkey2 = cv.take<unsigned long long>(nd);
  int32_t* hidx = cv.take<int32_t>(nd);
  int32_t* hidx2 = cv.take<int32_t>(nd);
  int32_t* order = cv.take<int32_t>(nd);
  int32_t* rank_of = cv.take<int32_t>(nd);
  unsigned char* cub_tmp = cv.take<unsigned char>(tmp1 > tmp2 ? tmp1 : tmp2);
  double* eps = cv.take<double>(nd);
  double* s2 = cv.take<double>(nd);
  unsigned long long* na = cv.take<unsigned long long>(nd);
  unsigned long long* ncon = cv.take<unsigned long long>(nd);
  unsigned long long* acc = cv.take<unsigned long long>(9);
  DevResult* dres = cv.take<DevResult>(1);
  int* queues = cv.take<int>(nd + 1);
  double* tk_e = cv.take<double>((size_t)cap * grid);
  double* tk_a = cv.take<double>((size_t)cap * grid);
  uint64_t* tk_key = cv.take<uint64_t>((size_t)cap * grid * nw);
  int* tk_cnt = cv.take<int>(grid);
  unsigned long long* tk_tau = cv.take<unsigned long long>(grid);
  unsigned long long* d_hmax = cv.take<unsigned long long>(2);
  unsigned int* sel_hist = cv.take<unsigned int>(kSelBins);
  double* cand_e = cv.take<double>(maxc);
  double* cand_a = cv.take<double>(maxc);
  uint64_t* cand_key = cv.take<uint64_t>(maxc * nw);
  unsigned long long* skey = cv.take<unsigned long long>(maxc);
  unsigned long long* skey2 = cv.take<unsigned long long>(maxc);
  int32_t* perm = cv.take<int32_t>(maxc);
  int32_t* perm2 = cv.take<int32_t>(maxc);
  if (!cv.ok)
    return nfail(QP_EINVAL, "ndet or k too large for the 64 MiB static scratch of qp_pt2_eval_noalloc");
  const int64_t ent_per = bucket_entries_per_record(nel);
  const int64_t ent_cap = (int64_t)nd * ent_per;
  const size_t dwords = (size_t)(nbat + 31) / 32;
  const int nper = nbat;
  const size_t per_slot = wave_slot_bytes(sizeof(GenMeta), nel, nbat, nw, nd, 1, nper);
  // each of the 12 per-slot arrays carved below may start with up to 255
  // bytes of alignment padding: keep 12 x 256 bytes aside for them
  const size_t left = kScratchBytes > cv.off + 12 * 256 ? kScratchBytes - cv.off - 12 * 256 : 0;
  int64_t W = (int64_t)(left / per_slot);
  if (W < 1)
    return nfail(QP_EINVAL, "ndet too large for the 64 MiB static scratch of qp_pt2_eval_noalloc");
  const int64_t ngen = ndet;
  if (W > ngen) W = ngen;
  const int64_t nwaves = (ngen + W - 1) / W;
  const size_t wsl = (size_t)W;
  GenMeta* meta = cv.take<GenMeta>(wsl);
  uint64_t* r_words = cv.take<uint64_t>(nd * nw * wsl);
  double* r_coef = cv.take<double>(nd * wsl);
  uint64_t* r_hmask = cv.take<uint64_t>(nd * wsl);
  uint64_t* r_part = cv.take<uint64_t>(nd * wsl);
  uint32_t* r_flag = cv.take<uint32_t>(nd * wsl);
  int* b_ofs = cv.take<int>((size_t)(nbat + 2) * wsl);
  ulonglong2* e_hp = cv.take<ulonglong2>((size_t)ent_cap * wsl);
  uint32_t* e_rec = cv.take<uint32_t>((size_t)ent_cap * wsl);
  double* it_sum = cv.take<double>((size_t)2 * nper * wsl);
  uint32_t* b_dead = cv.take<uint32_t>(dwords * wsl);
  if (!cv.ok) return nfail(QP_EINVAL, "ndet too large for the 64 MiB static scratch of qp_pt2_eval_noalloc");

  // ---- clear what must start at zero; integral tables; validation ----
  // accumulator words: 0, 1 digest, 2 min |D|, 3 tiny, 4 threshold, 6 error
  // flags, 7 candidates, 8 bits of max |c_I|
  static const unsigned long long init[9] = {0, 0, 0x7FF0000000000000ull, 0, 0, 0, 0, 0, 0};
  NTRY(cudaMemcpyAsync(acc, init, sizeof(init), cudaMemcpyHostToDevice, st));
  int* d_err = reinterpret_cast<int*>(acc + 6);
  int* d_ncand = reinterpret_cast<int*>(acc + 7);
  NTRY(cudaMemsetAsync(d_hmax, 0, 2 * sizeof(unsigned long long), st));
  sym_kernel<<<(norb * norb + 255) / 256, 256, 0, st>>>(norb, h, d_err);
  const int64_t npair = (int64_t)norb * (norb + 1) / 2, P = npair * (npair + 1) / 2;
  absmax_kernel<<<(norb * norb + 255) / 256, 256, 0, st>>>((int64_t)norb * norb, h, d_hmax);
  absmax_kernel<<<(unsigned)((P + 255) / 256 < 4096 ? (P + 255) / 256 : 4096), 256, 0, st>>>(P, eri, d_hmax + 1);
  jk_kernel<<<(norb * norb + 255) / 256, 256, 0, st>>>(norb, eri, d_J, d_K);
  const int nb = (int)((ndet + 255) / 256);
  validate_kernel<<<nb, 256, 0, st>>>(ndet, nint, norb, n_alpha, n_beta, dets, coefs, hkey, hidx, rkey, rank_of, d_err,
                                      acc + 8);
  NTRY_Q(cudaGetLastError());
  NTRY_Q(cub::DeviceRadixSort::SortPairs(cub_tmp, tmp1, hkey, hkey2, hidx, hidx2, (int)ndet, 0, 64, st));
  dup_kernel<<<nb, 256, 0, st>>>(ndet, nint, dets, hkey2, hidx2, d_err);
  NTRY_Q(cub::DeviceRadixSort::SortPairs(cub_tmp, tmp1, rkey, rkey2, rank_of, order, (int)ndet, 0, 64, st));
  rank_kernel<<<nb, 256, 0, st>>>(ndet, order, rank_of);
  int herr = 0;
  NTRY_Q(cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  NTRY_Q(cudaStreamSynchronize(st));
  if (herr & 16) return nfail(QP_ESYM, "h is not symmetric");
  if (herr & 1) return nfail(QP_EINVAL, "a determinant has the wrong occupation or bits beyond norb");
  if (herr & 4) return nfail(QP_EINVAL, "a coefficient is not finite");
  if (herr & 2) return nfail(QP_EDUP, "duplicate determinant in Psi0");

  // ---- the sweep, in waves ----
  NTRY(cudaMemsetAsync(eps, 0, 8 * nd, st));
  NTRY(cudaMemsetAsync(s2, 0, 8 * nd, st));
  NTRY(cudaMemsetAsync(na, 0, 8 * nd, st));
  NTRY(cudaMemsetAsync(ncon, 0, 8 * nd, st));
  NTRY(cudaMemsetAsync(queues, 0, 4 * (nd + 1), st));
  NTRY(cudaMemsetAsync(tk_cnt, 0, 4 * (size_t)grid, st));
  NTRY(cudaMemsetAsync(tk_tau, 0, 8 * (size_t)grid, st));
  NTRY(cudaMemsetAsync(sel_hist, 0, 4 * (size_t)kSelBins, st));
  SweepParams p{};
  p.norb = norb;
  p.nalpha = n_alpha;
  p.nbeta = n_beta;
  p.nel = nel;
  p.nbat = nbat;
  p.ntile = 1;
  p.chunk = 1;
  p.timeout_ns = 0ull;
  p.t_start = nullptr;
  p.nper = nper;
  p.cmax_bits = acc + 8;
  p.hmax_bits = d_hmax;
  p.it_sum = it_sum;
  p.it_stride = 2;
  p.e_hp = e_hp;
  p.e_rec = e_rec;
  p.ndet = ndet;
  p.dets = dets;
  p.coefs = coefs;
  p.order = order;
  p.rank_of = rank_of;
  p.h = h;
  p.eri = eri;
  p.Jm = d_J;
  p.Km = d_K;
  p.e0 = e0;
  p.shard_index = 0;
  p.shard_count = 1;
  p.meta = meta;
  p.r_words = r_words;
  p.r_coef = r_coef;
  p.r_hmask = r_hmask;
  p.r_part = r_part;
  p.r_flag = r_flag;
  p.b_ofs = b_ofs;
  p.b_dead = b_dead;
  p.ent_cap = ent_cap;
  p.eps = eps;
  p.s2 = s2;
  p.na = na;
  p.ncon = ncon;
  p.digest = acc + 0;
  p.min_den_bits = acc + 2;
  p.n_tiny = acc + 3;
  p.k = k;
  p.cap = cap;
  p.tk_e = tk_e;
  p.tk_a = tk_a;
  p.tk_key = tk_key;
  p.tk_cnt = tk_cnt;
  p.tk_tau = tk_tau;
  p.tau_bits = acc + 4;
  p.sel_hist = sel_hist;
  p.max_cells = max_cells;
  p.err = d_err;
  for (int64_t w = 0; w < nwaves; w++) {
    p.wave_start = (int)(w * W);
    p.wave_slots = (int)((ngen - w * W) < W ? (ngen - w * W) : W);
    p.last_wave = (w == nwaves - 1);
    p.queue = queues + w;
    NTRY_Q(cudaMemsetAsync(it_sum, 0, sizeof(double) * 2 * (size_t)nper * p.wave_slots, st));
    NTRY_Q(launch_prep(nint, p, p.wave_slots, st));
    NTRY_Q(launch_batch_packed(nint, p, grid, smem, st));
    NTRY_Q(launch_reduce_items(p, st));
  }
  finalize_kernel<<<1, 1024, 0, st>>>(ndet, eps, s2, reinterpret_cast<const long long*>(na),
                                      reinterpret_cast<const long long*>(ncon), dres);
  NTRY_Q(cudaGetLastError());

  // ---- selection ----
  int64_t nsel = 0;
  if (k > 0) {
    gather_kernel<<<grid, 256, 0, st>>>(grid, nint, cap, tk_cnt, tk_e, tk_a, tk_key, p.tau_bits, cand_e, cand_a,
                                        cand_key, d_ncand, (int64_t)maxc, d_err);
    int ncand = 0;
    NTRY_Q(cudaMemcpyAsync(&ncand, d_ncand, sizeof(int), cudaMemcpyDeviceToHost, st));
    NTRY_Q(cudaStreamSynchronize(st));
    if (ncand > 0) {
      const int sb = (ncand + 255) / 256;
      iota_kernel<<<sb, 256, 0, st>>>(ncand, perm);
      int32_t *pa = perm, *pb = perm2;
      for (int pass = 0; pass <= nw; pass++) {
        const int word = (pass < nw) ? (nw - 1 - pass) : nw;
        sortkey_kernel<<<sb, 256, 0, st>>>(ncand, nint, word, cand_e, cand_key, pa, skey);
        NTRY_Q(cub::DeviceRadixSort::SortPairs(cub_tmp, tmp2, skey, skey2, pa, pb, ncand, 0, 64, st));
        int32_t* t = pa;
        pa = pb;
        pb = t;
      }
      nsel = ncand < k ? ncand : k;
      select_out_kernel<<<(int)((nsel + 255) / 256), 256, 0, st>>>((int)nsel, nint, pa, cand_e, cand_a, cand_key,
                                                                 sel_dets, sel_e, nullptr);
      NTRY_Q(cudaGetLastError());
    }
  }

  DevResult hres;
  unsigned long long hacc[9];
  NTRY_Q(cudaMemcpyAsync(&hres, dres, sizeof(hres), cudaMemcpyDeviceToHost, st));
  NTRY_Q(cudaMemcpyAsync(hacc, acc, sizeof(hacc), cudaMemcpyDeviceToHost, st));
  NTRY_Q(cudaStreamSynchronize(st));
  if (reinterpret_cast<int*>(hacc + 6)[0] & 8) return nfail(QP_ECUDA, "internal error: bucket capacity exceeded");
  if (reinterpret_cast<int*>(hacc + 6)[0] & 64)
    return nfail(QP_ENOTSUP, "coefficients times integrals beyond 2^93: outside the exact accumulator's range");
  res->e_pt2 = hres.e_pt2;
  res->sum_e_over_d = hres.s2;
  res->n_perturbers = hres.na;
  res->n_connections = hres.ncon;
  res->n_selected = nsel;
  res->n_tiny = (int64_t)hacc[3];
  res->perturber_digest[0] = hacc[0];
  res->perturber_digest[1] = hacc[1];
  double md;
  memcpy(&md, &hacc[2], sizeof(md));
  res->min_abs_denominator = md;
  res->z = 1.0 / (1.0 + res->sum_e_over_d);  // renormalised PT2 (Sec. "Renormalized PT2")
  res->e_rpt2 = e0 + res->z * res->e_pt2;
  if (hres.na > 0 && md < 1e-12) return nfail(QP_ESINGULAR, "a denominator E0 - H_aa is below 1e-12");
  return QP_OK;
}
