// davidson.cu -- the Hamiltonian over Psi0 and its lowest eigenpair on sm_103a
// (Quantum Package 2.0, arXiv:1902.08154, Sec. "Davidson diagonalization":
// the variational step of CIPSI, E0 and c_I as the lowest eigenpair of H in
// the internal space).
//
//   * H is built once per call as a CSR matrix of the pairs (I, J) at
//     excitation degree 1 or 2 (Slater-Condon rules, Eqs. Hij), plus its
//     diagonal.  Pairs are found through the spin-up and spin-down strings
//     of the determinants (the paper's DISCIUS-like search, see below), or,
//     as a cross-check, by a tiled all-pairs test (each CTA keeps a tile of
//     rows in shared memory and streams every determinant once); they are
//     written in any order and then sorted by column within each row, so that
//     the products below add in a fixed order.
//   * sigma = H u by one warp per row.
//   * Davidson's method (E. R. Davidson, J. Comput. Phys. 17, 87 (1975)) with
//     the diagonal preconditioner t = r / (theta - H_II): basis vectors,
//     their products with H and every dot product stay on the device; only
//     the small subspace matrix goes to the host, where a cyclic Jacobi
//     eigensolver (Golub & Van Loan, Sec. 8.5) diagonalises it.
#include <cuda_runtime.h>

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <cub/device/device_segmented_radix_sort.cuh>
#include <cmath>
#include <cstring>
#include <vector>

#include "../../include/qp_pt2.h"
#include "common.cuh"

namespace qp {
namespace {

constexpr int kRows = 64;  // rows of H per CTA in the pair search
constexpr int kMaxBasis = 32;

#define DV_TRY(expr)                                                \
  do {                                                              \
    cudaError_t e_ = (expr);                                        \
    if (e_ != cudaSuccess) return report(QP_ECUDA, cudaGetErrorString(e_)); \
  } while (0)

// Up to two set bits of m (spin-orbital codes base + bit), in ascending order.
template <int NINT>
__device__ __forceinline__ void take_bits(const uint64_t* m, int base, int* out, int* n) {
#pragma unroll
  for (int w = 0; w < NINT; w++) {
    uint64_t b = m[w];
    while (b && *n < 2) {
      out[(*n)++] = base + 64 * w + __ffsll((long long)b) - 1;
      b &= b - 1;
    }
  }
}

// <I|H|J> for two determinants at excitation degree 1 or 2: holes are the
// spin orbitals of I missing from J, particles those of J missing from I.
template <int NINT>
__device__ double hij_pair(const uint64_t* I, const uint64_t* J, int norb, const double* h, const double* eri) {
  int ho[2], pa[2], nh = 0, np = 0;
  for (int s = 0; s < 2; s++) {
    uint64_t x[NINT], y[NINT];
#pragma unroll
    for (int w = 0; w < NINT; w++) {
      x[w] = I[s * NINT + w] & ~J[s * NINT + w];
      y[w] = J[s * NINT + w] & ~I[s * NINT + w];
    }
    take_bits<NINT>(x, s * norb, ho, &nh);
    take_bits<NINT>(y, s * norb, pa, &np);
  }
  if (nh == 1) {  // single a -> b: h_ab + sum_{q in I} [(ab|qq) - delta (aq|qb)]
    const int s = ho[0] >= norb, a = ho[0] - s * norb, b = pa[0] - s * norb;
    double v = h[a * norb + b];
    for (int t = 0; t < 2; t++) {
#pragma unroll
      for (int w = 0; w < NINT; w++) {
        uint64_t bits = I[t * NINT + w];
        while (bits) {
          const int q = 64 * w + __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          v += eri[eri_index(a, b, q, q)];
          if (t == s) v -= eri[eri_index(a, q, q, b)];
        }
      }
    }
    const int par = count_between<NINT>(I + s * NINT, a < b ? a : b, a < b ? b : a) & 1;
    return par ? -v : v;
  }
  // double: holes h1 < h2 and particles p1 < p2 (codes), paired 1-1 and 2-2
  const int s1 = ho[0] >= norb, s2 = ho[1] >= norb;
  const int h1 = ho[0] - s1 * norb, h2 = ho[1] - s2 * norb;
  const int p1 = pa[0] - s1 * norb, p2 = pa[1] - s2 * norb;
  uint64_t w1[NINT];
#pragma unroll
  for (int w = 0; w < NINT; w++) w1[w] = I[s1 * NINT + w];
  int par = count_between<NINT>(w1, h1 < p1 ? h1 : p1, h1 < p1 ? p1 : h1);
#pragma unroll
  for (int w = 0; w < NINT; w++) {  // apply h1 -> p1, then count h2 -> p2 on the result
    if (w == (h1 >> 6)) w1[w] &= ~(1ull << (h1 & 63));
    if (w == (p1 >> 6)) w1[w] |= 1ull << (p1 & 63);
  }
  par += (s1 == s2) ? count_between<NINT>(w1, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2)
                    : count_between<NINT>(I + s2 * NINT, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  double v = eri[eri_index(h1, p1, h2, p2)];
  if (s1 == s2) v -= eri[eri_index(h1, p2, h2, p1)];
  return (par & 1) ? -v : v;
}

// H_II = sum_i h_ii + sum_{i<j} [(ii|jj) - delta_spin (ij|ji)] over I's spin orbitals.
template <int NINT>
__global__ void diag_kernel(int64_t n, const uint64_t* dets, int norb, const double* h, const double* Jm,
                            const double* Km, double* diag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint64_t* d = dets + i * 2 * NINT;
  int occ[kMaxElec], ne = 0;
  for (int s = 0; s < 2; s++)
    for (int w = 0; w < NINT; w++) {
      uint64_t b = d[s * NINT + w];
      while (b && ne < kMaxElec) {
        occ[ne++] = s * norb + 64 * w + __ffsll((long long)b) - 1;
        b &= b - 1;
      }
    }
  double e = 0.0;
  for (int a = 0; a < ne; a++) {
    const int sa = occ[a] >= norb, pa = occ[a] - sa * norb;
    e += h[pa * norb + pa];
    for (int b = 0; b < a; b++) {
      const int sb = occ[b] >= norb, pb = occ[b] - sb * norb;
      e += Jm[pa * norb + pb];
      if (sa == sb) e -= Km[pa * norb + pb];
    }
  }
  diag[i] = e;
}

// Pair search over a tile of kRows rows: COUNT pass writes row counts,
// otherwise (col, <I|H|J>) pairs go to each row's next free slots.
template <int NINT, bool COUNT>
__global__ void pairs_kernel(int64_t n, const uint64_t* dets, int norb, const double* h, const double* eri,
                             int* rowcnt, const int64_t* rowptr, int* cursor, int* cols, double* vals, int* err) {
  constexpr int NW = 2 * NINT;
  __shared__ uint64_t rows[kRows][NW];
  __shared__ int cnt[kRows];
  const int64_t r0 = (int64_t)blockIdx.x * kRows;
  const int nr = (int)((n - r0) < kRows ? (n - r0) : kRows);
  for (int t = threadIdx.x; t < nr * NW; t += blockDim.x) rows[t / NW][t % NW] = dets[(r0 + t / NW) * NW + t % NW];
  if (threadIdx.x < kRows) cnt[threadIdx.x] = 0;
  __syncthreads();
  for (int64_t j = threadIdx.x; j < n; j += blockDim.x) {
    uint64_t J[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) J[w] = dets[j * NW + w];
    for (int r = 0; r < nr; r++) {
      int x = 0;
#pragma unroll
      for (int w = 0; w < NW; w++) x += __popcll(rows[r][w] ^ J[w]);
      if (x > 4) continue;
      if (x == 0) {
        if (r0 + r != j) atomicOr(err, 1);  // a repeated determinant
        continue;
      }
      if (COUNT) {
        atomicAdd(&cnt[r], 1);
      } else {
        const int64_t pos = rowptr[r0 + r] + atomicAdd(&cursor[r0 + r], 1);
        cols[pos] = (int)j;
        vals[pos] = hij_pair<NINT>(rows[r], J, norb, h, eri);
      }
    }
  }
  if (COUNT) {
    __syncthreads();
    if (threadIdx.x < nr) rowcnt[r0 + threadIdx.x] = cnt[threadIdx.x];
  }
}

// ---------------------------------------------------------------------------
// Connected pairs through the alpha and beta strings (Appendix "Davidson
// diagonalization": Psi0 = sum C_IJ |I_up J_dn>, same-spin excitations found
// along a row or a column of C, opposite-spin doubles by a spin-up single
// excitation followed by a spin-down one).  The determinants are grouped by
// their spin-up string and by their spin-down string; for row I:
//   (a) J with the spin-down string of I: spin-up excitation of degree 1 or 2;
//   (b) J with the spin-up string of I: spin-down excitation of degree 1 or 2;
//   (c) J whose spin-up string is a single excitation of I's (the string
//       neighbour lists) and whose spin-down string is a single excitation of
//       I's: the opposite-spin doubles.
// Every connected pair is met exactly once, and the work per row is the
// length of its lists instead of N_det.
// ---------------------------------------------------------------------------
struct SpinStrings {
  int nu = 0;             // distinct strings
  int* sid = nullptr;     // [n] string index of each determinant
  int* ptr = nullptr;     // [nu + 1] offsets into grp
  int* grp = nullptr;     // [n] determinants ordered by string
  uint64_t* ukey = nullptr;  // [nu][nint] the distinct strings
  int* nb_ptr = nullptr;  // [nu + 1] single-excitation neighbours (spin-up strings only)
  int* nb = nullptr;
};

__global__ void str_key_kernel(int64_t n, int nw, int off, const uint64_t* dets, const int* perm,
                               unsigned long long* key, int* val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int j = perm ? perm[i] : (int)i;
  key[i] = dets[(size_t)j * nw + off];
  val[i] = j;
}

template <int NINT>
__global__ void str_flag_kernel(int64_t n, int spin, const uint64_t* dets, const int* grp, int* flag) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  int f = (i == 0);
  if (i > 0) {
    const uint64_t* a = dets + (size_t)grp[i] * 2 * NINT + spin * NINT;
    const uint64_t* b = dets + (size_t)grp[i - 1] * 2 * NINT + spin * NINT;
#pragma unroll
    for (int w = 0; w < NINT; w++) f |= (a[w] != b[w]);
  }
  flag[i] = f;
}

template <int NINT>
__global__ void str_index_kernel(int64_t n, int spin, const uint64_t* dets, const int* grp, const int* flag,
                                 const int* incl, int* sid, int* ptr, uint64_t* ukey) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int id = incl[i] - 1;
  sid[grp[i]] = id;
  if (flag[i]) {
    ptr[id] = (int)i;
#pragma unroll
    for (int w = 0; w < NINT; w++) ukey[(size_t)id * NINT + w] = dets[(size_t)grp[i] * 2 * NINT + spin * NINT + w];
  }
}

// Single-excitation neighbours among the distinct strings (count, then fill).
template <int NINT, bool COUNT>
__global__ void str_nb_kernel(int nu, const uint64_t* ukey, int* cnt, const int* nb_ptr, int* nb) {
  const int u = blockIdx.x * blockDim.x + threadIdx.x;
  if (u >= nu) return;
  uint64_t a[NINT];
#pragma unroll
  for (int w = 0; w < NINT; w++) a[w] = ukey[(size_t)u * NINT + w];
  int c = 0;
  for (int v = 0; v < nu; v++) {
    int d = 0;
#pragma unroll
    for (int w = 0; w < NINT; w++) d += __popcll(a[w] ^ ukey[(size_t)v * NINT + w]);
    if (d == 2) {
      if (!COUNT) nb[nb_ptr[u] + c] = v;
      c++;
    }
  }
  if (COUNT) cnt[u] = c;
}

template <int NINT>
__device__ __forceinline__ int spin_degree(const uint64_t* I, const uint64_t* J, int spin) {
  int d = 0;
#pragma unroll
  for (int w = 0; w < NINT; w++) d += __popcll(I[spin * NINT + w] ^ J[spin * NINT + w]);
  return d >> 1;
}

// One warp per row I: COUNT writes the number of connected J, otherwise the
// (column, <I|H|J>) pairs go to the row's next free slots.
template <int NINT, bool COUNT>
__global__ void str_pairs_kernel(int64_t n, const uint64_t* dets, int norb, const double* h, const double* eri,
                                 const int* aid, const int* aptr, const int* agrp, const int* anb_ptr,
                                 const int* anb, const int* bid, const int* bptr, const int* bgrp, int* rowcnt,
                                 const int64_t* rowptr, int* cursor, int* cols, double* vals, int* err) {
  constexpr int NW = 2 * NINT;
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  uint64_t I[NW];
#pragma unroll
  for (int w = 0; w < NW; w++) I[w] = dets[(size_t)row * NW + w];
  int cnt = 0;
  auto emit = [&](int j) {
    if (COUNT) {
      cnt++;
    } else {
      const int64_t pos = rowptr[row] + atomicAdd(&cursor[row], 1);
      cols[pos] = j;
      vals[pos] = hij_pair<NINT>(I, dets + (size_t)j * NW, norb, h, eri);
    }
  };
  {  // (a) the same spin-down string: spin-up excitations
    const int b = bid[row];
    for (int k = bptr[b] + lane; k < bptr[b + 1]; k += 32) {
      const int j = bgrp[k];
      if (j == (int)row) continue;
      const int d = spin_degree<NINT>(I, dets + (size_t)j * NW, 0);
      if (d == 0) atomicOr(err, 1);  // a repeated determinant
      else if (d <= 2) emit(j);
    }
  }
  const int a = aid[row];
  for (int k = aptr[a] + lane; k < aptr[a + 1]; k += 32) {  // (b) the same spin-up string
    const int j = agrp[k];
    if (j == (int)row) continue;
    const int d = spin_degree<NINT>(I, dets + (size_t)j * NW, 1);
    if (d >= 1 && d <= 2) emit(j);
  }
  for (int q = anb_ptr[a]; q < anb_ptr[a + 1]; q++) {  // (c) spin-up single, then spin-down single
    const int a2 = anb[q];
    for (int k = aptr[a2] + lane; k < aptr[a2 + 1]; k += 32) {
      const int j = agrp[k];
      if (spin_degree<NINT>(I, dets + (size_t)j * NW, 1) == 1) emit(j);
    }
  }
  if (COUNT) {
#pragma unroll
    for (int o = 16; o; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if (lane == 0) rowcnt[row] = cnt;
  }
}

// Y[k] = H X[k] for nvec vectors of length n: one warp per row.
__global__ void spmv_kernel(int64_t n, int nvec, const int64_t* rowptr, const int* cols, const double* vals,
                            const double* diag, const double* X, double* Y) {
  const int64_t row = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (row >= n) return;
  for (int k = 0; k < nvec; k++) {
    const double* x = X + (size_t)k * n;
    double acc = 0.0;
    for (int64_t q = rowptr[row] + lane; q < rowptr[row + 1]; q += 32) acc += vals[q] * x[cols[q]];
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (lane == 0) Y[(size_t)k * n + row] = diag[row] * x[row] + acc;
  }
}

// out[k] = V[k] . y for k < m (one CTA per k).
__global__ void dots_kernel(int64_t n, const double* V, const double* y, double* out) {
  const double* v = V + (size_t)blockIdx.x * n;
  double acc = 0.0;
  for (int64_t i = threadIdx.x; i < n; i += blockDim.x) acc += v[i] * y[i];
  __shared__ double part[32];
#pragma unroll
  for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x < 32) {
    acc = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if (threadIdx.x == 0) out[blockIdx.x] = acc;
  }
}

// out = sum_k s[k] V[k] (+ beta * out when accumulate).
__global__ void combine_kernel(int64_t n, int m, const double* V, const double* s, double* out, double beta) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double acc = beta != 0.0 ? beta * out[i] : 0.0;
  for (int k = 0; k < m; k++) acc += s[k] * V[(size_t)k * n + i];
  out[i] = acc;
}

// r = w - theta x; t = r / (theta - H_II), with |theta - H_II| kept above 1e-6.
__global__ void correction_kernel(int64_t n, const double* x, const double* w, const double* diag, double theta,
                                  double* r, double* t) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double ri = w[i] - theta * x[i];
  double den = theta - diag[i];
  if (fabs(den) < 1e-6) den = den < 0 ? -1e-6 : 1e-6;
  r[i] = ri;
  t[i] = ri / den;
}

__global__ void scale_kernel(int64_t n, double a, const double* x, double* y) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = a * x[i];
}

// Eigenpairs of the symmetric m x m matrix a (row-major, overwritten) by
// cyclic Jacobi rotations; eigenvalues in w, eigenvectors in the columns of v.
void jacobi_eigen(int m, std::vector<double>& a, std::vector<double>& w, std::vector<double>& v) {
  v.assign((size_t)m * m, 0.0);
  for (int i = 0; i < m; i++) v[(size_t)i * m + i] = 1.0;
  for (int sweep = 0; sweep < 100; sweep++) {
    double off = 0.0, tot = 0.0;
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) {
        tot += a[(size_t)i * m + j] * a[(size_t)i * m + j];
        if (i != j) off += a[(size_t)i * m + j] * a[(size_t)i * m + j];
      }
    if (off <= 1e-30 * tot || off == 0.0) break;
    for (int p = 0; p < m; p++)
      for (int q = p + 1; q < m; q++) {
        const double apq = a[(size_t)p * m + q];
        if (apq == 0.0) continue;
        const double app = a[(size_t)p * m + p], aqq = a[(size_t)q * m + q];
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < m; k++) {  // A <- J^T A J
          const double akp = a[(size_t)k * m + p], akq = a[(size_t)k * m + q];
          a[(size_t)k * m + p] = c * akp - s * akq;
          a[(size_t)k * m + q] = s * akp + c * akq;
        }
        for (int k = 0; k < m; k++) {
          const double apk = a[(size_t)p * m + k], aqk = a[(size_t)q * m + k];
          a[(size_t)p * m + k] = c * apk - s * aqk;
          a[(size_t)q * m + k] = s * apk + c * aqk;
        }
        for (int k = 0; k < m; k++) {
          const double vkp = v[(size_t)k * m + p], vkq = v[(size_t)k * m + q];
          v[(size_t)k * m + p] = c * vkp - s * vkq;
          v[(size_t)k * m + q] = s * vkp + c * vkq;
        }
      }
  }
  w.resize(m);
  for (int i = 0; i < m; i++) w[i] = a[(size_t)i * m + i];
}

// Device buffers of one Hamiltonian (freed on scope exit).
struct DevMem {
  std::vector<void*> ptrs;
  ~DevMem() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <typename T>
  T* alloc(size_t count) {
    void* p = nullptr;
    if (cudaMalloc(&p, sizeof(T) * (count ? count : 1)) != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<T*>(p);
  }
};

struct HMat {
  int64_t n = 0, nnz = 0;
  int64_t* rowptr = nullptr;
  int* cols = nullptr;
  double *vals = nullptr, *diag = nullptr;
};

// The determinants grouped by their string of one spin (radix sort of the
// string words, least significant word first), the distinct strings, and
// for the spin-up strings their single-excitation neighbours.
int build_strings(const CtxView& c, int64_t n, const uint64_t* d_dets, int spin, bool neighbours, DevMem& mem,
                  SpinStrings* S) {
  cudaStream_t st = c.st;
  const int nint = c.nint, nw = 2 * nint;
  const unsigned nb = (unsigned)((n + 255) / 256);
  unsigned long long* key = mem.alloc<unsigned long long>(n);
  unsigned long long* key2 = mem.alloc<unsigned long long>(n);
  int* val = mem.alloc<int>(n);
  int* perm = mem.alloc<int>(n);
  int* flag = mem.alloc<int>(n);
  int* incl = mem.alloc<int>(n);
  S->sid = mem.alloc<int>(n);
  S->grp = perm;
  if (!key || !key2 || !val || !perm || !flag || !incl || !S->sid)
    return report(QP_ENOMEM, "device allocation for the spin strings failed");
  size_t tmp = 0, tmp2 = 0;
  cub::DeviceRadixSort::SortPairs(nullptr, tmp, key, key2, val, perm, (int)n, 0, 64, st);
  cub::DeviceScan::InclusiveSum(nullptr, tmp2, flag, incl, (int)n, st);
  void* d_tmp = mem.alloc<unsigned char>(tmp > tmp2 ? tmp : tmp2);
  if (!d_tmp) return report(QP_ENOMEM, "device allocation for the spin strings failed");
  for (int w = nint - 1; w >= 0; w--) {  // least significant word first; the sorts are stable
    str_key_kernel<<<nb, 256, 0, st>>>(n, nw, spin * nint + w, d_dets, w == nint - 1 ? nullptr : perm, key, val);
    DV_TRY(cub::DeviceRadixSort::SortPairs(d_tmp, tmp, key, key2, val, perm, (int)n, 0, 64, st));
  }
  if (nint == 1) str_flag_kernel<1><<<nb, 256, 0, st>>>(n, spin, d_dets, perm, flag);
  else str_flag_kernel<2><<<nb, 256, 0, st>>>(n, spin, d_dets, perm, flag);
  DV_TRY(cub::DeviceScan::InclusiveSum(d_tmp, tmp2, flag, incl, (int)n, st));
  int nu = 0;
  DV_TRY(cudaMemcpyAsync(&nu, incl + (n - 1), sizeof(int), cudaMemcpyDeviceToHost, st));
  DV_TRY(cudaStreamSynchronize(st));
  S->nu = nu;
  S->ptr = mem.alloc<int>((size_t)nu + 1);
  S->ukey = mem.alloc<uint64_t>((size_t)nu * nint);
  if (!S->ptr || !S->ukey) return report(QP_ENOMEM, "device allocation for the spin strings failed");
  if (nint == 1) str_index_kernel<1><<<nb, 256, 0, st>>>(n, spin, d_dets, perm, flag, incl, S->sid, S->ptr, S->ukey);
  else str_index_kernel<2><<<nb, 256, 0, st>>>(n, spin, d_dets, perm, flag, incl, S->sid, S->ptr, S->ukey);
  const int nn = (int)n;
  DV_TRY(cudaMemcpyAsync(S->ptr + nu, &nn, sizeof(int), cudaMemcpyHostToDevice, st));
  if (!neighbours) return QP_OK;
  int* cnt = mem.alloc<int>((size_t)nu + 1);
  S->nb_ptr = mem.alloc<int>((size_t)nu + 1);
  if (!cnt || !S->nb_ptr) return report(QP_ENOMEM, "device allocation for the spin strings failed");
  DV_TRY(cudaMemsetAsync(cnt, 0, sizeof(int) * ((size_t)nu + 1), st));
  const unsigned nbu = (unsigned)((nu + 127) / 128);
  if (nint == 1) str_nb_kernel<1, true><<<nbu, 128, 0, st>>>(nu, S->ukey, cnt, nullptr, nullptr);
  else str_nb_kernel<2, true><<<nbu, 128, 0, st>>>(nu, S->ukey, cnt, nullptr, nullptr);
  size_t tmp3 = 0;
  cub::DeviceScan::ExclusiveSum(nullptr, tmp3, cnt, S->nb_ptr, nu + 1, st);
  void* d_tmp3 = mem.alloc<unsigned char>(tmp3);
  if (!d_tmp3) return report(QP_ENOMEM, "device allocation for the spin strings failed");
  DV_TRY(cub::DeviceScan::ExclusiveSum(d_tmp3, tmp3, cnt, S->nb_ptr, nu + 1, st));
  int tot = 0;
  DV_TRY(cudaMemcpyAsync(&tot, S->nb_ptr + nu, sizeof(int), cudaMemcpyDeviceToHost, st));
  DV_TRY(cudaStreamSynchronize(st));
  S->nb = mem.alloc<int>((size_t)tot);
  if (!S->nb) return report(QP_ENOMEM, "device allocation for the spin strings failed");
  if (nint == 1) str_nb_kernel<1, false><<<nbu, 128, 0, st>>>(nu, S->ukey, nullptr, S->nb_ptr, S->nb);
  else str_nb_kernel<2, false><<<nbu, 128, 0, st>>>(nu, S->ukey, nullptr, S->nb_ptr, S->nb);
  DV_TRY(cudaGetLastError());
  return QP_OK;
}

// search: kSearchStrings (default) or kSearchAllPairs (the tiled test of
// every pair, O(N_det^2), kept as a cross-check)
int build_h(const CtxView& c, int64_t n, const uint64_t* d_dets, DevMem& mem, HMat* H, int search = 0) {
  cudaStream_t st = c.st;
  H->n = n;
  int* rowcnt = mem.alloc<int>(n + 1);
  int* cursor = mem.alloc<int>(n);
  int* err = mem.alloc<int>(1);
  H->rowptr = mem.alloc<int64_t>(n + 1);
  H->diag = mem.alloc<double>(n);
  int64_t* cnt64 = mem.alloc<int64_t>(n + 1);
  if (!rowcnt || !cursor || !err || !H->rowptr || !H->diag || !cnt64)
    return report(QP_ENOMEM, "device allocation for the Hamiltonian failed");
  DV_TRY(cudaMemsetAsync(err, 0, sizeof(int), st));
  DV_TRY(cudaMemsetAsync(rowcnt, 0, sizeof(int) * (n + 1), st));
  DV_TRY(cudaMemsetAsync(cursor, 0, sizeof(int) * n, st));
  const unsigned tiles = (unsigned)((n + kRows - 1) / kRows), nb = (unsigned)((n + 255) / 256);
  const unsigned nwarp = (unsigned)((n * 32 + 255) / 256);
  SpinStrings SA, SB;
  int rc;
  if (search == 0) {
    if ((rc = build_strings(c, n, d_dets, 0, true, mem, &SA)) || (rc = build_strings(c, n, d_dets, 1, false, mem, &SB)))
      return rc;
  }
  // one pass of the pair search: COUNT (row counts) or fill
  auto pairs = [&](bool count, const int64_t* rowptr, int* cols, double* vals) {
    if (search == 0) {
      if (c.nint == 1) {
        if (count)
          str_pairs_kernel<1, true><<<nwarp, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, SA.sid, SA.ptr, SA.grp,
                                                           SA.nb_ptr, SA.nb, SB.sid, SB.ptr, SB.grp, rowcnt, rowptr,
                                                           cursor, cols, vals, err);
        else
          str_pairs_kernel<1, false><<<nwarp, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, SA.sid, SA.ptr, SA.grp,
                                                            SA.nb_ptr, SA.nb, SB.sid, SB.ptr, SB.grp, rowcnt, rowptr,
                                                            cursor, cols, vals, err);
      } else {
        if (count)
          str_pairs_kernel<2, true><<<nwarp, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, SA.sid, SA.ptr, SA.grp,
                                                           SA.nb_ptr, SA.nb, SB.sid, SB.ptr, SB.grp, rowcnt, rowptr,
                                                           cursor, cols, vals, err);
        else
          str_pairs_kernel<2, false><<<nwarp, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, SA.sid, SA.ptr, SA.grp,
                                                            SA.nb_ptr, SA.nb, SB.sid, SB.ptr, SB.grp, rowcnt, rowptr,
                                                            cursor, cols, vals, err);
      }
    } else if (c.nint == 1) {
      if (count)
        pairs_kernel<1, true><<<tiles, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, rowcnt, nullptr, nullptr, nullptr,
                                                     nullptr, err);
      else
        pairs_kernel<1, false><<<tiles, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, nullptr, rowptr, cursor, cols,
                                                      vals, err);
    } else {
      if (count)
        pairs_kernel<2, true><<<tiles, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, rowcnt, nullptr, nullptr, nullptr,
                                                     nullptr, err);
      else
        pairs_kernel<2, false><<<tiles, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.eri, nullptr, rowptr, cursor, cols,
                                                      vals, err);
    }
  };
  if (c.nint == 1) diag_kernel<1><<<nb, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.Jm, c.Km, H->diag);
  else diag_kernel<2><<<nb, 256, 0, st>>>(n, d_dets, c.norb, c.h, c.Jm, c.Km, H->diag);
  pairs(true, nullptr, nullptr, nullptr);
  DV_TRY(cudaGetLastError());
  // row counts (int) -> 64-bit exclusive offsets
  std::vector<int> hc((size_t)n);
  DV_TRY(cudaMemcpyAsync(hc.data(), rowcnt, sizeof(int) * n, cudaMemcpyDeviceToHost, st));
  int herr = 0;
  DV_TRY(cudaMemcpyAsync(&herr, err, sizeof(int), cudaMemcpyDeviceToHost, st));
  DV_TRY(cudaStreamSynchronize(st));
  if (herr) return report(QP_EDUP, "duplicate determinant in Psi0");
  std::vector<int64_t> hp((size_t)n + 1, 0);
  for (int64_t i = 0; i < n; i++) hp[i + 1] = hp[i] + hc[i];
  H->nnz = hp[n];
  DV_TRY(cudaMemcpyAsync(H->rowptr, hp.data(), sizeof(int64_t) * (n + 1), cudaMemcpyHostToDevice, st));
  H->cols = mem.alloc<int>(H->nnz);
  H->vals = mem.alloc<double>(H->nnz);
  int* cols2 = mem.alloc<int>(H->nnz);
  double* vals2 = mem.alloc<double>(H->nnz);
  if (!H->cols || !H->vals || !cols2 || !vals2) return report(QP_ENOMEM, "device allocation for the Hamiltonian failed");
  pairs(false, H->rowptr, cols2, vals2);
  DV_TRY(cudaGetLastError());
  if (H->nnz > 0) {  // columns ascending within each row: a fixed order of the sums
    if (H->nnz >= (1ll << 31) || n >= (1ll << 31)) return report(QP_ENOTSUP, "Hamiltonian above 2^31 entries");
    size_t tmp = 0;
    cub::DeviceSegmentedRadixSort::SortPairs(nullptr, tmp, cols2, H->cols, vals2, H->vals, (int)H->nnz, (int)n,
                                             H->rowptr, H->rowptr + 1, 0, 32, st);
    void* d_tmp = mem.alloc<unsigned char>(tmp);
    if (!d_tmp) return report(QP_ENOMEM, "device allocation for the Hamiltonian failed");
    DV_TRY(cub::DeviceSegmentedRadixSort::SortPairs(d_tmp, tmp, cols2, H->cols, vals2, H->vals, (int)H->nnz,
                                                    (int)n, H->rowptr, H->rowptr + 1, 0, 32, st));
  }
  return QP_OK;
}

int check_inputs(const CtxView& c, int64_t n, const uint64_t* dets) {
  if (n < 1) return report(QP_EINVAL, "ndet must be positive");
  if (n >= (1ll << 31)) return report(QP_EINVAL, "ndet must be below 2^31");
  if (!dets) return report(QP_EINVAL, "dets is NULL");
  (void)c;
  return QP_OK;
}

// Copies a caller array to the device unless it is there already.
template <typename T>
int to_device(const T* src, size_t count, cudaStream_t st, DevMem& mem, const T** out) {
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, src) == cudaSuccess &&
      (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged)) {
    *out = src;
    return QP_OK;
  }
  cudaGetLastError();
  T* d = mem.alloc<T>(count);
  if (!d) return report(QP_ENOMEM, "device allocation failed");
  DV_TRY(cudaMemcpyAsync(d, src, sizeof(T) * count, cudaMemcpyHostToDevice, st));
  *out = d;
  return QP_OK;
}

int validate(const CtxView& c, int64_t n, const uint64_t* d_dets) {
  // occupation counts and bits beyond norb, on the host (one copy of Psi0)
  const int nw = 2 * c.nint;
  std::vector<uint64_t> hd((size_t)n * nw);
  DV_TRY(cudaMemcpyAsync(hd.data(), d_dets, sizeof(uint64_t) * n * nw, cudaMemcpyDeviceToHost, c.st));
  DV_TRY(cudaStreamSynchronize(c.st));
  for (int64_t i = 0; i < n; i++)
    for (int s = 0; s < 2; s++) {
      int cnt = 0;
      for (int w = 0; w < c.nint; w++) {
        const uint64_t b = hd[(size_t)i * nw + s * c.nint + w];
        const int lim = c.norb - 64 * w;  // orbitals held by this word
        const uint64_t valid = lim >= 64 ? ~0ull : (lim <= 0 ? 0ull : (1ull << lim) - 1);
        if (b & ~valid) return report(QP_EINVAL, "a bit beyond norb is set");
        cnt += __builtin_popcountll(b);
      }
      if (cnt != (s ? c.nbeta : c.nalpha)) return report(QP_EINVAL, "a determinant has the wrong occupation");
    }
  return QP_OK;
}

}  // namespace
}  // namespace qp

using namespace qp;

extern "C" int qp_pt2_sigma(qp_pt2_ctx* ctx, int64_t ndet, const uint64_t* dets, int nvec, const double* U,
                            double* S) {
  CtxView c;
  int rc = ctx_view(ctx, &c);
  if (rc) return rc;
  if ((rc = check_inputs(c, ndet, dets))) return rc;
  if (nvec < 1 || !U || !S) return report(QP_EINVAL, "nvec must be positive and U, S non-NULL");
  DevMem mem;
  const uint64_t* d_dets;
  const double* d_u;
  if ((rc = to_device(dets, (size_t)ndet * 2 * c.nint, c.st, mem, &d_dets))) return rc;
  if ((rc = validate(c, ndet, d_dets))) return rc;
  if ((rc = to_device(U, (size_t)ndet * nvec, c.st, mem, &d_u))) return rc;
  HMat H;
  if ((rc = build_h(c, ndet, d_dets, mem, &H))) return rc;
  double* d_s = mem.alloc<double>((size_t)ndet * nvec);
  if (!d_s) return report(QP_ENOMEM, "device allocation failed");
  spmv_kernel<<<(unsigned)((ndet * 32 + 255) / 256), 256, 0, c.st>>>(ndet, nvec, H.rowptr, H.cols, H.vals, H.diag,
                                                                     d_u, d_s);
  DV_TRY(cudaGetLastError());
  DV_TRY(cudaMemcpyAsync(S, d_s, sizeof(double) * ndet * nvec, cudaMemcpyDefault, c.st));
  DV_TRY(cudaStreamSynchronize(c.st));
  return QP_OK;
}

extern "C" int qp_pt2_hamiltonian(qp_pt2_ctx* ctx, int64_t ndet, const uint64_t* dets, int search, int64_t* nnz,
                                  int64_t* rowptr, int32_t* cols, double* vals, double* diag, double* build_ms) {
  CtxView c;
  int rc = ctx_view(ctx, &c);
  if (rc) return rc;
  if ((rc = check_inputs(c, ndet, dets))) return rc;
  if (!nnz) return report(QP_EINVAL, "nnz is NULL");
  if (search != 0 && search != 1) return report(QP_EINVAL, "search must be 0 (spin strings) or 1 (all pairs)");
  DevMem mem;
  const uint64_t* d_dets;
  if ((rc = to_device(dets, (size_t)ndet * 2 * c.nint, c.st, mem, &d_dets))) return rc;
  if ((rc = validate(c, ndet, d_dets))) return rc;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaEventCreate(&e0);
  cudaEventCreate(&e1);
  cudaEventRecord(e0, c.st);
  HMat H;
  rc = build_h(c, ndet, d_dets, mem, &H, search);
  cudaEventRecord(e1, c.st);
  cudaEventSynchronize(e1);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, e0, e1);
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (rc) return rc;
  *nnz = H.nnz;
  if (build_ms) *build_ms = ms;
  if (rowptr) DV_TRY(cudaMemcpyAsync(rowptr, H.rowptr, sizeof(int64_t) * (ndet + 1), cudaMemcpyDefault, c.st));
  if (cols && H.nnz) DV_TRY(cudaMemcpyAsync(cols, H.cols, sizeof(int) * H.nnz, cudaMemcpyDefault, c.st));
  if (vals && H.nnz) DV_TRY(cudaMemcpyAsync(vals, H.vals, sizeof(double) * H.nnz, cudaMemcpyDefault, c.st));
  if (diag) DV_TRY(cudaMemcpyAsync(diag, H.diag, sizeof(double) * ndet, cudaMemcpyDefault, c.st));
  DV_TRY(cudaStreamSynchronize(c.st));
  return QP_OK;
}

extern "C" int qp_pt2_davidson(qp_pt2_ctx* ctx, int64_t ndet, const uint64_t* dets, const double* guess,
                               double tol, int max_iter, double* coefs, double* e0, qp_pt2_davidson_info* info) {
  CtxView c;
  int rc = ctx_view(ctx, &c);
  if (rc) return rc;
  if ((rc = check_inputs(c, ndet, dets))) return rc;
  if (!coefs || !e0) return report(QP_EINVAL, "coefs or e0 is NULL");
  if (!(tol > 0.0) || max_iter < 1) return report(QP_EINVAL, "tol must be positive and max_iter at least 1");
  cudaStream_t st = c.st;
  const int64_t n = ndet;
  const unsigned nb = (unsigned)((n + 255) / 256), nspmv = (unsigned)((n * 32 + 255) / 256);
  DevMem mem;
  const uint64_t* d_dets;
  if ((rc = to_device(dets, (size_t)n * 2 * c.nint, st, mem, &d_dets))) return rc;
  if ((rc = validate(c, n, d_dets))) return rc;
  struct Events {  // destroyed on every return
    cudaEvent_t e[3] = {nullptr, nullptr, nullptr};
    Events() {
      for (auto& x : e) cudaEventCreate(&x);
    }
    ~Events() {
      for (auto& x : e)
        if (x) cudaEventDestroy(x);
    }
  } evs;
  cudaEvent_t ev0 = evs.e[0], ev1 = evs.e[1], ev2 = evs.e[2];
  cudaEventRecord(ev0, st);
  HMat H;
  if ((rc = build_h(c, n, d_dets, mem, &H))) return rc;
  cudaEventRecord(ev1, st);
  const int mmax = (int)(n < kMaxBasis ? n : kMaxBasis);
  double* V = mem.alloc<double>((size_t)mmax * n);
  double* W = mem.alloc<double>((size_t)mmax * n);
  double* x = mem.alloc<double>(n);
  double* w = mem.alloc<double>(n);
  double* r = mem.alloc<double>(n);
  double* t = mem.alloc<double>(n);
  double* d_small = mem.alloc<double>(2 * kMaxBasis + 2);
  if (!V || !W || !x || !w || !r || !t || !d_small) return report(QP_ENOMEM, "device allocation for Davidson failed");
  // first basis vector: the guess, or the determinant of lowest H_II
  std::vector<double> hv((size_t)n);
  if (guess) {
    DV_TRY(cudaMemcpyAsync(hv.data(), guess, sizeof(double) * n, cudaMemcpyDefault, st));
    DV_TRY(cudaStreamSynchronize(st));
  } else {
    DV_TRY(cudaMemcpyAsync(hv.data(), H.diag, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
    DV_TRY(cudaStreamSynchronize(st));
    int64_t best = 0;
    for (int64_t i = 1; i < n; i++)
      if (hv[i] < hv[best]) best = i;
    std::fill(hv.begin(), hv.end(), 0.0);
    hv[best] = 1.0;
  }
  double nrm = 0.0;
  for (double v : hv) nrm += v * v;
  if (!(nrm > 0.0) || !std::isfinite(nrm)) return report(QP_EINVAL, "the guess vector is zero or not finite");
  for (double& v : hv) v /= std::sqrt(nrm);
  DV_TRY(cudaMemcpyAsync(V, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  auto hmul = [&](const double* in, double* out) {
    spmv_kernel<<<nspmv, 256, 0, st>>>(n, 1, H.rowptr, H.cols, H.vals, H.diag, in, out);
  };
  auto dots = [&](int m, const double* base, const double* y, double* out_host) -> int {
    dots_kernel<<<m, 256, 0, st>>>(n, base, y, d_small);
    DV_TRY(cudaMemcpyAsync(out_host, d_small, sizeof(double) * m, cudaMemcpyDeviceToHost, st));
    DV_TRY(cudaStreamSynchronize(st));
    return QP_OK;
  };
  hmul(V, W);
  std::vector<double> G((size_t)kMaxBasis * kMaxBasis, 0.0), col(kMaxBasis), s_h, ev, evec;
  if ((rc = dots(1, V, W, col.data()))) return rc;
  G[0] = col[0];
  int m = 1, it = 0;
  double theta = G[0], rnorm = INFINITY;
  bool converged = false;
  for (;;) {
    // lowest Ritz pair of the subspace matrix
    std::vector<double> a((size_t)m * m);
    for (int i = 0; i < m; i++)
      for (int j = 0; j < m; j++) a[(size_t)i * m + j] = 0.5 * (G[(size_t)i * kMaxBasis + j] + G[(size_t)j * kMaxBasis + i]);
    jacobi_eigen(m, a, ev, evec);
    int lo = 0;
    for (int i = 1; i < m; i++)
      if (ev[i] < ev[lo]) lo = i;
    theta = ev[lo];
    s_h.resize(m);
    for (int i = 0; i < m; i++) s_h[i] = evec[(size_t)i * m + lo];
    DV_TRY(cudaMemcpyAsync(d_small, s_h.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
    combine_kernel<<<nb, 256, 0, st>>>(n, m, V, d_small, x, 0.0);
    combine_kernel<<<nb, 256, 0, st>>>(n, m, W, d_small, w, 0.0);
    correction_kernel<<<nb, 256, 0, st>>>(n, x, w, H.diag, theta, r, t);
    DV_TRY(cudaGetLastError());
    double rr;
    if ((rc = dots(1, r, r, &rr))) return rc;
    rnorm = std::sqrt(rr);
    if (rnorm <= tol) {
      converged = true;
      break;
    }
    if (++it > max_iter) break;
    if (m == mmax) {  // restart from the Ritz vector
      DV_TRY(cudaMemcpyAsync(V, x, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      DV_TRY(cudaMemcpyAsync(W, w, sizeof(double) * n, cudaMemcpyDeviceToDevice, st));
      G[0] = theta;
      m = 1;
    }
    // orthogonalise t against the basis twice, normalise, extend
    for (int pass = 0; pass < 2; pass++) {
      if ((rc = dots(m, V, t, col.data()))) return rc;
      for (int i = 0; i < m; i++) col[i] = -col[i];
      DV_TRY(cudaMemcpyAsync(d_small, col.data(), sizeof(double) * m, cudaMemcpyHostToDevice, st));
      combine_kernel<<<nb, 256, 0, st>>>(n, m, V, d_small, t, 1.0);
    }
    double tt;
    if ((rc = dots(1, t, t, &tt))) return rc;
    if (!(tt > 1e-28)) break;  // no new direction
    scale_kernel<<<nb, 256, 0, st>>>(n, 1.0 / std::sqrt(tt), t, V + (size_t)m * n);
    hmul(V + (size_t)m * n, W + (size_t)m * n);
    if ((rc = dots(m + 1, V, W + (size_t)m * n, col.data()))) return rc;
    for (int i = 0; i <= m; i++) {
      G[(size_t)i * kMaxBasis + m] = col[i];
      G[(size_t)m * kMaxBasis + i] = col[i];
    }
    m++;
  }
  // output: x normalised, with coefs[0] >= 0
  DV_TRY(cudaMemcpyAsync(hv.data(), x, sizeof(double) * n, cudaMemcpyDeviceToHost, st));
  cudaEventRecord(ev2, st);
  DV_TRY(cudaStreamSynchronize(st));
  double xx = 0.0;
  for (double v : hv) xx += v * v;
  const double sc = (hv[0] < 0 ? -1.0 : 1.0) / std::sqrt(xx);
  for (double& v : hv) v *= sc;
  // E0 as the Rayleigh quotient of the returned vector
  DV_TRY(cudaMemcpyAsync(x, hv.data(), sizeof(double) * n, cudaMemcpyHostToDevice, st));
  hmul(x, w);
  double xhx;
  if ((rc = dots(1, x, w, &xhx))) return rc;
  DV_TRY(cudaMemcpyAsync(coefs, x, sizeof(double) * n, cudaMemcpyDefault, st));
  DV_TRY(cudaStreamSynchronize(st));
  *e0 = xhx;
  if (info) {
    float a = 0.f, b = 0.f;
    cudaEventElapsedTime(&a, ev0, ev1);
    cudaEventElapsedTime(&b, ev1, ev2);
    info->iterations = it;
    info->residual = rnorm;
    info->nnz = H.nnz;
    info->converged = converged ? 1 : 0;
    info->build_ms = a;
    info->solve_ms = b;
  }
  return converged ? QP_OK : report(QP_ENOTCONV, "Davidson did not reach the residual tolerance");
}
