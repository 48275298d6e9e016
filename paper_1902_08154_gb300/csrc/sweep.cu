// sweep.cu -- persistent sm_103a kernel of the deterministic EN-PT2 +
// selection sweep (Quantum Package 2.0, arXiv:1902.08154, Appendix "CIPSI
// selection and PT2 energy").
//
// One CTA owns one generator I at a time; CTAs take generators from a device
// work queue in rank order (decreasing c_I^2).  For its generator the CTA
//  1. builds the Fock diagonal of I, so that <alpha|H|alpha> costs a few
//     flops per alpha (Appendix, "pre-compute the diagonal of the Fock
//     matrix");
//  2. applies the coarse filter: the internal J within excitation degree 4
//     of I, stored as compact records (holes of I missing from J as a mask
//     over I's occupied list, particles of J outside I, coefficient, and
//     whether J ranks before I);
//  3. walks the batches.  A batch is a hole set H of I (|H| = 1 or 2); its
//     cells are the particle sets R outside I with the spins of H, so the
//     batch holds the alpha = I - H + R.  With K = I - H, t = |K - J| and
//     X = J - K, deg(J, alpha) = t + |H| - |R n X|, so J reaches the batch only
//     if t <= 2 (the fine filter) and reaches cell R iff |R n X| >= t+|H|-2.
//       loop 1: J ranked before I ban the cells they reach (a J that reaches
//               every cell kills the batch); a later J equal to some alpha
//               bans that cell (alpha is internal);
//       loop 2: J ranked at or after I add c_J <J|H|alpha> into A(R) for the
//               cells they reach that are not banned;
//       cells:  every cell left is a perturber of I: e = A^2/(E0 - H_aa),
//               added to eps_I and offered to the CTA's selection buffer.
// Matrix elements use the Slater-Condon rules (Eqs. Hij) with phases from a
// masked popcount of J's spin string.
#include <cfloat>
#include <cstdio>

#include "common.cuh"

namespace qp {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr unsigned kFull = 0xffffffffu;

// ---------------------------------------------------------------------------
// Per-CTA static shared state
// ---------------------------------------------------------------------------
template <int NINT>
struct GenShared {
  uint64_t I[2 * NINT];
  int occ[kMaxElec];         // spin-orbital codes s*norb+q of I, ordered
  int vir[2][kMaxOrb];       // virtual orbitals of I per spin
  int vidx[2][kMaxOrb];      // orbital -> virtual index (-1: occupied)
  int nv[2];
  double F[2][kMaxOrb];      // Fock diagonal of I per spin
  double hii;
  int g, gi, nrec;
  int wsum[kWarps];
  // selection
  int tkcnt;
  unsigned long long tau;
  int hist[256];
  uint64_t pw[1 + 2 * NINT];
  uint64_t thr[1 + 2 * NINT];
  int need, group, digit, found_w, found_sh;
  // reductions
  double red_d[kWarps][2];
  long long red_l[kWarps][3];
  unsigned long long red_u[kWarps][3];
};

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ long long warp_sum_ll(long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_sum_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_xor_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) v ^= __shfl_xor_sync(kFull, v, o);
  return v;
}
__device__ __forceinline__ unsigned long long warp_min_u(unsigned long long v) {
#pragma unroll
  for (int o = 16; o; o >>= 1) {
    unsigned long long w = __shfl_xor_sync(kFull, v, o);
    v = w < v ? w : v;
  }
  return v;
}

// Block-wide exclusive scan of a 0/1 flag; returns this thread's position and
// writes the block total to *total (all threads).
template <int NINT>
__device__ __forceinline__ int block_scan_flag(bool f, GenShared<NINT>& S, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned b = __ballot_sync(kFull, f);
  int before = __popc(b & ((1u << lane) - 1));
  if (lane == 0) S.wsum[warp] = __popc(b);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; w++) {
    int c = S.wsum[w];
    off += (w < warp) ? c : 0;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return off + before;
}

// ---------------------------------------------------------------------------
// Batch geometry
// ---------------------------------------------------------------------------
struct Batch {
  int h;            // number of holes (1, 2)
  int kind;         // 0 single, 1 same-spin double, 2 opposite-spin double
  int ia, ib;       // occupied indices of the holes in I
  int ca, cb;       // their spin-orbital codes
  int sa, sb;       // their spins
  int qa, qb;       // their orbitals
  uint64_t hm;      // hole mask over I's occupied list
  int ncell;
};

// cell <-> particle orbitals (r in spin sa, s in spin sb)
template <int NINT>
__device__ __forceinline__ void cell_orbitals(const Batch& B, const GenShared<NINT>& S, int c,
                                              int* r, int* s) {
  if (B.kind == 0) {
    *r = S.vir[B.sa][c];
    *s = -1;
  } else if (B.kind == 2) {
    int nv1 = S.nv[1];
    *r = S.vir[0][c / nv1];
    *s = S.vir[1][c % nv1];
  } else {
    int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)c)) * 0.5f);
    while (y * (y - 1) / 2 > c) y--;
    while ((y + 1) * y / 2 <= c) y++;
    int x = c - y * (y - 1) / 2;
    *r = S.vir[B.sa][x];
    *s = S.vir[B.sa][y];
  }
}

__device__ __forceinline__ int pair_cell(int x, int y) {  // x != y virtual indices
  int lo = x < y ? x : y, hi = x < y ? y : x;
  return hi * (hi - 1) / 2 + lo;
}

// Particles of J outside I, filtered to a spin, as orbitals.
__device__ __forceinline__ int particles_of_spin(uint64_t part, int norb, int spin, int* out) {
  int n = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    int c = (int)((part >> (16 * i)) & 0xFFFF);
    if (c == 0xFFFF) continue;
    int s = c >= norb;
    if (s == spin) out[n++] = c - s * norb;
  }
  return n;
}

// Visit (with the 32 lanes of a warp, each cell once) the cells of batch B
// reached by a record with t = tt.  For tt <= 2 the rules are those of the
// file header.  `all` cases visit every cell.
template <int NINT, typename Fn>
__device__ __forceinline__ void for_reached_cells(const Batch& B, const GenShared<NINT>& S, int norb,
                                                  uint64_t part, int tt, int lane, Fn&& fn) {
  const bool all = (B.h == 1) ? (tt <= 1) : (tt == 0);
  if (all) {
    for (int c = lane; c < B.ncell; c += 32) fn(c);
    return;
  }
  if (B.kind == 0) {  // tt == 2: r in the particles of J
    int P[4];
    int np = particles_of_spin(part, norb, B.sa, P);
    if (lane < np) fn(S.vidx[B.sa][P[lane]]);
    return;
  }
  if (B.kind == 1) {
    int P[4];
    int np = particles_of_spin(part, norb, B.sa, P);
    int nv = S.nv[B.sa];
    if (tt == 1) {  // pairs touching P
      for (int i = 0; i < np; i++) {
        int x = S.vidx[B.sa][P[i]];
        for (int y = lane; y < nv; y += 32) {
          if (y == x) continue;
          bool dup = false;  // pair {P[j], P[i]} with j < i was visited from P[j]
          for (int j = 0; j < i; j++) dup |= (S.vidx[B.sa][P[j]] == y);
          if (!dup) fn(pair_cell(x, y));
        }
      }
    } else {  // tt == 2: pairs inside P
      int m = 0;
      for (int i = 0; i < np; i++)
        for (int j = i + 1; j < np; j++) {
          if (m == lane) fn(pair_cell(S.vidx[B.sa][P[i]], S.vidx[B.sa][P[j]]));
          m++;
        }
    }
    return;
  }
  // kind 2: cells (r up, s down)
  int Pa[4], Pb[4];
  int na = particles_of_spin(part, norb, 0, Pa);
  int nb = particles_of_spin(part, norb, 1, Pb);
  const int nv0 = S.nv[0], nv1 = S.nv[1];
  if (tt == 1) {
    for (int i = 0; i < na; i++) {
      int x = S.vidx[0][Pa[i]];
      for (int y = lane; y < nv1; y += 32) fn(x * nv1 + y);
    }
    for (int j = 0; j < nb; j++) {
      int y = S.vidx[1][Pb[j]];
      for (int x = lane; x < nv0; x += 32) {
        bool dup = false;  // rows of Pa were visited above
        for (int i = 0; i < na; i++) dup |= (S.vidx[0][Pa[i]] == x);
        if (!dup) fn(x * nv1 + y);
      }
    }
  } else {
    int m = 0;
    for (int i = 0; i < na; i++)
      for (int j = 0; j < nb; j++) {
        if (m == lane) fn(S.vidx[0][Pa[i]] * nv1 + S.vidx[1][Pb[j]]);
        m++;
      }
  }
}

// <J|H|alpha> with alpha = K + R, K = I - H.  X = J - K, T = K - J.
// holes(J -> alpha) = X - R, particles = T + (R - X).
template <int NINT>
__device__ __forceinline__ double element(const SweepParams& p, const uint64_t* Jw, const int* X, int nx,
                                          const int* T, int nt, int r, int s) {
  const int norb = p.norb;
  int ho[2], pa[2], nh = 0, npp = 0;
  for (int i = 0; i < nx; i++) {
    int x = X[i];
    if (x != r && x != s && nh < 2) ho[nh++] = x;
  }
  for (int i = 0; i < nt && npp < 2; i++) pa[npp++] = T[i];
  bool r_in = false, s_in = false;
  for (int i = 0; i < nx; i++) {
    r_in |= (X[i] == r);
    s_in |= (X[i] == s);
  }
  if (!r_in && npp < 2) pa[npp++] = r;
  if (s >= 0 && !s_in && npp < 2) pa[npp++] = s;
  if (nh == 0 || nh != npp) return 0.0;  // not reached: such cells are banned
  if (nh == 1) {
    const int sp = ho[0] >= norb, a = ho[0] - sp * norb, b = pa[0] - sp * norb;
    const uint64_t* sw = Jw + sp * NINT;
    int lo = a < b ? a : b, hi = a < b ? b : a;
    double sign = (count_between<NINT>(sw, lo, hi) & 1) ? -1.0 : 1.0;
    double v = p.h[a * norb + b];
#pragma unroll
    for (int t = 0; t < 2; t++) {
#pragma unroll
      for (int w = 0; w < NINT; w++) {
        uint64_t bits = Jw[t * NINT + w];
        while (bits) {
          int q = 64 * w + __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          v += p.eri[eri_index(a, b, q, q)];
          if (t == sp) v -= p.eri[eri_index(a, q, q, b)];
        }
      }
    }
    return sign * v;
  }
  // double: order holes and particles by spin-orbital code, pair 1-1, 2-2
  if (ho[0] > ho[1]) { int t = ho[0]; ho[0] = ho[1]; ho[1] = t; }
  if (pa[0] > pa[1]) { int t = pa[0]; pa[0] = pa[1]; pa[1] = t; }
  const int s1 = ho[0] >= norb, s2 = ho[1] >= norb;
  const int h1 = ho[0] - s1 * norb, p1 = pa[0] - s1 * norb;
  const int h2 = ho[1] - s2 * norb, p2 = pa[1] - s2 * norb;
  uint64_t w1[NINT];
#pragma unroll
  for (int w = 0; w < NINT; w++) w1[w] = Jw[s1 * NINT + w];
  int n1 = count_between<NINT>(w1, h1 < p1 ? h1 : p1, h1 < p1 ? p1 : h1);
  // apply h1 -> p1, then count for h2 -> p2 on the result
  w1[h1 >> 6] &= ~(1ull << (h1 & 63));
  w1[p1 >> 6] |= (1ull << (p1 & 63));
  int n2;
  if (s2 == s1) {
    n2 = count_between<NINT>(w1, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  } else {
    n2 = count_between<NINT>(Jw + s2 * NINT, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  }
  double v = p.eri[eri_index(h1, p1, h2, p2)];
  if (s1 == s2) v -= p.eri[eri_index(h1, p2, h2, p1)];
  return ((n1 + n2) & 1) ? -v : v;
}

// ---------------------------------------------------------------------------
// Selection buffer compaction: keep the k best entries (|e| descending, key
// ascending) of the CTA's buffer.  MSD radix select over the composite
// (~bits(|e|), key words), 8-bit digits, then an ordered in-place compaction.
// ---------------------------------------------------------------------------
template <int NINT>
__device__ __forceinline__ uint64_t composite_word(const double* te, const uint64_t* tk, int i, int w) {
  if (w == 0) return ~(unsigned long long)__double_as_longlong(fabs(te[i]));
  return tk[(size_t)i * (2 * NINT) + (w - 1)];
}

template <int NINT>
__device__ bool prefix_match(const double* te, const uint64_t* tk, int i, const uint64_t* pw, int w, int keep_sh) {
  for (int v = 0; v < w; v++)
    if (composite_word<NINT>(te, tk, i, v) != pw[v]) return false;
  if (keep_sh >= 64) return true;
  return (composite_word<NINT>(te, tk, i, w) >> keep_sh) == (pw[w] >> keep_sh);
}

template <int NINT>
__device__ void compact_selection(const SweepParams& p, GenShared<NINT>& S, double* te, double* ta, uint64_t* tk) {
  constexpr int NW = 1 + 2 * NINT;
  const int tid = threadIdx.x;
  __syncthreads();
  const int n = S.tkcnt;
  const long long k = p.k;
  if (n <= k) return;
  if (tid == 0) {
    S.need = (int)k;
    for (int w = 0; w < NW; w++) S.pw[w] = 0;
    S.group = n;
    S.found_w = NW - 1;
    S.found_sh = 0;
  }
  __syncthreads();
  bool done = false;
  for (int w = 0; w < NW && !done; w++) {
    for (int sh = 56; sh >= 0; sh -= 8) {
      for (int b = tid; b < 256; b += kThreads) S.hist[b] = 0;
      __syncthreads();
      for (int i = tid; i < n; i += kThreads)
        if (prefix_match<NINT>(te, tk, i, S.pw, w, sh + 8))
          atomicAdd(&S.hist[(composite_word<NINT>(te, tk, i, w) >> sh) & 255], 1);
      __syncthreads();
      if (tid == 0) {
        int c = 0, d = 255;
        for (int b = 0; b < 256; b++) {
          if (c + S.hist[b] >= S.need) { d = b; break; }
          c += S.hist[b];
        }
        S.need -= c;
        S.group = S.hist[d];
        S.pw[w] |= (uint64_t)d << sh;
        S.found_w = w;
        S.found_sh = sh;
      }
      __syncthreads();
      if (S.group <= 1) { done = true; break; }
    }
  }
  // the threshold composite: the unique entry matching the prefix
  if (S.group == 1) {
    for (int i = tid; i < n; i += kThreads)
      if (prefix_match<NINT>(te, tk, i, S.pw, S.found_w, S.found_sh))
        for (int w = 0; w < NW; w++) S.thr[w] = composite_word<NINT>(te, tk, i, w);
  } else if (tid == 0) {
    for (int w = 0; w < NW; w++) S.thr[w] = S.pw[w];
  }
  __syncthreads();
  // ordered in-place compaction of entries <= threshold
  int out = 0;
  for (int base = 0; base < n; base += kThreads) {
    int i = base + tid;
    bool keep = false;
    double e = 0, a = 0;
    uint64_t key[2 * NINT];
    if (i < n) {
      int cmp = 0;
      for (int w = 0; w < NW && cmp == 0; w++) {
        uint64_t x = composite_word<NINT>(te, tk, i, w);
        cmp = x < S.thr[w] ? -1 : (x > S.thr[w] ? 1 : 0);
      }
      keep = cmp <= 0;
      e = te[i];
      a = ta[i];
#pragma unroll
      for (int w = 0; w < 2 * NINT; w++) key[w] = tk[(size_t)i * (2 * NINT) + w];
    }
    int total;
    int pos = block_scan_flag<NINT>(keep, S, &total);
    if (keep) {
      int o = out + pos;
      te[o] = e;
      ta[o] = a;
#pragma unroll
      for (int w = 0; w < 2 * NINT; w++) tk[(size_t)o * (2 * NINT) + w] = key[w];
    }
    out += total;
    __syncthreads();
  }
  if (tid == 0) {
    S.tkcnt = out;
    unsigned long long t = ~S.thr[0];
    if (t > S.tau) S.tau = t;
    atomicMax(p.tau_bits, t);
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The sweep kernel
// ---------------------------------------------------------------------------
template <int NINT>
__global__ void __launch_bounds__(kThreads) sweep_kernel(SweepParams p) {
  constexpr int NW = 2 * NINT;
  extern __shared__ __align__(16) unsigned char dyn[];
  double* A = reinterpret_cast<double*>(dyn);
  uint32_t* ban = reinterpret_cast<uint32_t*>(A + p.max_cells);
  __shared__ GenShared<NINT> S;

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int norb = p.norb, nel = p.nel;
  const size_t rbase = (size_t)blockIdx.x * (size_t)p.ndet;
  uint64_t* fw = p.f_words + rbase * NW;
  double* fc = p.f_coef + rbase;
  uint64_t* fhm = p.f_hmask + rbase;
  uint64_t* fpt = p.f_part + rbase;
  uint32_t* ffl = p.f_flag + rbase;
  double* te = p.tk_e + (size_t)blockIdx.x * (size_t)p.cap;
  double* ta = p.tk_a + (size_t)blockIdx.x * (size_t)p.cap;
  uint64_t* tk = p.tk_key + (size_t)blockIdx.x * (size_t)p.cap * NW;

  if (tid == 0) {
    S.tkcnt = 0;
    S.tau = 0;
  }

  for (;;) {
    __syncthreads();
    if (tid == 0) {
      const long long t = atomicAdd(p.queue, 1);
      const long long gg = p.shard_index + t * (long long)p.shard_count;
      S.g = gg < p.ndet ? (int)gg : (int)p.ndet;
      S.gi = (S.g < p.ndet) ? p.order[S.g] : 0;
    }
    __syncthreads();
    const int g = S.g;
    if (g >= p.ndet) break;
    if (tid < NW) S.I[tid] = p.dets[(size_t)S.gi * NW + tid];
    __syncthreads();
    if (tid == 0) {
      int n = 0;
      for (int s = 0; s < 2; s++) {
        int nv = 0;
        for (int q = 0; q < norb; q++) {
          if ((S.I[s * NINT + (q >> 6)] >> (q & 63)) & 1ull) {
            S.occ[n++] = s * norb + q;
            S.vidx[s][q] = -1;
          } else {
            S.vidx[s][q] = nv;
            S.vir[s][nv++] = q;
          }
        }
        S.nv[s] = nv;
      }
    }
    __syncthreads();
    // Fock diagonal F_s(q) = h_qq + sum_{j in I} [(qq|jj) - delta_s (qj|jq)]
    for (int x = tid; x < 2 * norb; x += kThreads) {
      const int s = x / norb, q = x - s * norb;
      double f = p.h[q * norb + q];
      for (int i = 0; i < nel; i++) {
        const int c = S.occ[i], sj = c >= norb, j = c - sj * norb;
        f += p.Jm[q * norb + j];
        if (sj == s) f -= p.Km[q * norb + j];
      }
      S.F[s][q] = f;
    }
    __syncthreads();
    if (tid == 0) {  // H_II = 1/2 sum_i (h_ii + F(i))
      double e = 0.0;
      for (int i = 0; i < nel; i++) {
        const int c = S.occ[i], s = c >= norb, q = c - s * norb;
        e += p.h[q * norb + q] + S.F[s][q];
      }
      S.hii = 0.5 * e;
    }

    // ---- coarse filter: J within degree 4 of I (I itself included) ----
    uint64_t Iw[NW];
#pragma unroll
    for (int w = 0; w < NW; w++) Iw[w] = S.I[w];
    int nrec = 0;
    for (long long base = 0; base < p.ndet; base += kThreads) {
      const long long j = base + tid;
      bool keep = false;
      uint64_t Jw[NW];
      if (j < p.ndet) {
        int d = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) {
          Jw[w] = p.dets[(size_t)j * NW + w];
          d += __popcll(Jw[w] ^ Iw[w]);
        }
        keep = d <= 8;
      }
      int total;
      int pos = block_scan_flag<NINT>(keep, S, &total);
      if (keep) {
        const int r = nrec + pos;
        uint64_t hmask = 0;
        uint64_t part = ~0ull;
        int npart = 0;
#pragma unroll
        for (int s = 0; s < 2; s++) {
          int below = (s == 0) ? 0 : p.nalpha;  // occupied index offset of spin s
#pragma unroll
          for (int w = 0; w < NINT; w++) {
            const uint64_t iw = Iw[s * NINT + w], jw = Jw[s * NINT + w];
            uint64_t miss = iw & ~jw;
            while (miss) {
              const int b = __ffsll((long long)miss) - 1;
              miss &= miss - 1;
              const int idx = below + __popcll(iw & ((1ull << b) - 1));
              hmask |= 1ull << idx;
            }
            uint64_t extra = jw & ~iw;
            while (extra) {
              const int b = __ffsll((long long)extra) - 1;
              extra &= extra - 1;
              const uint64_t code = (uint64_t)(s * norb + 64 * w + b);
              if (npart < 4) part = (part & ~(0xFFFFull << (16 * npart))) | (code << (16 * npart));
              npart++;
            }
            below += __popcll(iw);
          }
        }
#pragma unroll
        for (int w = 0; w < NW; w++) fw[(size_t)r * NW + w] = Jw[w];
        fc[r] = p.coefs[j];
        fhm[r] = hmask;
        fpt[r] = part;
        ffl[r] = (p.rank_of[j] < g) ? 1u : 0u;
      }
      nrec += total;
      __syncthreads();
    }
    __syncthreads();

    // ---- batches ----
    double acc_e = 0.0, acc_s2 = 0.0;
    long long acc_na = 0, acc_nc = 0;
    unsigned long long acc_d0 = 0, acc_d1 = 0, acc_min = 0x7FF0000000000000ull, acc_tiny = 0;
    const int nb1 = nel, nbat = nel + nel * (nel - 1) / 2;
    for (int b = 0; b < nbat; b++) {
      Batch B;
      if (b < nb1) {
        B.h = 1;
        B.ia = b;
        B.ib = -1;
      } else {
        const int t = b - nb1;
        int y = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)t)) * 0.5f);
        while (y * (y - 1) / 2 > t) y--;
        while ((y + 1) * y / 2 <= t) y++;
        B.h = 2;
        B.ib = y;
        B.ia = t - y * (y - 1) / 2;
      }
      B.ca = S.occ[B.ia];
      B.sa = B.ca >= norb;
      B.qa = B.ca - B.sa * norb;
      B.hm = 1ull << B.ia;
      if (B.h == 2) {
        B.cb = S.occ[B.ib];
        B.sb = B.cb >= norb;
        B.qb = B.cb - B.sb * norb;
        B.hm |= 1ull << B.ib;
        B.kind = (B.sa == B.sb) ? 1 : 2;
        const int nv = S.nv[B.sa];
        B.ncell = (B.kind == 1) ? nv * (nv - 1) / 2 : S.nv[0] * S.nv[1];
      } else {
        B.cb = -1;
        B.sb = -1;
        B.qb = -1;
        B.kind = 0;
        B.ncell = S.nv[B.sa];
      }
      if (B.ncell == 0) continue;
      for (int c = tid; c < B.ncell; c += kThreads) A[c] = 0.0;
      for (int c = tid; c < (B.ncell + 31) / 32; c += kThreads) ban[c] = 0u;
      __syncthreads();

      // loop 1: bans (and detection of a batch banned as a whole)
      bool dead = false;
      for (int r0 = warp * 32; r0 < nrec; r0 += kWarps * 32) {
        const int r = r0 + lane;
        bool act = false;
        int tt = 3;
        if (r < nrec) {
          const uint64_t hm = fhm[r];
          tt = __popcll(hm & ~B.hm);
          if (tt <= 2) {
            if (ffl[r] & 1u) {
              if ((B.h == 1 && tt <= 1) || (B.h == 2 && tt == 0)) dead = true;
              else act = true;
            } else if (tt == 0 && hm == B.hm) {
              act = true;  // J = I - H + X: the cell X is internal
            }
          }
        }
        unsigned m = __ballot_sync(kFull, act);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int rr = __shfl_sync(kFull, r, src);
          const int t2 = __shfl_sync(kFull, tt, src);
          const uint64_t part = fpt[rr];
          if (ffl[rr] & 1u) {
            for_reached_cells<NINT>(B, S, norb, part, t2, lane, [&](int c) {
              atomicOr(&ban[c >> 5], 1u << (c & 31));
            });
          } else if (lane == 0) {
            int P0[4], P1[4];
            int c;
            if (B.kind == 0) {
              particles_of_spin(part, norb, B.sa, P0);
              c = S.vidx[B.sa][P0[0]];
            } else if (B.kind == 1) {
              particles_of_spin(part, norb, B.sa, P0);
              c = pair_cell(S.vidx[B.sa][P0[0]], S.vidx[B.sa][P0[1]]);
            } else {
              particles_of_spin(part, norb, 0, P0);
              particles_of_spin(part, norb, 1, P1);
              c = S.vidx[0][P0[0]] * S.nv[1] + S.vidx[1][P1[0]];
            }
            atomicOr(&ban[c >> 5], 1u << (c & 31));
          }
        }
      }
      if (__syncthreads_or(dead)) continue;

      // loop 2: A(R) += c_J <J|H|I - H + R> over J ranked at or after I
      long long con = 0;
      for (int r0 = warp * 32; r0 < nrec; r0 += kWarps * 32) {
        const int r = r0 + lane;
        bool act = false;
        int tt = 3;
        if (r < nrec) {
          tt = __popcll(fhm[r] & ~B.hm);
          act = (tt <= 2) && !(ffl[r] & 1u);
        }
        unsigned m = __ballot_sync(kFull, act);
        while (m) {
          const int src = __ffs(m) - 1;
          m &= m - 1;
          const int rr = __shfl_sync(kFull, r, src);
          const int t2 = __shfl_sync(kFull, tt, src);
          const uint64_t part = fpt[rr];
          const uint64_t hm = fhm[rr];
          const double cj = fc[rr];
          uint64_t Jw[NW];
#pragma unroll
          for (int w = 0; w < NW; w++) Jw[w] = fw[(size_t)rr * NW + w];
          // X = (particles of J) + (holes of H that J keeps); T = holes of J not in H
          int X[4], T[2], nx = 0, nt = 0;
          for (int i = 0; i < 4; i++) {
            const int c = (int)((part >> (16 * i)) & 0xFFFF);
            if (c != 0xFFFF && nx < 4) X[nx++] = c;
          }
          if (!((hm >> B.ia) & 1ull) && nx < 4) X[nx++] = B.ca;
          if (B.h == 2 && !((hm >> B.ib) & 1ull) && nx < 4) X[nx++] = B.cb;
          uint64_t tm = hm & ~B.hm;
          while (tm && nt < 2) {
            const int i = __ffsll((long long)tm) - 1;
            tm &= tm - 1;
            T[nt++] = S.occ[i];
          }
          for_reached_cells<NINT>(B, S, norb, part, t2, lane, [&](int c) {
            if ((ban[c >> 5] >> (c & 31)) & 1u) return;
            int ro, so;
            cell_orbitals<NINT>(B, S, c, &ro, &so);
            const int rc = B.sa * norb + ro;
            const int sc = (B.h == 2) ? B.sb * norb + so : -1;
            const double v = element<NINT>(p, Jw, X, nx, T, nt, rc, sc);
            atomicAdd(&A[c], cj * v);
            con++;
          });
        }
      }
      __syncthreads();

      // cells: perturbers of I in this batch
      if (p.k > 0) {
        if (S.tkcnt + B.ncell > p.cap) compact_selection<NINT>(p, S, te, ta, tk);
        if (tid == 0) {
          const unsigned long long gt = *((volatile unsigned long long*)p.tau_bits);
          if (gt > S.tau) S.tau = gt;
        }
        __syncthreads();
      }
      const unsigned long long tau = S.tau;
      for (int c = tid; c < B.ncell; c += kThreads) {
        if ((ban[c >> 5] >> (c & 31)) & 1u) continue;
        int ro, so;
        cell_orbitals<NINT>(B, S, c, &ro, &so);
        const double a = A[c];
        double haa;
        if (B.h == 1) {
          const int s = B.sa;
          haa = S.hii - S.F[s][B.qa] + S.F[s][ro] - (p.Jm[B.qa * norb + ro] - p.Km[B.qa * norb + ro]);
        } else {
          const int s1 = B.sa, s2 = B.sb;  // r has spin s1, s has spin s2
          auto W = [&](int x, int sx, int y, int sy) {
            double v = p.Jm[x * norb + y];
            if (sx == sy) v -= p.Km[x * norb + y];
            return v;
          };
          haa = S.hii - S.F[s1][B.qa] - S.F[s2][B.qb] + W(B.qa, s1, B.qb, s2) + S.F[s1][ro] +
                S.F[s2][so] - W(ro, s1, B.qa, s1) - W(ro, s1, B.qb, s2) - W(so, s2, B.qa, s1) -
                W(so, s2, B.qb, s2) + W(ro, s1, so, s2);
        }
        const double D = p.e0 - haa;
        const double e = a * a / D;
        const double q = a / D;
        acc_e += e;
        acc_s2 += q * q;
        acc_na++;
        if (fabs(a) < 1e-14) acc_tiny++;
        const unsigned long long db = (unsigned long long)__double_as_longlong(fabs(D));
        acc_min = db < acc_min ? db : acc_min;
        // alpha's key
        uint64_t key[NW];
#pragma unroll
        for (int w = 0; w < NW; w++) key[w] = S.I[w];
        key[B.sa * NINT + (B.qa >> 6)] &= ~(1ull << (B.qa & 63));
        key[B.sa * NINT + (ro >> 6)] |= 1ull << (ro & 63);
        if (B.h == 2) {
          key[B.sb * NINT + (B.qb >> 6)] &= ~(1ull << (B.qb & 63));
          key[B.sb * NINT + (so >> 6)] |= 1ull << (so & 63);
        }
        uint64_t hk = 0;
#pragma unroll
        for (int w = 0; w < NW; w++) hk = splitmix64(hk ^ key[w]);
        acc_d0 += hk;
        acc_d1 ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
        if (p.k > 0) {
          const unsigned long long eb = (unsigned long long)__double_as_longlong(fabs(e));
          if (eb >= tau) {
            const int pos = atomicAdd(&S.tkcnt, 1);
            te[pos] = e;
            ta[pos] = a;
#pragma unroll
            for (int w = 0; w < NW; w++) tk[(size_t)pos * NW + w] = key[w];
          }
        }
      }
      acc_nc += con;
      __syncthreads();
    }

    // ---- per-generator reduction ----
    {
      double e = warp_sum(acc_e), s2 = warp_sum(acc_s2);
      long long na = warp_sum_ll(acc_na), nc = warp_sum_ll(acc_nc);
      unsigned long long d0 = warp_sum_u(acc_d0), d1 = warp_xor_u(acc_d1), mn = warp_min_u(acc_min);
      unsigned long long tiny = warp_sum_u(acc_tiny);
      if (lane == 0) {
        S.red_d[warp][0] = e;
        S.red_d[warp][1] = s2;
        S.red_l[warp][0] = na;
        S.red_l[warp][1] = nc;
        S.red_u[warp][0] = d0;
        S.red_u[warp][1] = d1;
        S.red_u[warp][2] = mn;
        S.red_l[warp][2] = (long long)tiny;
      }
      __syncthreads();
      if (tid == 0) {
        double te_ = 0, ts = 0;
        long long tn = 0, tc = 0, tt = 0;
        unsigned long long x0 = 0, x1 = 0, m = 0x7FF0000000000000ull;
        for (int w = 0; w < kWarps; w++) {
          te_ += S.red_d[w][0];
          ts += S.red_d[w][1];
          tn += S.red_l[w][0];
          tc += S.red_l[w][1];
          tt += S.red_l[w][2];
          x0 += S.red_u[w][0];
          x1 ^= S.red_u[w][1];
          m = S.red_u[w][2] < m ? S.red_u[w][2] : m;
        }
        p.eps[g] = te_;
        p.s2[g] = ts;
        p.na[g] = tn;
        p.ncon[g] = tc;
        if (tn) {
          atomicAdd(&p.digest[0], x0);
          atomicXor(&p.digest[1], x1);
          atomicMin(p.min_den_bits, m);
          atomicAdd(p.n_tiny, (unsigned long long)tt);
        }
      }
    }
  }
  // final compaction of the selection buffer
  if (p.k > 0) compact_selection<NINT>(p, S, te, ta, tk);
  if (tid == 0) p.tk_cnt[blockIdx.x] = S.tkcnt;
}

template __global__ void sweep_kernel<1>(SweepParams);
template __global__ void sweep_kernel<2>(SweepParams);

// host-side launch helpers --------------------------------------------------
cudaError_t launch_sweep(int nint, const SweepParams& p, int grid, size_t smem, cudaStream_t st) {
  if (nint == 1) {
    cudaFuncSetAttribute(sweep_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sweep_kernel<1><<<grid, kThreads, smem, st>>>(p);
  } else {
    cudaFuncSetAttribute(sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    sweep_kernel<2><<<grid, kThreads, smem, st>>>(p);
  }
  return cudaGetLastError();
}

int sweep_blocks_per_sm(int nint, size_t smem) {
  int n = 0;
  if (nint == 1) {
    cudaFuncSetAttribute(sweep_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<1>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(sweep_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sweep_kernel<2>, kThreads, smem);
  }
  return n;
}

int sweep_threads() { return kThreads; }

}  // namespace qp
