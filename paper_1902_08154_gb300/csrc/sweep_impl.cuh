// sweep_impl.cuh -- sm_103a kernels of the deterministic EN-PT2 + selection sweep
// (Quantum Package 2.0, arXiv:1902.08154, Appendix "CIPSI selection and PT2
// energy").
//
// Generators are taken in rank order (decreasing c_I^2) in waves of slots.
// Per wave two kernels run:
//
//  prep_kernel (one CTA per generator I of the wave)
//    - the Fock diagonal of I, so that <alpha|H|alpha> costs a few flops per
//      alpha (Appendix: "pre-compute the diagonal of the Fock matrix");
//    - the coarse filter: every internal J within excitation degree 4 of I,
//      stored as a record (its words, c_J, the holes of I missing from J as a
//      mask over I's occupied list, the particles of J outside I, and whether
//      J ranks before I);
//    - the fine filter, done once per generator by bucketing: a batch is a
//      hole set H of I (|H| = 1 or 2) holding the alpha = I - H + R for the
//      particle sets R outside I with the spins of H.  With K = I - H,
//      t = |K - J| and X = J - K, deg(J, alpha) = t + |H| - |R n X|, so J
//      reaches batch H only if t <= 2.  With Q the holes of J (d = |Q|),
//      t = d - |Q n H|: J with d <= 2 reaches every batch, d = 3 the batches
//      meeting Q, d = 4 the batches inside Q.  Records with d <= 2 go to one
//      shared bucket, those with d = 3 to the list of each of their holes
//      (a batch reads the lists of its holes), those with d = 4 to the
//      bucket of each pair of their holes.
//
//  batch_kernel (persistent CTAs, one (generator, batch) item at a time,
//  items of the heaviest generators first)
//    loop 1: J ranked before I ban the cells they reach (J that reach every
//            cell kill the batch); a later J equal to some alpha bans it;
//    loop 2: J ranked at or after I add c_J <J|H|alpha> into the shared-memory
//            accumulator A(R) of the cells they reach that are not banned.
//            J reaching every cell are spread over the whole CTA, J reaching a
//            row of cells over a warp, J reaching a few cells over a thread;
//    cells:  every cell left is a perturber of I: e = A^2/(E0 - H_aa) with
//            H_aa from per-batch row sums of the Fock diagonal, added to eps_I
//            and offered to the CTA's selection buffer.
// Matrix elements follow the Slater-Condon rules (Eqs. Hij) with phases from
// a masked popcount of J's spin string.
//
// Numerator precision: the batch kernel is a template on NT, the type of the
// integrals it gathers and of the products c_J <J|H|alpha>.  NT = double is
// the plain FP64 sweep; NT = float gathers FP32 integrals and forms FP32
// products, while each product is still added into the FP64 accumulator
// A(R) and the denominators, e_alpha and every reduction stay FP64.
// sweep.cu instantiates the FP64 kernels, sweep_mixed.cu the mixed ones.
#pragma once
#include <cfloat>
#include <cstdio>

#include "common.cuh"

namespace qp {

constexpr int kThreads = 256;
constexpr int kWarps = kThreads / 32;
constexpr int kChunk = 1536;  // bucket entries classified per round
constexpr int kGroup = 8;     // J reaching every cell, handled together
constexpr unsigned kFull = 0xffffffffu;
// Bit of a bucket entry's particle word that flags a J ranked before I (see
// part_code below).
constexpr uint64_t kBeforeBit = 1ull << 15;

__device__ __forceinline__ double warp_sum(double v) {
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
// the block total.  wsum: kWarps ints of shared memory.
__device__ __forceinline__ int block_scan_flag(bool f, int* wsum, int* total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  unsigned b = __ballot_sync(kFull, f);
  int before = __popc(b & ((1u << lane) - 1));
  if (lane == 0) wsum[warp] = __popc(b);
  __syncthreads();
  int off = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < kWarps; w++) {
    int c = wsum[w];
    off += (w < warp) ? c : 0;
    tot += c;
  }
  __syncthreads();
  *total = tot;
  return off + before;
}

// Integrals in the numerator precision.
// E4: the four-index layout of the context (eri4_index); else the packed
// array (the no-allocation entry point, which has only the caller's copy).
template <typename NT, bool E4>
__device__ __forceinline__ const NT* numer_eri(const SweepParams& p) {
  if constexpr (sizeof(NT) == 8) return reinterpret_cast<const NT*>(E4 ? p.eri4 : p.eri);
  else return reinterpret_cast<const NT*>(E4 ? p.eri4_32 : p.eri32);
}

// Position of (pq|rs) in the gather layout.
template <bool E4>
__device__ __forceinline__ int gidx(int p, int q, int r, int s, int norb) {
  if constexpr (E4) return eri4_index(p, q, r, s, norb);
  else return eri_index(p, q, r, s);
}
template <typename NT>
__device__ __forceinline__ const NT* numer_h(const SweepParams& p);
template <>
__device__ __forceinline__ const double* numer_h<double>(const SweepParams& p) { return p.h; }
template <>
__device__ __forceinline__ const float* numer_h<float>(const SweepParams& p) { return p.h32; }

// 1/d by Newton-Raphson iteration for the reciprocal, r <- r + r (1 - d r),
// from the hardware's approximate FP64 reciprocal (PTX rcp.approx.ftz.f64,
// relative error below 2^-22).  Each step squares the relative error: two
// steps reach the rounding level of FP64 (a few ulp) with four FMAs on the
// FP64 pipe instead of a correctly rounded division; one step leaves a
// relative error near 2^-44, used by the mixed-precision sweep, whose
// budget is 1e-6 Eh.  |d| must be a normal number (the sweep's denominators
// are bounded away from 0 and infinity; others take the plain division).
template <int STEPS>
__device__ __forceinline__ double recip_nr(double d) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(d));
#pragma unroll
  for (int i = 0; i < STEPS; i++) {
    const double e = fma(-d, r, 1.0);
    r = fma(r, e, r);
  }
  return r;
}

// Nanoseconds of the device's global timer.
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

// Bit pattern of |x|.  The mask is applied in inline PTX: written in C++ the
// compiler recognises it as fabs and issues it on the FP64 pipe.
__device__ __forceinline__ unsigned long long abs_bits(double x) {
  unsigned long long b;
  asm("and.b64 %0, %1, 0x7FFFFFFFFFFFFFFF;" : "=l"(b) : "l"((unsigned long long)__double_as_longlong(x)));
  return b;
}

// v with its sign flipped when neg: a bit operation, no floating-point pipe.
__device__ __forceinline__ double flip_sign(double v, bool neg) {
  return __longlong_as_double(__double_as_longlong(v) ^ ((long long)neg << 63));
}
__device__ __forceinline__ float flip_sign(float v, bool neg) {
  return __int_as_float(__float_as_int(v) ^ ((int)neg << 31));
}

// ---------------------------------------------------------------------------
// Exact accumulation of the numerator A_alpha = sum_J c_J <J|H|alpha> in the
// one-state sweep.  Each product (FP64, or FP32 in the mixed form) is
// converted, with one rounding at 2^-F, to a 96-bit two's-complement integer
// in units of 2^-F and added with integer arithmetic, so that A_alpha does
// not depend on the order of the additions: the J of a batch reach a cell
// from different warps, and integer sums give the same bits on every run
// and every grid.  F is the same for a whole sweep: with
// B = max_I |c_I| * N_det * Hmax, where Hmax bounds every |<J|H|alpha>|
// (max |h| + 2 (n_el + 1) max |(pq|rs)|), |A_alpha| <= B < 2^(94 - F), so no
// sum leaves the 95-bit range and every product lies below 2^94 * 2^-F.  The
// sum is rounded once to FP64 in the cells pass; it keeps everything above
// 2^-F (about 1e-21 on the workloads here), more than an FP64 sum of the
// same products keeps.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int fix_scale(const SweepParams& p) {
  const double cmax = __longlong_as_double((long long)*p.cmax_bits);
  const double hmx = __longlong_as_double((long long)p.hmax_bits[0]);
  const double emx = __longlong_as_double((long long)p.hmax_bits[1]);
  const double hmax = hmx + 2.0 * (double)(p.nel + 1) * emx;
  const double bound = cmax * (double)p.ndet * hmax;
  if (!(bound > 0.0)) return 100;
  // floor(log2(bound)) from the exponent field; 2^(e+1) > bound
  const int e = (int)((((unsigned long long)__double_as_longlong(bound)) >> 52) & 0x7FF) - 1023;
  int F = 93 - e;
  if (F > 126) F = 126;
  if (F < 0) {  // coefficients times integrals beyond 2^93: not representable
    atomicOr(p.err, 64);
    F = 0;
  }
  return F;
}

// m * 2^sh as a 96-bit integer (lo, hi), negated when neg; m < 2^53 and
// m * 2^sh < 2^94; for sh < 0 the bits below 2^0 are rounded (half up).
__device__ __forceinline__ void fix_of_mant(unsigned long long m, int sh, bool neg, unsigned long long& lo,
                                            int& hi) {
  unsigned long long l;
  unsigned int h;
  if (sh >= 64) {
    l = 0ull;
    h = (unsigned int)(m << (sh - 64));
  } else if (sh > 0) {
    l = m << sh;
    h = (unsigned int)(m >> (64 - sh));
  } else if (sh == 0) {
    l = m;
    h = 0u;
  } else {
    const int r = -sh;
    l = (r < 64) ? (m >> r) + ((m >> (r - 1)) & 1ull) : 0ull;
    h = 0u;
  }
  if (neg) {
    l = ~l + 1ull;
    h = ~h + (l == 0ull ? 1u : 0u);
  }
  lo = l;
  hi = (int)h;
}

__device__ __forceinline__ void fix_of(double x, int F, unsigned long long& lo, int& hi) {
  const unsigned long long b = (unsigned long long)__double_as_longlong(x);
  const int e = (int)((b >> 52) & 0x7FF);
  if (e == 0) {  // zero, or below 2^-1022: nothing at 2^-F (F <= 126)
    lo = 0ull;
    hi = 0;
    return;
  }
  fix_of_mant((b & 0x000FFFFFFFFFFFFFull) | 0x0010000000000000ull, e - 1075 + F, (b >> 63) != 0ull, lo, hi);
}

__device__ __forceinline__ void fix_of(float x, int F, unsigned long long& lo, int& hi) {
  const unsigned int b = (unsigned int)__float_as_int(x);
  const int e = (int)((b >> 23) & 0xFF);
  if (e == 0) {
    lo = 0ull;
    hi = 0;
    return;
  }
  fix_of_mant((unsigned long long)((b & 0x7FFFFFu) | 0x800000u), e - 150 + F, (b >> 31) != 0u, lo, hi);
}

__device__ __forceinline__ void fix_add(unsigned long long& lo, int& hi, unsigned long long l2, int h2) {
  lo += l2;
  hi += h2 + (lo < l2 ? 1 : 0);
}

// Adds (l, h) into the shared-memory accumulator of cell cc: the low words
// add modulo 2^64 and each carry out of them is added to the high word, so
// the total is exact whatever the order of the atomics.
__device__ __forceinline__ void fix_atomic_add(unsigned long long* Alo, int* Ahi, int cc, unsigned long long l,
                                               int h) {
  const unsigned long long old = atomicAdd(&Alo[cc], l);
  const int dh = h + ((old + l < old) ? 1 : 0);
  if (dh) atomicAdd(&Ahi[cc], dh);
}

// (lo, hi) * 2^-F rounded to FP64 (nearest, ties away from zero): the top
// 53 bits of the magnitude, with integer operations only.
__device__ __forceinline__ double fix_to_double(unsigned long long lo, int hi, int F) {
  const bool neg = hi < 0;
  if (neg) {
    lo = ~lo + 1ull;
    hi = (int)(~(unsigned int)hi + (lo == 0ull ? 1u : 0u));
  }
  int n;  // bit length of the magnitude
  if (hi) n = 96 - __clz(hi);
  else if (lo) n = 64 - __clzll((long long)lo);
  else return 0.0;
  unsigned long long mant;
  if (n <= 53) {
    mant = lo << (53 - n);
  } else {
    const int s = n - 53;  // 1 .. 42
    const unsigned long long q = (lo >> s) | ((unsigned long long)(unsigned int)hi << (64 - s));
    mant = q + ((lo >> (s - 1)) & 1ull);
    if (mant >> 53) {
      mant >>= 1;
      n++;
    }
  }
  const unsigned long long ex = (unsigned long long)(n - 1 - F + 1023);
  return __longlong_as_double((long long)((neg ? 0x8000000000000000ull : 0ull) | (ex << 52) |
                                          (mant & 0x000FFFFFFFFFFFFFull)));
}

__device__ __forceinline__ int pair_batch(int nel, int i, int j) {  // i < j
  return nel + j * (j - 1) / 2 + i;
}

// Buckets reached by a record with hole mask hm (see the file header).
template <typename Fn>
__device__ __forceinline__ void for_buckets(uint64_t hm, int nel, int nbat, Fn&& fn) {
  const int d = __popcll(hm);
  if (d <= 2) {
    fn(nbat);
    return;
  }
  int Q[4], n = 0;
  uint64_t m = hm;
  while (m && n < 4) {
    Q[n++] = __ffsll((long long)m) - 1;
    m &= m - 1;
  }
  if (d == 3) {  // the list of each hole q: read by the batches holding q
    for (int i = 0; i < 3; i++) fn(Q[i]);
  } else {  // d == 4
    for (int i = 0; i < 4; i++)
      for (int j = i + 1; j < 4; j++) fn(pair_batch(nel, Q[i], Q[j]));
  }
}

// ---------------------------------------------------------------------------
// prep kernel: one CTA per generator slot of the wave
// ---------------------------------------------------------------------------
template <int NINT>
__device__ __forceinline__ void prep_slot(const SweepParams& p, const int slot) {
  constexpr int NW = 2 * NINT;
  __shared__ int s_cnt[kMaxBatch + 2];
  __shared__ uint32_t s_dead[(kMaxBatch + 31) / 32];
  __shared__ int s_wsum[kWarps];
  __shared__ uint64_t sI[NW];
  __shared__ int s_occ[kMaxElec];
  const int tid = threadIdx.x;
  const int norb = p.norb, nel = p.nel, nbat = p.nbat;
  GenMeta* M = p.meta + slot;
  // the slot's per-item sums start from zero (an item that adds nothing
  // does not write its sums)
  for (int j = tid; j < p.nper * p.it_stride; j += kThreads) p.it_sum[(size_t)slot * p.nper * p.it_stride + j] = 0.0;
  const long long t = (long long)p.wave_start + slot;
  const long long gg = p.gen_list ? (long long)p.gen_list[t] : p.shard_index + t * (long long)p.shard_count;
  if (gg >= p.ndet) {
    if (tid == 0) {
      M->g = -1;
      M->nrec = 0;
    }
    return;
  }
  const int g = (int)gg, gi = p.order[g];
  if (tid < NW) sI[tid] = p.dets[(size_t)gi * NW + tid];
  __syncthreads();
  if (tid == 0) {
    int n = 0;
    for (int s = 0; s < 2; s++)
      for (int q = 0; q < norb; q++)
        if ((sI[s * NINT + (q >> 6)] >> (q & 63)) & 1ull) s_occ[n++] = s * norb + q;
    M->g = g;
    M->cI = p.coefs[gi];
    for (int w = 0; w < 4; w++) M->I[w] = w < NW ? sI[w] : 0ull;
  }
  __syncthreads();
  if (tid < nel) M->occ[tid] = s_occ[tid];
  // Fock diagonal F_s(q) = h_qq + sum_{j in I} [(qq|jj) - delta_s (qj|jq)]
  for (int x = tid; x < 2 * norb; x += kThreads) {
    const int s = x / norb, q = x - s * norb;
    double f = p.h[q * norb + q];
    for (int i = 0; i < nel; i++) {
      const int c = s_occ[i], sj = c >= norb, j = c - sj * norb;
      f += p.Jm[q * norb + j];
      if (sj == s) f -= p.Km[q * norb + j];
    }
    M->F[s][q] = f;
  }
  __syncthreads();
  if (tid == 0) {  // H_II = 1/2 sum_i (h_ii + F(i))
    double e = 0.0;
    for (int i = 0; i < nel; i++) {
      const int c = s_occ[i], s = c >= norb, q = c - s * norb;
      e += p.h[q * norb + q] + M->F[s][q];
    }
    M->hii = 0.5 * e;
  }

  // ---- coarse filter: J within degree 4 of I (I itself included) ----
  const size_t rb = (size_t)slot * (size_t)p.ndet;
  uint64_t* rw = p.r_words + rb * NW;
  double* rc = p.r_coef + rb;
  uint64_t* rh = p.r_hmask + rb;
  uint64_t* rp = p.r_part + rb;
  uint32_t* rf = p.r_flag + rb;
  uint64_t Iw[NW];
#pragma unroll
  for (int w = 0; w < NW; w++) Iw[w] = sI[w];
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
    const int pos = block_scan_flag(keep, s_wsum, &total);
    if (keep) {
      const int r = nrec + pos;
      uint64_t hmask = 0, part = 0x7FFF7FFF7FFF7FFFull;  // four unused fields (kNoPart)
      int npart = 0;
#pragma unroll
      for (int s = 0; s < 2; s++) {
        int below = (s == 0) ? 0 : p.nalpha;
#pragma unroll
        for (int w = 0; w < NINT; w++) {
          const uint64_t iw = Iw[s * NINT + w], jw = Jw[s * NINT + w];
          uint64_t miss = iw & ~jw;
          while (miss) {
            const int b = __ffsll((long long)miss) - 1;
            miss &= miss - 1;
            hmask |= 1ull << (below + __popcll(iw & ((1ull << b) - 1)));
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
      for (int w = 0; w < NW; w++) rw[(size_t)r * NW + w] = Jw[w];
      rc[r] = p.coefs[j];
      for (int st = 1; st < p.nst; st++) rc[st * p.rc_stride + r] = p.coefs[(size_t)st * p.ndet + j];
      rh[r] = hmask;
      rp[r] = part;
      rf[r] = (p.rank_of[j] < g) ? 1u : 0u;
    }
    nrec += total;
  }
  if (tid == 0) M->nrec = nrec;

  // ---- buckets: counting sort of the records into the batches they reach ----
  for (int b = tid; b <= nbat + 1; b += kThreads) s_cnt[b] = 0;
  __syncthreads();
  for (int r = tid; r < nrec; r += kThreads)
    for_buckets(rh[r], nel, nbat, [&](int b) { atomicAdd(&s_cnt[b], 1); });
  __syncthreads();
  if (tid == 0) {
    int run = 0;
    for (int b = 0; b <= nbat; b++) {
      const int c = s_cnt[b];
      s_cnt[b] = run;
      run += c;
    }
    s_cnt[nbat + 1] = run;
    if (run > p.ent_cap) atomicOr(p.err, 8);
  }
  __syncthreads();
  int* ofs = p.b_ofs + (size_t)slot * (nbat + 2);
  for (int b = tid; b <= nbat + 1; b += kThreads) ofs[b] = s_cnt[b];
  __syncthreads();
  ulonglong2* e_hp = p.e_hp + (size_t)slot * (size_t)p.ent_cap;
  uint32_t* e_rec = p.e_rec + (size_t)slot * (size_t)p.ent_cap;
  const long long cap = p.ent_cap;
  for (int r = tid; r < nrec; r += kThreads) {
    const uint32_t before = rf[r] & 1u;
    const uint64_t hm = rh[r], pt = rp[r] | (before ? kBeforeBit : 0ull);
    const uint32_t rec = (uint32_t)r | (before << 31);
    for_buckets(hm, nel, nbat, [&](int b) {
      const int o = atomicAdd(&s_cnt[b], 1);
      if (o < cap) {
        e_hp[o] = make_ulonglong2(hm, pt);
        e_rec[o] = rec;
      }
    });
  }

  // ---- batches banned as a whole: a J ranked before I with t <= 1 (one
  // hole) or t = 0 (two holes) reaches every cell.  Only J with d <= 2 can:
  // d = 1 (holes {q}) kills every one-hole batch and the pairs holding q;
  // d = 2 (holes {q1, q2}) kills {q1}, {q2} and {q1, q2}. ----
  const int dw = (nbat + 31) / 32;
  for (int w = tid; w < dw; w += kThreads) s_dead[w] = 0u;
  __syncthreads();
  auto kill = [&](int b) { atomicOr(&s_dead[b >> 5], 1u << (b & 31)); };
  for (int r = tid; r < nrec; r += kThreads) {
    if (!(rf[r] & 1u)) continue;
    const uint64_t hm = rh[r];
    const int d = __popcll(hm);
    if (d == 1) {
      const int q = __ffsll((long long)hm) - 1;
      for (int i = 0; i < nel; i++) kill(i);
      for (int o = 0; o < nel; o++)
        if (o != q) kill(pair_batch(nel, q < o ? q : o, q < o ? o : q));
    } else if (d == 2) {
      const int q1 = __ffsll((long long)hm) - 1;
      const int q2 = __ffsll((long long)(hm & (hm - 1))) - 1;
      kill(q1);
      kill(q2);
      kill(pair_batch(nel, q1, q2));
    }
  }
  __syncthreads();
  uint32_t* dead = p.b_dead + (size_t)slot * dw;
  for (int w = tid; w < dw; w += kThreads) dead[w] = s_dead[w];
}

// One CTA per generator slot of the wave.
template <int NINT>
__global__ void __launch_bounds__(kThreads) prep_kernel(const __grid_constant__ SweepParams p) {
  prep_slot<NINT>(p, blockIdx.x);
}

// ---------------------------------------------------------------------------
// Several instances in one launch (a wave of each of their sweeps).  ps[i] is
// instance i's parameters for this wave; slot_ofs / item_ofs number the
// instances' generator slots / work items one instance after the other.
// ---------------------------------------------------------------------------
static_assert(sizeof(SweepParams) % 8 == 0, "parameters are copied by 8-byte words");

// Copy the parameters of instance i to shared memory (all threads).
__device__ __forceinline__ void load_params(SweepParams& dst, const SweepParams* ps, int i) {
  const unsigned long long* src = reinterpret_cast<const unsigned long long*>(ps + i);
  unsigned long long* d = reinterpret_cast<unsigned long long*>(&dst);
  for (int w = threadIdx.x; w < (int)(sizeof(SweepParams) / 8); w += blockDim.x) d[w] = src[w];
}

// The last instance whose first slot (item) is at or below x.
template <typename T>
__device__ __forceinline__ int instance_of(const T* ofs, int n, long long x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if ((long long)ofs[mid] <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// One CTA per generator slot of every instance of the wave.
template <int NINT>
__global__ void __launch_bounds__(kThreads) prep_multi_kernel(const __grid_constant__ MultiWave m) {
  __shared__ SweepParams Ps;
  __shared__ int s_inst;
  if (threadIdx.x == 0) s_inst = instance_of(m.slot_ofs, m.n, blockIdx.x);
  __syncthreads();
  const int i = s_inst;
  load_params(Ps, m.ps, i);
  __syncthreads();
  prep_slot<NINT>(Ps, (int)blockIdx.x - m.slot_ofs[i]);
}

// ---------------------------------------------------------------------------
// batch kernel
// ---------------------------------------------------------------------------
template <int NINT, typename NT>
struct BatchShared {
  uint64_t I[2 * NINT];
  int occ[kMaxElec];
  int vir[2][kMaxOrb];
  int vidx[2][kMaxOrb];
  int nv[2];
  double F[2][kMaxOrb];
  double u0[kMaxOrb], u1[kMaxOrb];  // per-batch row sums for H_aa
  double dx[kMaxOrb];               // E0 - base - u0[x]
  // two-hole batches: <I|H|I - H + R> by the pair tables of the all-cell
  // fast path, built for J = I (its X is the hole pair H itself)
  int iRow[kMaxOrb], iCol[kMaxOrb];
  NT cI;
  double hii, base;
  float inv_nv1;
  uint64_t kbase[2 * NINT];  // I with the batch's holes removed
  int g, slot;
  long long item, inext, iend;
  // storage of one phase of a work item at a time: the J lists of loops 2
  // and 3, the selection histogram, the per-thread sums of the reduction
  union {
    struct {
      // records of the J reaching every cell; of the J reaching rows (from
      // the front) and a few cells (from the back)
      int L0[kChunk], L12[kChunk];
    } l;
    int hist[256];
    double red_t[2][kThreads];  // per-thread e and (A/D)^2 sums of the item
  } u;
  int n0, n1, n2;
  int cnext;  // next row-reaching J (then subset block) to draw
  // a group of J reaching every cell, processed by the whole CTA
  uint64_t gJw[kGroup][2 * NINT];
  NT gcj[kGroup];
  uint32_t gX[kGroup], gT[kGroup];
  int gnx[kGroup], gnt[kGroup];
  // two-hole batches: J = K + {x1, x2}; per particle orbital of each slot the
  // pair index tri(x, r) with the phase parity in bit 31
  // (loop 2); the gradient's per-orbital weights use the same storage in
  // the cells pass and after loop 3
  union {
    struct {
      int gRow[kGroup][kMaxOrb], gCol[kGroup][kMaxOrb];
    } g;
    struct {
      double rowW2[kMaxOrb], colW2[kMaxOrb];  // sums of (A/D)^2 over the cells of each particle orbital
    } w;
    // loop 1: flags of the rows (rowm) and columns (colm) of cells that J
    // ranked before I reach as a whole (by virtual orbital index)
    struct {
      uint32_t rowm[kMaxOrb], colm[kMaxOrb];
    } m;
  } v;
  int gx1[kGroup], gx2[kGroup], gsr[kGroup], gsc[kGroup];
  // four-index layout: the slab of each J's pair (x1, x2) and of the batch's
  // holes; the pair tables then hold orbitals, not pair indices
  int gB[kGroup], ibase;
  // two-hole batches, after loop 1: bit x of frow (fcol) set when row
  // (column) x of cells is banned as a whole by a J ranked before I
  uint32_t frow[kMaxOrb / 32], fcol[kMaxOrb / 32];
  int wsum[kWarps];
  // selection
  int tkcnt;
  unsigned long long tau;
  uint64_t pw[1 + 2 * NINT];
  uint64_t thr[1 + 2 * NINT];
  int need, group, found_w, found_sh;
  // reductions
  unsigned long long red_u[kWarps][6];
  double sw2;
};

struct Batch {
  int h;            // number of holes (1, 2)
  int kind;         // 0 single, 1 same-spin double, 2 opposite-spin double
  int ia, ib;       // occupied indices of the holes in I
  int ca, cb;       // their spin-orbital codes
  int sa, sb;       // their spins
  int qa, qb;       // their orbitals
  uint64_t hm;      // hole mask over I's occupied list
  int ncell;
  int clo, nct;     // this work item's cells: [clo, clo + nct) (a tile of the batch)
};

template <int NINT, typename NT>
__device__ __forceinline__ void cell_orbitals(const Batch& B, const BatchShared<NINT, NT>& S, int c, int* r,
                                              int* s, int* x, int* y) {
  if (B.kind == 0) {
    *x = c;
    *y = -1;
    *r = S.vir[B.sa][c];
    *s = -1;
  } else if (B.kind == 2) {
    const int nv1 = S.nv[1];
    int xx = __float2int_rz((float)c * S.inv_nv1);  // c < 2^14: exact up to one step
    if (xx * nv1 > c) xx--;
    if ((xx + 1) * nv1 <= c) xx++;
    *x = xx;
    *y = c - xx * nv1;
    *r = S.vir[0][xx];
    *s = S.vir[1][*y];
  } else {
    int yy = (int)((1.0f + sqrtf(1.0f + 8.0f * (float)c)) * 0.5f);
    while (yy * (yy - 1) / 2 > c) yy--;
    while ((yy + 1) * yy / 2 <= c) yy++;
    *x = c - yy * (yy - 1) / 2;
    *y = yy;
    *r = S.vir[B.sa][*x];
    *s = S.vir[B.sa][yy];
  }
}

// Bans cell c (an index over the whole batch) when it lies in this item's tile.
__device__ __forceinline__ void ban_cell(uint32_t* ban, const Batch& B, int c) {
  const int cc = c - B.clo;
  if ((unsigned)cc < (unsigned)B.nct) atomicOr(&ban[cc >> 5], 1u << (cc & 31));
}

__device__ __forceinline__ int pair_cell(int x, int y) {  // x != y virtual indices
  int lo = x < y ? x : y, hi = x < y ? y : x;
  return hi * (hi - 1) / 2 + lo;
}

// Small sets are packed 8 bits per entry into a 32-bit register (orbitals
// < 128, spin-orbital codes < 256) with the count kept beside them: arrays
// indexed at run time would live in local memory.
__device__ __forceinline__ int pk(uint32_t v, int i) { return (int)((v >> (8 * i)) & 0xFFu); }

// A bucket entry's particle word: four 16-bit fields, each the spin-orbital
// code s*norb + q (< 256) of a particle of J outside I, or kNoPart.  Bit 15
// (the top bit of the first field, which always holds a particle when it is
// set) flags a J ranked before I, so that one 16-byte load of the entry
// (hole mask, particle word) is all the classification reads.
constexpr int kNoPart = 0x7FFF;
__device__ __forceinline__ int part_code(uint64_t part, int i) { return (int)((part >> (16 * i)) & 0x7FFF); }

// Particles of J outside I, filtered to a spin, as orbitals (packed).
__device__ __forceinline__ uint32_t particles_of_spin(uint64_t part, int norb, int spin, int* n) {
  uint32_t out = 0;
  int k = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int c = part_code(part, i);
    if (c == kNoPart) continue;
    const int s = c >= norb;
    if (s == spin) {
      out |= (uint32_t)(c - s * norb) << (8 * k);
      k++;
    }
  }
  *n = k;
  return out;
}

// Cells inside the particles of J (t = 2): visited by one thread.
template <int NINT, typename NT, typename Fn>
__device__ __forceinline__ void for_subset_cells(const Batch& B, const BatchShared<NINT, NT>& S, int norb,
                                                 uint64_t part, Fn&& fn) {
  if (B.kind == 0) {
    int np;
    const uint32_t P = particles_of_spin(part, norb, B.sa, &np);
    for (int i = 0; i < np; i++) fn(S.vidx[B.sa][pk(P, i)]);
  } else if (B.kind == 1) {
    int np;
    const uint32_t P = particles_of_spin(part, norb, B.sa, &np);
    for (int i = 0; i < np; i++)
      for (int j = i + 1; j < np; j++) fn(pair_cell(S.vidx[B.sa][pk(P, i)], S.vidx[B.sa][pk(P, j)]));
  } else {
    int na, nb;
    const uint32_t Pa = particles_of_spin(part, norb, 0, &na);
    const uint32_t Pb = particles_of_spin(part, norb, 1, &nb);
    for (int i = 0; i < na; i++)
      for (int j = 0; j < nb; j++) fn(S.vidx[0][pk(Pa, i)] * S.nv[1] + S.vidx[1][pk(Pb, j)]);
  }
}

// True when some cell inside the particles of J lies in this item's tile and
// is not banned: a J with t = 2 that reaches no such cell adds nothing and is
// dropped at classification (most of them: their one cell is usually banned
// by an earlier generator, or its spins do not match the batch's).
template <int NINT, typename NT>
__device__ __forceinline__ bool subset_live(const Batch& B, const BatchShared<NINT, NT>& S, int norb,
                                            uint64_t part, const uint32_t* ban) {
  bool live = false;
  for_subset_cells<NINT, NT>(B, S, norb, part, [&](int c) {
    const int cc = c - B.clo;
    live |= (unsigned)cc < (unsigned)B.nct && !((ban[cc >> 5] >> (cc & 31)) & 1u);
  });
  return live;
}

__device__ __forceinline__ bool flagged(const uint32_t* f, int x) { return (f[x >> 5] >> (x & 31)) & 1u; }

// True when some row or column of cells that a J with t = 1 reaches (the
// rows of its particles) is not banned as a whole.  Rows flagged in loop 1
// hold no live cell, so a J whose rows are all flagged adds nothing: it is
// dropped at classification (the rows and columns of a J ranked after I are
// mostly those of earlier J with the same particles).
template <int NINT, typename NT>
__device__ __forceinline__ bool row_live(const Batch& B, const BatchShared<NINT, NT>& S, int norb, uint64_t part) {
  bool live = false;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int c = part_code(part, i);
    if (c == kNoPart) continue;
    const int s = c >= norb, q = c - s * norb;
    if (B.kind == 2) live |= !flagged(s ? S.fcol : S.frow, S.vidx[s][q]);
    else if (s == B.sa) live |= !flagged(S.frow, S.vidx[s][q]);
  }
  return live;
}

// Cells touching the particles of J (two-hole batch, t = 1): visited by the
// 32 lanes of a warp, each cell once.  Rows and columns banned as a whole are
// skipped (a cell they share with another row is banned too).  fn(c, pc, zc)
// gets the cell index, the spin-orbital code of the particle of J whose row
// it is and the code of the cell's other orbital.
template <int NINT, typename NT, typename Fn>
__device__ __forceinline__ void for_row_cells(const Batch& B, const BatchShared<NINT, NT>& S, int norb,
                                              uint64_t part, int lane, Fn&& fn) {
  if (B.kind == 1) {
    int np;
    const uint32_t P = particles_of_spin(part, norb, B.sa, &np);
    const int nv = S.nv[B.sa];
    for (int i = 0; i < np; i++) {
      const int x = S.vidx[B.sa][pk(P, i)];
      if (flagged(S.frow, x)) continue;
      for (int y = lane; y < nv; y += 32) {
        if (y == x) continue;
        bool dup = false;  // pair {P[j], P[i]}, j < i, was visited from P[j]
        for (int j = 0; j < i; j++) dup |= (S.vidx[B.sa][pk(P, j)] == y);
        if (!dup) fn(pair_cell(x, y), B.sa * norb + pk(P, i), B.sa * norb + S.vir[B.sa][y]);
      }
    }
  } else {  // kind 2
    int na, nb;
    const uint32_t Pa = particles_of_spin(part, norb, 0, &na);
    const uint32_t Pb = particles_of_spin(part, norb, 1, &nb);
    const int nv0 = S.nv[0], nv1 = S.nv[1];
    for (int i = 0; i < na; i++) {
      const int x = S.vidx[0][pk(Pa, i)];
      if (flagged(S.frow, x)) continue;
      for (int y = lane; y < nv1; y += 32) fn(x * nv1 + y, pk(Pa, i), norb + S.vir[1][y]);
    }
    for (int j = 0; j < nb; j++) {
      const int y = S.vidx[1][pk(Pb, j)];
      if (flagged(S.fcol, y)) continue;
      for (int x = lane; x < nv0; x += 32) {
        bool dup = false;  // rows of Pa were visited above
        for (int i = 0; i < na; i++) dup |= (S.vidx[0][pk(Pa, i)] == x);
        if (!dup) fn(x * nv1 + y, norb + pk(Pb, j), S.vir[0][x]);
      }
    }
  }
}

// X = (particles of J) + (holes of H that J keeps); T = holes of J not in H.
// Both sets are spin-orbital codes, packed (see pk).
template <int NINT, typename NT>
__device__ __forceinline__ void excitation_sets(const Batch& B, const BatchShared<NINT, NT>& S, uint64_t part,
                                                uint64_t hm, uint32_t* X, int* nx, uint32_t* T, int* nt) {
  int a = 0, b = 0;
  uint32_t xs = 0, ts = 0;
#pragma unroll
  for (int i = 0; i < 4; i++) {
    const int c = part_code(part, i);
    if (c != kNoPart && a < 4) xs |= (uint32_t)c << (8 * a++);
  }
  if (!((hm >> B.ia) & 1ull) && a < 4) xs |= (uint32_t)B.ca << (8 * a++);
  if (B.h == 2 && !((hm >> B.ib) & 1ull) && a < 4) xs |= (uint32_t)B.cb << (8 * a++);
  uint64_t tm = hm & ~B.hm;
  while (tm && b < 2) {
    const int i = __ffsll((long long)tm) - 1;
    tm &= tm - 1;
    ts |= (uint32_t)S.occ[i] << (8 * b++);
  }
  *X = xs;
  *nx = a;
  *T = ts;
  *nt = b;
}

// <J|H|alpha> with alpha = K + R, K = I - H.
// holes(J -> alpha) = X - R, particles = T + (R - X).
// Kept out of line: one copy serves every caller, which keeps the batch
// kernel's code small enough for the instruction cache.
// Jw points to the record's words in global or shared memory; the sets are
// packed codes; nothing is passed through local memory.
template <int NINT, typename NT, bool E4>
__device__ __noinline__ NT element(const NT* eri, const NT* hh, int norb, const uint64_t* Jw, uint32_t X, int nx,
                                   uint32_t T, int nt, int r, int s) {
  int ho[2], pa[2], nh = 0, npp = 0;
  bool r_in = false, s_in = false;
  for (int i = 0; i < nx; i++) {
    const int x = pk(X, i);
    r_in |= (x == r);
    s_in |= (x == s);
    if (x != r && x != s && nh < 2) ho[nh++] = x;
  }
  for (int i = 0; i < nt && npp < 2; i++) pa[npp++] = pk(T, i);
  if (!r_in && npp < 2) pa[npp++] = r;
  if (s >= 0 && !s_in && npp < 2) pa[npp++] = s;
  if (nh == 0 || nh != npp) return NT(0);  // not reached: such cells are banned
  if (nh == 1) {
    const int sp = ho[0] >= norb, a = ho[0] - sp * norb, b = pa[0] - sp * norb;
    const uint64_t* sw = Jw + sp * NINT;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const bool neg = count_between<NINT>(sw, lo, hi) & 1;
    NT v = hh[a * norb + b];
#pragma unroll
    for (int t = 0; t < 2; t++) {
#pragma unroll
      for (int w = 0; w < NINT; w++) {
        uint64_t bits = Jw[t * NINT + w];
        while (bits) {
          const int q = 64 * w + __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          v += eri[gidx<E4>(a, b, q, q, norb)];
          if (t == sp) v -= eri[gidx<E4>(a, q, q, b, norb)];
        }
      }
    }
    return flip_sign(v, neg);
  }
  // double: order holes and particles by spin-orbital code, pair 1-1, 2-2
  if (ho[0] > ho[1]) { const int t = ho[0]; ho[0] = ho[1]; ho[1] = t; }
  if (pa[0] > pa[1]) { const int t = pa[0]; pa[0] = pa[1]; pa[1] = t; }
  const int s1 = ho[0] >= norb, s2 = ho[1] >= norb;
  const int h1 = ho[0] - s1 * norb, p1 = pa[0] - s1 * norb;
  const int h2 = ho[1] - s2 * norb, p2 = pa[1] - s2 * norb;
  uint64_t w1[NINT];
#pragma unroll
  for (int w = 0; w < NINT; w++) w1[w] = Jw[s1 * NINT + w];
  const int n1 = count_between<NINT>(w1, h1 < p1 ? h1 : p1, h1 < p1 ? p1 : h1);
  // apply h1 -> p1, then count for h2 -> p2 on the result
  w1[h1 >> 6] &= ~(1ull << (h1 & 63));
  w1[p1 >> 6] |= (1ull << (p1 & 63));
  const int n2 = (s2 == s1) ? count_between<NINT>(w1, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2)
                            : count_between<NINT>(Jw + s2 * NINT, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  NT v = eri[gidx<E4>(h1, p1, h2, p2, norb)];
  if (s1 == s2) v -= eri[gidx<E4>(h1, p2, h2, p1, norb)];
  return flip_sign(v, (n1 + n2) & 1);
}

// <J|H|alpha> for a cell of the row pass whose substitution from J is a
// double: holes u0 < u1 (X without the row's particle), particles q (the
// hole of J outside the batch) and z (the cell's other orbital, not in X).
// The same pairing and phases as element(), inline: the row pass evaluates
// most of its cells here.
template <int NINT, typename NT, bool E4>
__device__ __forceinline__ NT row_double(const NT* eri, int norb, const uint64_t* jw, int u0, int u1, int q, int z) {
  const int pa0 = q < z ? q : z, pa1 = q < z ? z : q;
  const int s1 = u0 >= norb, s2 = u1 >= norb;
  const int h1 = u0 - s1 * norb, p1 = pa0 - s1 * norb;
  const int h2 = u1 - s2 * norb, p2 = pa1 - s2 * norb;
  uint64_t w1[NINT];
#pragma unroll
  for (int w = 0; w < NINT; w++) w1[w] = s1 ? jw[NINT + w] : jw[w];
  const int n1 = count_between<NINT>(w1, h1 < p1 ? h1 : p1, h1 < p1 ? p1 : h1);
  if (s2 == s1) {
    w1[h1 >> 6] &= ~(1ull << (h1 & 63));
    w1[p1 >> 6] |= (1ull << (p1 & 63));
  } else {
#pragma unroll
    for (int w = 0; w < NINT; w++) w1[w] = s2 ? jw[NINT + w] : jw[w];
  }
  const int n2 = count_between<NINT>(w1, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  NT v = eri[gidx<E4>(h1, p1, h2, p2, norb)];
  if (s1 == s2) v -= eri[gidx<E4>(h1, p2, h2, p1, norb)];
  return flip_sign(v, (n1 + n2) & 1);
}

// Gradient of one matrix element: adds w * d<J|H|alpha>/d(theta) into dh
// (symmetric halves) and the packed integrals, with the same case analysis
// as element().
template <int NINT>
__device__ __noinline__ void element_grad(double* g_dh, double* g_deri, int norb, const uint64_t* Jw, uint32_t X,
                                          int nx, uint32_t T, int nt, int r, int s, double w) {
  int ho[2], pa[2], nh = 0, npp = 0;
  bool r_in = false, s_in = false;
  for (int i = 0; i < nx; i++) {
    const int x = pk(X, i);
    r_in |= (x == r);
    s_in |= (x == s);
    if (x != r && x != s && nh < 2) ho[nh++] = x;
  }
  for (int i = 0; i < nt && npp < 2; i++) pa[npp++] = pk(T, i);
  if (!r_in && npp < 2) pa[npp++] = r;
  if (s >= 0 && !s_in && npp < 2) pa[npp++] = s;
  if (nh == 0 || nh != npp) return;
  if (nh == 1) {
    const int sp = ho[0] >= norb, a = ho[0] - sp * norb, b = pa[0] - sp * norb;
    const uint64_t* sw = Jw + sp * NINT;
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    const double ws = (count_between<NINT>(sw, lo, hi) & 1) ? -w : w;
    atomicAdd(&g_dh[a * norb + b], 0.5 * ws);
    atomicAdd(&g_dh[b * norb + a], 0.5 * ws);
#pragma unroll
    for (int t = 0; t < 2; t++) {
#pragma unroll
      for (int wd = 0; wd < NINT; wd++) {
        uint64_t bits = Jw[t * NINT + wd];
        while (bits) {
          const int q = 64 * wd + __ffsll((long long)bits) - 1;
          bits &= bits - 1;
          atomicAdd(&g_deri[eri_index(a, b, q, q)], ws);
          if (t == sp) atomicAdd(&g_deri[eri_index(a, q, q, b)], -ws);
        }
      }
    }
    return;
  }
  if (ho[0] > ho[1]) { const int t = ho[0]; ho[0] = ho[1]; ho[1] = t; }
  if (pa[0] > pa[1]) { const int t = pa[0]; pa[0] = pa[1]; pa[1] = t; }
  const int s1 = ho[0] >= norb, s2 = ho[1] >= norb;
  const int h1 = ho[0] - s1 * norb, p1 = pa[0] - s1 * norb;
  const int h2 = ho[1] - s2 * norb, p2 = pa[1] - s2 * norb;
  uint64_t w1[NINT];
#pragma unroll
  for (int wd = 0; wd < NINT; wd++) w1[wd] = Jw[s1 * NINT + wd];
  const int n1 = count_between<NINT>(w1, h1 < p1 ? h1 : p1, h1 < p1 ? p1 : h1);
  w1[h1 >> 6] &= ~(1ull << (h1 & 63));
  w1[p1 >> 6] |= (1ull << (p1 & 63));
  const int n2 = (s2 == s1) ? count_between<NINT>(w1, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2)
                            : count_between<NINT>(Jw + s2 * NINT, h2 < p2 ? h2 : p2, h2 < p2 ? p2 : h2);
  const double ws = ((n1 + n2) & 1) ? -w : w;
  atomicAdd(&g_deri[eri_index(h1, p1, h2, p2)], ws);
  if (s1 == s2) atomicAdd(&g_deri[eri_index(h1, p2, h2, p1)], -ws);
}

// w * dW(x, y)/d(theta), W(x, y) = (xx|yy) - delta_spin (xy|yx)
__device__ __forceinline__ void w_grad(const SweepParams& p, int x, int sx, int y, int sy, double w) {
  atomicAdd(&p.g_deri[eri_index(x, x, y, y)], w);
  if (sx == sy) atomicAdd(&p.g_deri[eri_index(x, y, y, x)], -w);
}

// ---------------------------------------------------------------------------
// Selection buffer compaction: keep the k best entries (|e| descending, key
// ascending) of the CTA's buffer.  MSD radix select over the composite
// (~bits(|e|), key words), 8-bit digits, then an ordered in-place compaction.
// ---------------------------------------------------------------------------
// Selection histogram bins: the binary exponent of |e| (2^-100 .. 2^27) and
// the top 3 mantissa bits, so that a bin's lower edge is a double whose bits
// are easy to form.  Values below 2^-100 fall in bin 0, whose edge is taken as
// 0; values of 2^28 and above fall in the last bin, whose edge is below them.
__device__ __forceinline__ int sel_bin(unsigned long long ebits) {
  const int ex = (int)(ebits >> 52) - 923;
  if (ex < 0) return 0;
  if (ex > 127) return kSelBins - 1;
  return ex * 8 + (int)((ebits >> 49) & 7ull);
}
__device__ __forceinline__ unsigned long long sel_bin_edge(int b) {
  return ((unsigned long long)(b / 8 + 923) << 52) | ((unsigned long long)(b % 8) << 49);
}

// A lower bound of the k-th largest |e| of the whole sweep: the lower edge of
// the highest bin at which at least k distinct perturbers (each counted once,
// when offered to a selection buffer) have |e| at or above the edge.
static __device__ unsigned long long hist_threshold(const unsigned int* hist, long long k) {
  const int lane = threadIdx.x & 31;
  constexpr int per = kSelBins / 32;
  // lane l owns bins [l*per, (l+1)*per); sums from the top
  unsigned long long mine = 0;
  for (int b = 0; b < per; b++) mine += hist[lane * per + b];
  unsigned long long suffix = mine;
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long v = __shfl_down_sync(0xffffffffu, suffix, o);
    if (lane + o < 32) suffix += v;
  }
  // suffix = counts in bins of lanes >= lane; the lane whose block holds the
  // k-th count from the top walks its bins
  const unsigned long long above_me = suffix - mine;
  unsigned long long res = 0;
  const bool holder = (above_me < (unsigned long long)k) && (suffix >= (unsigned long long)k);
  if (holder) {
    unsigned long long cum = above_me;
    for (int b = per - 1; b >= 0; b--) {
      cum += hist[lane * per + b];
      if (cum >= (unsigned long long)k) {
        const int bin = lane * per + b;
        res = bin > 0 ? sel_bin_edge(bin) : 0ull;
        break;
      }
    }
  }
  // broadcast from the holder lane (at most one)
  const unsigned m = __ballot_sync(0xffffffffu, holder);
  if (m == 0) return 0ull;
  return __shfl_sync(0xffffffffu, res, __ffs(m) - 1);
}

template <int NINT>
__device__ __forceinline__ uint64_t composite_word(const double* te, const uint64_t* tk, int i, int w) {
  if (w == 0) return ~((unsigned long long)__double_as_longlong(te[i]) & 0x7FFFFFFFFFFFFFFFull);
  return tk[(size_t)i * (2 * NINT) + (w - 1)];
}

template <int NINT>
__device__ bool prefix_match(const double* te, const uint64_t* tk, int i, const uint64_t* pw, int w,
                             int keep_sh) {
  for (int v = 0; v < w; v++)
    if (composite_word<NINT>(te, tk, i, v) != pw[v]) return false;
  if (keep_sh >= 64) return true;
  return (composite_word<NINT>(te, tk, i, w) >> keep_sh) == (pw[w] >> keep_sh);
}

template <int NINT, typename NT>
__device__ __noinline__ void compact_selection(const SweepParams& p, BatchShared<NINT, NT>& S, double* te,
                                               double* ta, uint64_t* tk) {
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
      for (int b = tid; b < 256; b += kThreads) S.u.hist[b] = 0;
      __syncthreads();
      for (int i = tid; i < n; i += kThreads)
        if (prefix_match<NINT>(te, tk, i, S.pw, w, sh + 8))
          atomicAdd(&S.u.hist[(composite_word<NINT>(te, tk, i, w) >> sh) & 255], 1);
      __syncthreads();
      if (tid == 0) {
        int c = 0, d = 255;
        for (int b = 0; b < 256; b++) {
          if (c + S.u.hist[b] >= S.need) {
            d = b;
            break;
          }
          c += S.u.hist[b];
        }
        S.need -= c;
        S.group = S.u.hist[d];
        S.pw[w] |= (uint64_t)d << sh;
        S.found_w = w;
        S.found_sh = sh;
      }
      __syncthreads();
      if (S.group <= 1) {
        done = true;
        break;
      }
    }
  }
  if (S.group == 1) {
    for (int i = tid; i < n; i += kThreads)
      if (prefix_match<NINT>(te, tk, i, S.pw, S.found_w, S.found_sh))
        for (int w = 0; w < NW; w++) S.thr[w] = composite_word<NINT>(te, tk, i, w);
  } else if (tid == 0) {
    for (int w = 0; w < NW; w++) S.thr[w] = S.pw[w];
  }
  __syncthreads();
  int out = 0;
  for (int base = 0; base < n; base += kThreads) {
    const int i = base + tid;
    bool keep = false;
    double e = 0, a = 0;
    uint64_t key[2 * NINT];
    if (i < n) {
      int cmp = 0;
      for (int w = 0; w < NW && cmp == 0; w++) {
        const uint64_t x = composite_word<NINT>(te, tk, i, w);
        cmp = x < S.thr[w] ? -1 : (x > S.thr[w] ? 1 : 0);
      }
      keep = cmp <= 0;
      e = te[i];
      a = ta[i];
#pragma unroll
      for (int w = 0; w < 2 * NINT; w++) key[w] = tk[(size_t)i * (2 * NINT) + w];
    }
    int total;
    const int pos = block_scan_flag(keep, S.wsum, &total);
    if (keep) {
      const int o = out + pos;
      te[o] = e;
      ta[o] = a;
#pragma unroll
      for (int w = 0; w < 2 * NINT; w++) tk[(size_t)o * (2 * NINT) + w] = key[w];
    }
    out += total;
  }
  __syncthreads();
  if (tid < 32) {
    const unsigned long long th = hist_threshold(p.sel_hist, k);
    if (tid == 0) {
      S.tkcnt = out;
      unsigned long long t = ~S.thr[0];
      t = th > t ? th : t;
      if (t > S.tau) S.tau = t;
      atomicMax(p.tau_bits, t);
    }
  }
  __syncthreads();
}

// The CTA's dynamic shared memory for the sweep of p and the sweep's sizes,
// formed by the kernel once (once per instance in the multi-instance kernel)
// and kept across work items.  Multi-state form: one FP64 accumulator per
// state (stride mc), then the ban bits, the CTA group's coefficients per
// state, c_I per state and the weights w_s; one-state form: the exact 96-bit
// accumulators (low words, then high words), then the ban bits.
struct ItemEnv {
  double* A;
  unsigned long long* Alo;
  int* Ahi;
  uint32_t* ban;
  double *ms_gc, *ms_cI, *ms_w;
  int mc, nst, norb, nel, nbat, nper;
};

template <bool MS>
__device__ __forceinline__ ItemEnv item_env(const SweepParams& p) {
  extern __shared__ __align__(16) unsigned char dyn[];
  ItemEnv E;
  E.mc = p.max_cells;
  E.A = reinterpret_cast<double*>(dyn);
  E.Alo = reinterpret_cast<unsigned long long*>(dyn);
  E.Ahi = reinterpret_cast<int*>(E.Alo + E.mc);
  E.ban = MS ? reinterpret_cast<uint32_t*>(E.A + p.nst * E.mc) : reinterpret_cast<uint32_t*>(E.Ahi + ((E.mc + 1) & ~1));
  E.ms_gc = reinterpret_cast<double*>(E.ban + (((E.mc + 31) / 32 + 1) & ~1));
  E.ms_cI = E.ms_gc + kGroup * kMaxStates;
  E.ms_w = E.ms_cI + kMaxStates;
  E.nst = MS ? p.nst : 1;
  E.norb = p.norb;
  E.nel = p.nel;
  E.nbat = p.nbat;
  E.nper = p.nper;
  return E;
}

// One work item of the sweep of p (a generator slot's hole-set batch, or a
// row tile of one): bans, the accumulation of A_alpha, the cells pass and the
// item's sums.  Used by the kernel of one sweep and by the kernel whose queue
// spans the waves of several instances.
template <int NINT, typename NT, bool GRAD, bool MS, bool E4>
__device__ __forceinline__ void batch_item(const SweepParams& p, BatchShared<NINT, NT>& S, const long long item,
                                           const int F, double* te, double* ta, uint64_t* tk, const ItemEnv& E,
                                           const NT* eri_n, const NT* h_n) {
  constexpr int NW = 2 * NINT;
  double* A = E.A;
  unsigned long long* Alo = E.Alo;
  int* Ahi = E.Ahi;
  uint32_t* ban = E.ban;
  double* ms_gc = E.ms_gc;
  double* ms_cI = E.ms_cI;
  double* ms_w = E.ms_w;
  const int mc = E.mc, nst = E.nst;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int norb = E.norb, nel = E.nel, nbat = E.nbat;
  const int nper = E.nper;

  const int slot = (int)(item / nper), j = (int)(item - (long long)slot * nper);
  // item j < nbat: batch j (the first row tile of a split batch); j >= nbat:
  // row tile 1 + (j - nbat) / (n_alpha n_beta) of opposite-spin batch
  // (j - nbat) % (n_alpha n_beta)
  int b = j, tile = 0;
  if (j >= nbat) {
    const int na = p.nalpha, nab = p.nalpha * p.nbeta;
    const int k = (j - nbat) % nab;
    tile = 1 + (j - nbat) / nab;
    const int ia = k % na, ib = na + k / na;
    b = nel + ib * (ib - 1) / 2 + ia;
  }
  const GenMeta* M = p.meta + slot;
  if (M->g < 0) return;
  if ((p.b_dead[(size_t)slot * ((nbat + 31) / 32) + (b >> 5)] >> (b & 31)) & 1u) return;
  if (slot != S.slot) {  // load the generator
    __syncthreads();
    if (tid < NW) S.I[tid] = M->I[tid];
    if (tid < nel) S.occ[tid] = M->occ[tid];
    for (int x = tid; x < 2 * norb; x += kThreads) S.F[x / norb][x % norb] = M->F[x / norb][x % norb];
    __syncthreads();
    for (int x = tid; x < 2 * norb; x += kThreads) {
      const int s = x / norb, q = x - s * norb;
      const uint64_t* sw = S.I + s * NINT;
      const bool occ = (sw[q >> 6] >> (q & 63)) & 1ull;
      int below = 0;  // occupied orbitals of spin s below q
#pragma unroll
      for (int w = 0; w < NINT; w++) {
        const int lim = q - 64 * w;
        if (lim >= 64) below += __popcll(sw[w]);
        else if (lim > 0) below += __popcll(sw[w] & ((1ull << lim) - 1));
      }
      const int v = q - below;
      S.vidx[s][q] = occ ? -1 : v;
      if (!occ) S.vir[s][v] = q;
    }
    if (tid < 2) {
      int n = 0;
#pragma unroll
      for (int w = 0; w < NINT; w++) n += __popcll(S.I[tid * NINT + w]);
      S.nv[tid] = norb - n;
    }
    if (tid == 0) {
      S.hii = M->hii;
      S.cI = (NT)M->cI;
      S.g = M->g;
      S.slot = slot;
    }
    if constexpr (MS) {
      if (tid < nst) {
        ms_cI[tid] = p.coefs[(size_t)tid * p.ndet + p.order[M->g]];
        const double m = __longlong_as_double((long long)p.st_cmax[tid]);
        ms_w[tid] = 1.0 / (m * m);
      }
    }
    __syncthreads();
  }
  const int g = S.g;

  // ---- batch geometry ----
  Batch B;
  if (b < nel) {
    B.h = 1;
    B.ia = b;
    B.ib = -1;
  } else {
    const int t = b - nel;
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
  B.clo = 0;
  B.nct = B.ncell;
  if (p.ntile > 1 && B.kind == 2) {  // rows [tile h, min((tile + 1) h, nv0))
    const int h = (S.nv[0] + p.ntile - 1) / p.ntile;
    const int r0 = tile * h, r1 = min(r0 + h, S.nv[0]);
    B.clo = r0 * S.nv[1];
    B.nct = (r1 - r0) * S.nv[1];
  }
  if (B.nct <= 0) return;

  // bucket lists: this batch's bucket, then the shared bucket (degree <= 2)
  const int* ofs = p.b_ofs + (size_t)slot * (nbat + 2);
  // entries: the batch's own bucket (one-hole batch {a}: the d = 3 records
  // holding a; two-hole batch: the d = 4 records holding both holes), then
  // for a two-hole batch {a, b} the d = 3 lists of a and of b (a record
  // holding both is taken from a's list only), then the shared bucket
  const int ob = ofs[b], nb_ = ofs[b + 1] - ob, oa = ofs[nbat], na_ = ofs[nbat + 1] - oa;
  const int o1 = (B.h == 2) ? ofs[B.ia] : 0, n1_ = (B.h == 2) ? ofs[B.ia + 1] - o1 : 0;
  const int o2 = (B.h == 2) ? ofs[B.ib] : 0, n2_ = (B.h == 2) ? ofs[B.ib + 1] - o2 : 0;
  const int s1 = nb_, s2 = s1 + n1_, s3 = s2 + n2_;
  const int total = s3 + na_;
  const size_t rb = (size_t)slot * (size_t)p.ndet;
  const uint64_t* rw = p.r_words + rb * NW;
  const double* rc = p.r_coef + rb;
  const uint64_t* rhm = p.r_hmask + rb;  // hole mask and particle word of each record
  const uint64_t* rpt = p.r_part + rb;
  const size_t eb = (size_t)slot * (size_t)p.ent_cap;
  const ulonglong2* ehp = p.e_hp + eb;
  const uint32_t* erec = p.e_rec + eb;
  // position of the i-th entry of this batch in the slot's entry arrays
  auto entry = [&](int i) {
    return i < s1 ? ob + i : (i < s2 ? o1 + i - s1 : (i < s3 ? o2 + i - s2 : oa + i - s3));
  };
  // a d = 3 record of b's list that also holds a was taken from a's list
  auto dup = [&](int i, uint64_t hm) { return i >= s2 && i < s3 && ((hm >> B.ia) & 1ull); };

  if (tid == 0) {
    S.inv_nv1 = S.nv[1] > 0 ? 1.0f / (float)S.nv[1] : 0.0f;
#pragma unroll
    for (int w = 0; w < NW; w++) S.kbase[w] = S.I[w];
    S.kbase[B.sa * NINT + (B.qa >> 6)] &= ~(1ull << (B.qa & 63));
    if (B.h == 2) S.kbase[B.sb * NINT + (B.qb >> 6)] &= ~(1ull << (B.qb & 63));
  }
  // zero the accumulator, the bans; row sums for H_aa
  if constexpr (MS) {
    for (int st = 0; st < nst; st++)
      for (int c = tid; c < B.nct; c += kThreads) A[st * mc + c] = 0.0;
  } else {
    for (int c = tid; c < B.nct; c += kThreads) {
      Alo[c] = 0ull;
      Ahi[c] = 0;
    }
  }
  for (int c = tid; c < (B.nct + 31) / 32; c += kThreads) ban[c] = 0u;
  {
    auto W = [&](int x, int sx, int y, int sy) {
      double v = p.Jm[x * norb + y];
      if (sx == sy) v -= p.Km[x * norb + y];
      return v;
    };
    if (B.kind == 0) {
      const int s = B.sa;
      for (int x = tid; x < S.nv[s]; x += kThreads) {
        const int r = S.vir[s][x];
        S.u0[x] = S.F[s][r] - W(r, s, B.qa, s);
      }
      if (tid == 0) S.base = S.hii - S.F[s][B.qa];
    } else {
      const int s1 = B.sa, s2 = B.sb;
      for (int x = tid; x < S.nv[s1]; x += kThreads) {
        const int r = S.vir[s1][x];
        S.u0[x] = S.F[s1][r] - W(r, s1, B.qa, s1) - W(r, s1, B.qb, s2);
      }
      if (B.kind == 2)
        for (int y = tid; y < S.nv[s2]; y += kThreads) {
          const int s = S.vir[s2][y];
          S.u1[y] = S.F[s2][s] - W(s, s2, B.qa, s1) - W(s, s2, B.qb, s2);
        }
      if (tid == 0) {
        S.base = S.hii - S.F[s1][B.qa] - S.F[s2][B.qb] + W(B.qa, s1, B.qb, s2);
        S.ibase = (B.qa * norb + B.qb) * norb * norb;
      }
      // pair tables of J = I: rows tri(qa, r) and columns tri(qb, s) with
      // the phases of qa -> r and qb -> s on I's strings
      const int sl2 = (B.kind == 2) ? 1 : s1;
      const int nva = S.nv[s1];
      for (int v = tid; v < nva + S.nv[sl2]; v += kThreads) {
        if (v < nva) {
          const int r = S.vir[s1][v];
          const int par = count_between<NINT>(S.I + s1 * NINT, r < B.qa ? r : B.qa, r < B.qa ? B.qa : r) & 1;
          S.iRow[v] = (E4 ? r : tri(B.qa, r)) | (par << 31);
        } else {
          const int sv = S.vir[sl2][v - nva];
          int par = count_between<NINT>(S.I + sl2 * NINT, sv < B.qb ? sv : B.qb, sv < B.qb ? B.qb : sv) & 1;
          if (B.kind == 1) {
            const int lo = sv < B.qb ? sv : B.qb, hi = sv < B.qb ? B.qb : sv;
            par ^= (B.qa > lo && B.qa < hi) ? 1 : 0;
          }
          S.iCol[v - nva] = (E4 ? sv : tri(B.qb, sv)) | (par << 31);
        }
      }
    }
  }
  __syncthreads();
  for (int x = tid; x < S.nv[B.sa]; x += kThreads) S.dx[x] = (p.e0 - S.base) - S.u0[x];
  if (p.tgt_on) {  // cells outside the target space contribute nothing: ban them
    for (int cc = tid; cc < B.nct; cc += kThreads) {
      int ro, so, x, y;
      cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
      const int kwr = B.sa * NINT + (ro >> 6), kws = (B.h == 2) ? B.sb * NINT + (so >> 6) : -1;
      bool ok = true;
      int moved = 0;
#pragma unroll
      for (int w = 0; w < NW; w++) {
        const uint64_t k = S.kbase[w] | (w == kwr ? 1ull << (ro & 63) : 0ull) | (w == kws ? 1ull << (so & 63) : 0ull);
        ok &= (k & p.tgt_core[w]) == p.tgt_core[w];
        ok &= (k & p.tgt_del[w]) == 0ull;
        moved += __popcll(k ^ p.tgt_ref[w]);
      }
      if (p.tgt_max_exc >= 0) ok &= (moved >> 1) <= p.tgt_max_exc;
      if (!ok) atomicOr(&ban[cc >> 5], 1u << (cc & 31));
    }
  }

  // ---- loop 1: bans.  J ranked before I that reach a whole row or column
  // of cells (two-hole batch, t = 1) flag it in rowm / colm; the flags are
  // turned into cell bans after the loop ----
  for (int x = tid; x < kMaxOrb; x += kThreads) {
    S.v.m.rowm[x] = 0u;
    S.v.m.colm[x] = 0u;
  }
  __syncthreads();
  bool dead = false;
  for (int c0 = 0; c0 < total; c0 += kChunk) {
    bool dl = false;
    const int c1 = min(c0 + kChunk, total);
    // each thread's next entry is loaded while it classifies the current one
    ulonglong2 enx = (c0 + tid < c1) ? ehp[entry(c0 + tid)] : make_ulonglong2(0ull, 0ull);
    for (int i = c0 + tid; i < c1; i += kThreads) {
      const ulonglong2 en = enx;
      if (i + kThreads < c1) enx = ehp[entry(i + kThreads)];
      const uint64_t hm = en.x, part = en.y;
      if (dup(i, hm)) continue;
      const int t = __popcll(hm & ~B.hm);
      if (t > 2) continue;
      if (part & kBeforeBit) {
        if ((B.h == 1 && t <= 1) || (B.h == 2 && t == 0)) {
          dl = true;
        } else if (B.h == 2 && t == 1) {
          int na_, nb_;
          const uint32_t Pa = particles_of_spin(part, norb, B.kind == 2 ? 0 : B.sa, &na_);
          for (int q = 0; q < na_; q++) S.v.m.rowm[S.vidx[B.kind == 2 ? 0 : B.sa][pk(Pa, q)]] = 1u;
          if (B.kind == 2) {
            const uint32_t Pb = particles_of_spin(part, norb, 1, &nb_);
            for (int q = 0; q < nb_; q++) S.v.m.colm[S.vidx[1][pk(Pb, q)]] = 1u;
          }
        } else {  // t == 2
          for_subset_cells<NINT, NT>(B, S, norb, part, [&](int c) { ban_cell(ban, B, c); });
        }
      } else if (t == 0 && hm == B.hm) {  // J = I - H + X with X a cell: alpha is internal
        int n0, n1, c;
        if (B.kind == 0) {
          const uint32_t P0 = particles_of_spin(part, norb, B.sa, &n0);
          c = S.vidx[B.sa][pk(P0, 0)];
        } else if (B.kind == 1) {
          const uint32_t P0 = particles_of_spin(part, norb, B.sa, &n0);
          c = pair_cell(S.vidx[B.sa][pk(P0, 0)], S.vidx[B.sa][pk(P0, 1)]);
        } else {
          const uint32_t P0 = particles_of_spin(part, norb, 0, &n0);
          const uint32_t P1 = particles_of_spin(part, norb, 1, &n1);
          c = S.vidx[0][pk(P0, 0)] * S.nv[1] + S.vidx[1][pk(P1, 0)];
        }
        ban_cell(ban, B, c);
      }
    }
    if (__syncthreads_or(dl)) {
      dead = true;
      break;
    }
  }
  if (dead) return;
  if (B.h == 2) {  // flagged rows and columns: one ban word per warp and round
    for (int c0 = 0; c0 < B.nct; c0 += kThreads) {
      const int cc = c0 + tid;
      bool bn = false;
      if (cc < B.nct) {
        int ro, so, x, y;
        cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
        bn = (S.v.m.rowm[x] | (B.kind == 2 ? S.v.m.colm[y] : S.v.m.rowm[y])) != 0u;
      }
      const unsigned bw = __ballot_sync(kFull, bn);
      if (lane == 0 && bw) ban[(c0 >> 5) + warp] |= bw;
    }
    // the flags as bit masks, kept through loop 2 (their storage is reused)
    static_assert(kWarps >= 2 * (kMaxOrb / 32), "one warp per mask word");
    if (warp < 2 * (kMaxOrb / 32)) {
      const int w = warp % (kMaxOrb / 32), x = 32 * w + lane;
      const unsigned f = __ballot_sync(kFull, (warp < kMaxOrb / 32 ? S.v.m.rowm[x] : S.v.m.colm[x]) != 0u);
      if (lane == 0) (warp < kMaxOrb / 32 ? S.frow : S.fcol)[w] = f;
    }
    __syncthreads();
  }

  // ---- loop 2: A(R) += c_J <J|H|I - H + R> over J ranked at or after I.
  // In the one-state form every term goes into the exact accumulator, so
  // the order in which J are listed and cells are reached does not matter ----
  unsigned long long con = 0;
  for (int c0 = 0; c0 < total; c0 += kChunk) {
    if (tid == 0) {
      S.n0 = 0;
      S.n1 = 0;
      S.n2 = 0;
      S.cnext = 0;
    }
    __syncthreads();
    const int c1 = min(c0 + kChunk, total);
    ulonglong2 enx = (c0 + tid < c1) ? ehp[entry(c0 + tid)] : make_ulonglong2(0ull, 0ull);
    for (int i = c0 + tid; i < c1; i += kThreads) {
      const ulonglong2 en = enx;
      const int o = entry(i);
      if (i + kThreads < c1) enx = ehp[entry(i + kThreads)];
      const uint64_t hmr = en.x, part = en.y;
      if (part & kBeforeBit) continue;
      if (dup(i, hmr)) continue;
      if (B.h == 2 && hmr == 0ull) continue;  // J = I: added in the cells pass
      const int t = __popcll(hmr & ~B.hm);
      if (t > 2) continue;
      const bool all = (B.h == 1) ? (t <= 1) : (t == 0);
      const int rec = (int)(erec[o] & 0x7FFFFFFFu);
      if (all) S.u.l.L0[atomicAdd(&S.n0, 1)] = rec;
      else if (t == 1) {
        if (row_live<NINT, NT>(B, S, norb, part)) S.u.l.L12[atomicAdd(&S.n1, 1)] = rec;
      }
      else if (subset_live<NINT, NT>(B, S, norb, part, ban)) S.u.l.L12[kChunk - 1 - atomicAdd(&S.n2, 1)] = rec;
    }
    __syncthreads();
    // J reaching every cell: the whole CTA, kGroup of them per pass.
    // In a two-hole batch such a J is K + {x1, x2}; for a cell R disjoint
    // from {x1, x2} the element is a double substitution x1 x2 -> R whose
    // pair indices and phase split into a row part and a column part,
    // precomputed once per J; the cells meeting the particles of J are single
    // substitutions of J and go to the row pass.
    const int n0 = S.n0;
    for (int g0 = 0; g0 < n0; g0 += kGroup) {
      const int m = min(kGroup, n0 - g0);
      if (tid < m) {
        const int r = S.u.l.L0[g0 + tid];
#pragma unroll
        for (int w = 0; w < NW; w++) S.gJw[tid][w] = rw[(size_t)r * NW + w];
        S.gcj[tid] = (NT)rc[r];
        if constexpr (MS)
          for (int st = 0; st < nst; st++) ms_gc[tid * kMaxStates + st] = rc[st * p.rc_stride + r];
        uint32_t xs, ts;
        int nxs, nts;
        const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
        excitation_sets<NINT, NT>(B, S, en.y, en.x, &xs, &nxs, &ts, &nts);
        S.gX[tid] = xs;
        S.gT[tid] = ts;
        S.gnx[tid] = nxs;
        S.gnt[tid] = nts;
        if (B.h == 2) {
          const int a = pk(xs, 0), bb = pk(xs, 1);
          const int x1 = a < bb ? a : bb, x2 = a < bb ? bb : a;
          S.gx1[tid] = x1;
          S.gx2[tid] = x2;
          const int s1 = x1 >= norb, s2 = x2 >= norb;
          S.gsr[tid] = S.vidx[s1][x1 - s1 * norb];
          S.gsc[tid] = S.vidx[s2][x2 - s2 * norb];
          S.gB[tid] = ((x1 - s1 * norb) * norb + (x2 - s2 * norb)) * norb * norb;
        }
      }
      __syncthreads();
      const int sl1 = B.sa, sl2 = (B.kind == 2) ? 1 : B.sa;
      const int nva = S.nv[sl1], nvb = S.nv[sl2];
      if (B.h == 2) {
        const int per = nva + nvb;
        for (int idx = tid; idx < m * per; idx += kThreads) {
          const int j = idx / per;
          const int v = idx - j * per;
          const uint64_t* Jw = S.gJw[j];
          const int x1 = S.gx1[j] - sl1 * norb, x2 = S.gx2[j] - sl2 * norb;
          if (v < nva) {
            const int r = S.vir[sl1][v];
            int par = 0;
            if (r != x1) par = count_between<NINT>(Jw + sl1 * NINT, r < x1 ? r : x1, r < x1 ? x1 : r) & 1;
            S.v.g.gRow[j][v] = (E4 ? r : tri(x1, r)) | (par << 31);
          } else {
            const int sv = S.vir[sl2][v - nva];
            int par = 0;
            if (sv != x2) par = count_between<NINT>(Jw + sl2 * NINT, sv < x2 ? sv : x2, sv < x2 ? x2 : sv) & 1;
            if (B.kind == 1) {
              const int lo = sv < x2 ? sv : x2, hi = sv < x2 ? x2 : sv;
              par ^= (x1 > lo && x1 < hi) ? 1 : 0;
            }
            S.v.g.gCol[j][v - nva] = (E4 ? sv : tri(x2, sv)) | (par << 31);
          }
        }
        __syncthreads();
      }
      for (int cc = tid; cc < B.nct; cc += kThreads) {
        if ((ban[cc >> 5] >> (cc & 31)) & 1u) continue;
        int ro, so, x, y;
        cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
        const int rcode = B.sa * norb + ro;
        const int scode = (B.h == 2) ? B.sb * norb + so : -1;
        unsigned long long acc_lo = 0ull;  // exact sum of this group's products
        int acc_hi = 0;
        double accs[kMaxStates];  // multi-state form: one sum per state
#pragma unroll
        for (int st = 0; st < kMaxStates; st++) accs[st] = 0.0;
        for (int j = 0; j < m; j++) {
          bool general = true;
          NT v = NT(0);
          if (B.h == 2) {
            const int sr = S.gsr[j], sc = S.gsc[j];
            if (B.kind == 2) {
              if (x != sr && y != sc) {
                const int rt = S.v.g.gRow[j][x], ct = S.v.g.gCol[j][y];
                v = flip_sign(eri_n[E4 ? S.gB[j] + (rt & 0x7fffffff) * norb + (ct & 0x7fffffff) : tri(rt & 0x7fffffff, ct & 0x7fffffff)],
                              (rt ^ ct) < 0);
                general = false;
              }
            } else if (x != sr && x != sc && y != sr && y != sc) {
              const int a1 = S.v.g.gRow[j][x], b2 = S.v.g.gCol[j][y];
              const int a2 = S.v.g.gRow[j][y], b1 = S.v.g.gCol[j][x];
              if constexpr (E4)
                v = eri_n[S.gB[j] + (a1 & 0x7fffffff) * norb + (b2 & 0x7fffffff)] - eri_n[S.gB[j] + (b2 & 0x7fffffff) * norb + (a1 & 0x7fffffff)];
              else
                v = eri_n[tri(a1 & 0x7fffffff, b2 & 0x7fffffff)] - eri_n[tri(a2 & 0x7fffffff, b1 & 0x7fffffff)];
              const int x2 = S.gx2[j] - B.sa * norb;
              const int lo = so < x2 ? so : x2, hi = so < x2 ? x2 : so;
              const int par = ((a1 ^ b2) < 0 ? 1 : 0) ^ ((ro > lo && ro < hi) ? 1 : 0);
              v = flip_sign(v, par);
              general = false;
            }
          }
          if (general) {
            // two-hole batch: a cell touching the particles of J is a single
            // substitution of J (or J itself, banned); those cells go by rows
            // in the row pass below, with every lane of a warp on a cell
            if (B.h == 2) continue;
            v = element<NINT, NT, E4>(eri_n, h_n, norb, S.gJw[j], S.gX[j], S.gnx[j], S.gT[j], S.gnt[j], rcode, scode);
          }
          con++;
          if constexpr (MS) {
#pragma unroll
            for (int st = 0; st < kMaxStates; st++)
              if (st < nst) accs[st] = fma(ms_gc[j * kMaxStates + st], (double)v, accs[st]);
          } else {
            unsigned long long l;
            int hh;
            fix_of(S.gcj[j] * v, F, l, hh);
            fix_add(acc_lo, acc_hi, l, hh);
          }
        }
        if constexpr (MS) {
#pragma unroll
          for (int st = 0; st < kMaxStates; st++)
            if (st < nst) A[st * mc + cc] += accs[st];
        } else {
          unsigned long long lo = Alo[cc];
          int hi = Ahi[cc];
          fix_add(lo, hi, acc_lo, acc_hi);
          Alo[cc] = lo;
          Ahi[cc] = hi;
        }
      }
      __syncthreads();
    }
    // J reaching a row of cells (one warp each; in a two-hole batch the J
    // reaching every cell come after them, for the cells touching their
    // particles), then J reaching a few cells (one lane each, 32 per draw),
    // drawn by the warps as they free up
    {
      const int n1 = S.n1 + (B.h == 2 ? n0 : 0), n2 = S.n2;
      for (;;) {
        int jd = 0;
        if (lane == 0) jd = atomicAdd(&S.cnext, 1);
        jd = __shfl_sync(kFull, jd, 0);
        if (jd < n1) {
          const int r = jd < S.n1 ? S.u.l.L12[jd] : S.u.l.L0[jd - S.n1];
          const uint64_t* Jw = rw + (size_t)r * NW;
          const NT cj = (NT)rc[r];
          double cjs[kMaxStates];
          if constexpr (MS) {
#pragma unroll
            for (int st = 0; st < kMaxStates; st++) cjs[st] = st < nst ? rc[st * p.rc_stride + r] : 0.0;
          }
          const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
          const uint64_t part = en.y;
          uint32_t X, T;
          int nx, nt;
          excitation_sets<NINT, NT>(B, S, part, en.x, &X, &nx, &T, &nt);
          for_row_cells<NINT, NT>(B, S, norb, part, lane, [&](int c, int pc, int zc) {
            const int cc = c - B.clo;
            if ((unsigned)cc >= (unsigned)B.nct || ((ban[cc >> 5] >> (cc & 31)) & 1u)) return;
            // holes of the substitution J -> alpha: X without the row's
            // particle; a double unless the other orbital is in X too or J
            // reaches every cell (then a single, by the general routine)
            bool zin = false;
            int u0 = -1, u1 = -1;
#pragma unroll
            for (int i = 0; i < 4; i++) {
              if (i >= nx) break;
              const int xc = pk(X, i);
              zin |= xc == zc;
              if (xc != pc) {
                if (u0 < 0) u0 = xc;
                else u1 = xc;
              }
            }
            NT v;
            if (nt == 1 && !zin && u1 >= 0)
              v = row_double<NINT, NT, E4>(eri_n, norb, Jw, u0 < u1 ? u0 : u1, u0 < u1 ? u1 : u0, pk(T, 0), zc);
            else
              v = element<NINT, NT, E4>(eri_n, h_n, norb, Jw, X, nx, T, nt, pc, zc);
            if constexpr (MS) {
#pragma unroll
              for (int st = 0; st < kMaxStates; st++)
                if (st < nst) atomicAdd(&A[st * mc + cc], cjs[st] * (double)v);
            } else {
              unsigned long long l;
              int hh;
              fix_of(cj * v, F, l, hh);
              fix_atomic_add(Alo, Ahi, cc, l, hh);
            }
            con++;
          });
        } else {
          const int j0 = (jd - n1) * 32;
          if (j0 >= n2) break;
          const int j = j0 + lane;
          if (j < n2) {
            const int r = S.u.l.L12[kChunk - 1 - j];
            const uint64_t* Jw = rw + (size_t)r * NW;
            const NT cj = (NT)rc[r];
            double cjs[kMaxStates];
            if constexpr (MS) {
#pragma unroll
              for (int st = 0; st < kMaxStates; st++) cjs[st] = st < nst ? rc[st * p.rc_stride + r] : 0.0;
            }
            const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
          const uint64_t part = en.y;
            uint32_t X, T;
            int nx, nt;
            excitation_sets<NINT, NT>(B, S, part, en.x, &X, &nx, &T, &nt);
            for_subset_cells<NINT, NT>(B, S, norb, part, [&](int c) {
              const int cc = c - B.clo;
              if ((unsigned)cc >= (unsigned)B.nct || ((ban[cc >> 5] >> (cc & 31)) & 1u)) return;
              int ro, so, x, y;
              cell_orbitals<NINT, NT>(B, S, c, &ro, &so, &x, &y);
              const int rcode = B.sa * norb + ro;
              const int scode = (B.h == 2) ? B.sb * norb + so : -1;
              if constexpr (MS) {
                const double v = (double)element<NINT, NT, E4>(eri_n, h_n, norb, Jw, X, nx, T, nt, rcode, scode);
#pragma unroll
                for (int st = 0; st < kMaxStates; st++)
                  if (st < nst) atomicAdd(&A[st * mc + cc], cjs[st] * v);
              } else {
                unsigned long long l;
                int hh;
                fix_of(cj * element<NINT, NT, E4>(eri_n, h_n, norb, Jw, X, nx, T, nt, rcode, scode), F, l, hh);
                fix_atomic_add(Alo, Ahi, cc, l, hh);
              }
              con++;
            });
          }
        }
      }
    }
    __syncthreads();
  }

  // ---- cells: the perturbers of I in this batch ----
  if (GRAD) {  // loop 2 is over: the pair tables' storage takes the weights
    for (int x = tid; x < kMaxOrb; x += kThreads) {
      S.v.w.rowW2[x] = 0.0;
      S.v.w.colW2[x] = 0.0;
    }
    __syncthreads();
  }
  if (p.k > 0) {
    if (S.tkcnt + B.nct > p.cap) compact_selection<NINT, NT>(p, S, te, ta, tk);
    if (tid == 0) {
      const unsigned long long gt = *((volatile unsigned long long*)p.tau_bits);
      if (gt > S.tau) S.tau = gt;
    }
    __syncthreads();
  }
  const unsigned long long tau = S.tau;
  double acc_e = 0.0, acc_s2 = 0.0;
  unsigned long long acc_na = 0, acc_d0 = 0, acc_d1 = 0, acc_min = 0x7FF0000000000000ull, acc_tiny = 0;
  double acc_es[kMaxStates], acc_s2s[kMaxStates];  // multi-state form: sums per state
#pragma unroll
  for (int st = 0; st < kMaxStates; st++) acc_es[st] = acc_s2s[st] = 0.0;
  if constexpr (MS) {
    for (int cc = tid; cc < B.nct; cc += kThreads) {
      if ((ban[cc >> 5] >> (cc & 31)) & 1u) continue;
      int ro, so, x, y;
      cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
      double vI = 0.0;  // <I|H|alpha> for the generator's own term
      if (B.h == 2) {
        const int a1 = S.iRow[x], b2 = S.iCol[y];
        if (B.kind == 2) {
          vI = (double)flip_sign(eri_n[E4 ? S.ibase + (a1 & 0x7fffffff) * norb + (b2 & 0x7fffffff) : tri(a1 & 0x7fffffff, b2 & 0x7fffffff)],
                                 (a1 ^ b2) < 0);
        } else {
          const int a2 = S.iRow[y], b1 = S.iCol[x];
          NT v;
          if constexpr (E4)
            v = eri_n[S.ibase + (a1 & 0x7fffffff) * norb + (b2 & 0x7fffffff)] - eri_n[S.ibase + (b2 & 0x7fffffff) * norb + (a1 & 0x7fffffff)];
          else
            v = eri_n[tri(a1 & 0x7fffffff, b2 & 0x7fffffff)] - eri_n[tri(a2 & 0x7fffffff, b1 & 0x7fffffff)];
          const int lo = so < B.qb ? so : B.qb, hi = so < B.qb ? B.qb : so;
          vI = (double)flip_sign(v, ((a1 ^ b2) < 0 ? 1 : 0) ^ ((ro > lo && ro < hi) ? 1 : 0));
        }
        con++;
      }
      // E0_s - H_aa = ((E0_s - base) - u0[x]) - rest, as the one-state form
      double rest = 0.0;
      if (B.kind == 2) rest = S.u1[y] + p.Jm[ro * norb + so];
      else if (B.kind == 1) rest = S.u0[y] + (p.Jm[ro * norb + so] - p.Km[ro * norb + so]);
      double crit = 0.0, a0 = 0.0;
#pragma unroll
      for (int st = 0; st < kMaxStates; st++) {
        if (st >= nst) break;
        const double a = A[st * mc + cc] + ms_cI[st] * vI;
        double D = (p.st_e0[st] - S.base) - S.u0[x];
        if (B.kind != 0) D -= rest;
        const unsigned long long dex = ((unsigned long long)__double_as_longlong(D) >> 52) & 0x7FFull;
        const double inv = (dex > 523ull && dex < 1523ull) ? recip_nr<2>(D) : 1.0 / D;
        const double q = a * inv;
        const double e = a * q;
        acc_es[st] += e;
        acc_s2s[st] += q * q;
        crit += ms_w[st] * e;  // c_alpha,s A_s / max_I c_Is^2
        const unsigned long long db = abs_bits(D);
        acc_min = db < acc_min ? db : acc_min;
        if (st == 0) a0 = a;
      }
      acc_na++;
      if (abs_bits(a0) < 0x3D06849B86A12B9Bull) acc_tiny++;
      uint64_t key[NW];
      const int kwr = B.sa * NINT + (ro >> 6), kws = (B.h == 2) ? B.sb * NINT + (so >> 6) : -1;
#pragma unroll
      for (int w = 0; w < NW; w++)
        key[w] = S.kbase[w] | (w == kwr ? 1ull << (ro & 63) : 0ull) | (w == kws ? 1ull << (so & 63) : 0ull);
      uint64_t hk = 0;
#pragma unroll
      for (int w = 0; w < NW; w++) hk = splitmix64(hk ^ key[w]);
      acc_d0 += hk;
      acc_d1 ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
      if (p.k > 0) {
        const unsigned long long eb = abs_bits(crit);
        if (eb >= tau) {
          atomicAdd(&p.sel_hist[sel_bin(eb)], 1u);
          const int pos = atomicAdd(&S.tkcnt, 1);
          te[pos] = crit;
          ta[pos] = a0;
#pragma unroll
          for (int w = 0; w < NW; w++) tk[(size_t)pos * NW + w] = key[w];
        }
      }
    }
    acc_e = acc_es[0];
    acc_s2 = acc_s2s[0];
  } else {
    for (int cc = tid; cc < B.nct; cc += kThreads) {
      if ((ban[cc >> 5] >> (cc & 31)) & 1u) continue;
      int ro, so, x, y;
      cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
      double a = fix_to_double(Alo[cc], Ahi[cc], F);
      if (B.h == 2) {  // the generator's own term c_I <I|H|alpha>
        NT v;
        const int a1 = S.iRow[x], b2 = S.iCol[y];
        if (B.kind == 2) {
          v = flip_sign(eri_n[E4 ? S.ibase + (a1 & 0x7fffffff) * norb + (b2 & 0x7fffffff) : tri(a1 & 0x7fffffff, b2 & 0x7fffffff)], (a1 ^ b2) < 0);
        } else {
          const int a2 = S.iRow[y], b1 = S.iCol[x];
          if constexpr (E4)
            v = eri_n[S.ibase + (a1 & 0x7fffffff) * norb + (b2 & 0x7fffffff)] - eri_n[S.ibase + (b2 & 0x7fffffff) * norb + (a1 & 0x7fffffff)];
          else
            v = eri_n[tri(a1 & 0x7fffffff, b2 & 0x7fffffff)] - eri_n[tri(a2 & 0x7fffffff, b1 & 0x7fffffff)];
          const int lo = so < B.qb ? so : B.qb, hi = so < B.qb ? B.qb : so;
          v = flip_sign(v, ((a1 ^ b2) < 0 ? 1 : 0) ^ ((ro > lo && ro < hi) ? 1 : 0));
        }
        a += (double)(S.cI * v);
        con++;
      }
      // D = E0 - H_aa from the per-batch row sums
      double D = S.dx[x];
      if (B.kind == 2) D -= S.u1[y] + p.Jm[ro * norb + so];
      else if (B.kind == 1) D -= S.u0[y] + (p.Jm[ro * norb + so] - p.Km[ro * norb + so]);
      // |D| in [2^-500, 2^500]: Newton reciprocal; otherwise the division
      const unsigned long long dex = ((unsigned long long)__double_as_longlong(D) >> 52) & 0x7FFull;
      const double inv = (dex > 523ull && dex < 1523ull) ? recip_nr<sizeof(NT) == 8 ? 2 : 1>(D) : 1.0 / D;
      const double q = a * inv;
      acc_e = fma(a, q, acc_e);  // e = A q
      acc_s2 += q * q;
      acc_na++;
      if (GRAD) {
        // numerator weight 2A/D for loop 3; (A/D)^2 weights the diagonal
        A[cc] = 2.0 * q;
        const double w2 = q * q;
        atomicAdd(&S.v.w.rowW2[x], w2);
        if (B.kind == 2) atomicAdd(&S.v.w.colW2[y], w2);
        if (B.kind == 1) atomicAdd(&S.v.w.rowW2[y], w2);
        if (B.h == 2) w_grad(p, ro, B.sa, so, B.sb, w2);
      }
      // |a| < 1e-14, compared on the bit pattern (no FP64 compare)
      if (abs_bits(a) < 0x3D06849B86A12B9Bull) acc_tiny++;
      // |D| and |e| as bit patterns, off the FP64 pipe
      const unsigned long long db = abs_bits(D);
      acc_min = db < acc_min ? db : acc_min;
      uint64_t key[NW];  // alpha's words; selects keep them in registers
      const int kwr = B.sa * NINT + (ro >> 6), kws = (B.h == 2) ? B.sb * NINT + (so >> 6) : -1;
#pragma unroll
      for (int w = 0; w < NW; w++)
        key[w] = S.kbase[w] | (w == kwr ? 1ull << (ro & 63) : 0ull) | (w == kws ? 1ull << (so & 63) : 0ull);
      uint64_t hk = 0;
#pragma unroll
      for (int w = 0; w < NW; w++) hk = splitmix64(hk ^ key[w]);
      acc_d0 += hk;
      acc_d1 ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
      // e = A q is formed only when it can reach the threshold: with biased
      // exponents ea, eq of A and q, |A q| < 2^(ea + eq - 2044), so
      // ea + eq <= et + 1021 (et: the exponent of tau) puts it below tau
      const int ea = (int)(abs_bits(a) >> 52), eqx = (int)(abs_bits(q) >> 52);
      if (p.k > 0 && (tau == 0ull || ea + eqx > (int)(tau >> 52) + 1021)) {
        const double e = a * q;
        const unsigned long long eb = abs_bits(e);
        if (eb >= tau) {
          atomicAdd(&p.sel_hist[sel_bin(eb)], 1u);
          const int pos = atomicAdd(&S.tkcnt, 1);
          te[pos] = e;
          ta[pos] = a;
#pragma unroll
          for (int w = 0; w < NW; w++) tk[(size_t)pos * NW + w] = key[w];
        }
      }
    }
  }
  // ---- per-item reduction into the generator's totals ----
  {
    // FP64 sums through shared memory and one warp: a shuffle tree in every
    // warp would spend five FP64 adds per lane per quantity
    S.u.red_t[0][tid] = acc_e;
    S.u.red_t[1][tid] = acc_s2;
    const unsigned long long na = warp_sum_u(acc_na), nc = warp_sum_u(con), d0 = warp_sum_u(acc_d0);
    const unsigned long long d1 = warp_xor_u(acc_d1), mn = warp_min_u(acc_min), tiny = warp_sum_u(acc_tiny);
    if (lane == 0) {
      S.red_u[warp][0] = na;
      S.red_u[warp][1] = nc;
      S.red_u[warp][2] = d0;
      S.red_u[warp][3] = d1;
      S.red_u[warp][4] = mn;
      S.red_u[warp][5] = tiny;
    }
    __syncthreads();
    double se = 0.0, ss = 0.0;
    if (warp == 0) {
      for (int i = lane; i < kThreads; i += 32) {
        se += S.u.red_t[0][i];
        ss += S.u.red_t[1][i];
      }
      se = warp_sum(se);
      ss = warp_sum(ss);
    }
    if (tid == 0) {
      const double te_ = se, ts = ss;
      unsigned long long tn = 0, tc = 0, x0 = 0, x1 = 0, m = 0x7FF0000000000000ull, tt = 0;
      for (int w = 0; w < kWarps; w++) {
        tn += S.red_u[w][0];
        tc += S.red_u[w][1];
        x0 += S.red_u[w][2];
        x1 ^= S.red_u[w][3];
        m = S.red_u[w][4] < m ? S.red_u[w][4] : m;
        tt += S.red_u[w][5];
      }
      S.sw2 = ts;
      // the item's FP64 sums go to its own slot; the generator's eps_I
      // and sum A^2/D^2 are reduced from the slots in item order after the
      // wave (reduce_items_kernel), so they do not depend on which CTA
      // finished first
      double* its = p.it_sum + ((size_t)slot * nper + j) * p.it_stride;
      its[0] = te_;
      its[1] = ts;
      if (tn) {
        atomicAdd(&p.na[g], tn);
        atomicAdd(&p.ncon[g], tc);
        atomicAdd(&p.digest[0], x0);
        atomicXor(&p.digest[1], x1);
        atomicMin(p.min_den_bits, m);
        if (tt) atomicAdd(p.n_tiny, tt);
      }
    }
    if constexpr (MS) {  // the other states' eps and s2, one at a time
#pragma unroll
      for (int st = 1; st < kMaxStates; st++) {
        if (st >= nst) break;
        __syncthreads();
        S.u.red_t[0][tid] = acc_es[st];
        S.u.red_t[1][tid] = acc_s2s[st];
        __syncthreads();
        if (warp == 0) {
          double ue = 0.0, us = 0.0;
          for (int i = lane; i < kThreads; i += 32) {
            ue += S.u.red_t[0][i];
            us += S.u.red_t[1][i];
          }
          ue = warp_sum(ue);
          us = warp_sum(us);
          if (lane == 0) {
            double* its = p.it_sum + ((size_t)slot * nper + j) * p.it_stride;
            its[2 * st] = ue;
            its[2 * st + 1] = us;
          }
        }
      }
    }
  }
  if (GRAD) {
    __syncthreads();
    // ---- loop 3: c_J (2A/D) d<J|H|alpha> over the same (J, cell) pairs ----
    for (int c0 = 0; c0 < total; c0 += kChunk) {
      if (tid == 0) {
        S.n0 = 0;
        S.n1 = 0;
        S.n2 = 0;
        S.cnext = 0;
      }
      __syncthreads();
      const int c1 = min(c0 + kChunk, total);
      for (int i = c0 + tid; i < c1; i += kThreads) {
        const int o = entry(i);
        const ulonglong2 en = ehp[o];
        const uint64_t hmr = en.x, part = en.y;
        if (part & kBeforeBit) continue;
        if (dup(i, hmr)) continue;
        const int t = __popcll(hmr & ~B.hm);
        if (t > 2) continue;
        const bool all = (B.h == 1) ? (t <= 1) : (t == 0);
        const int rec = (int)(erec[o] & 0x7FFFFFFFu);
        if (all) S.u.l.L0[atomicAdd(&S.n0, 1)] = rec;
        else if (t == 1) {
          if (row_live<NINT, NT>(B, S, norb, part)) S.u.l.L12[atomicAdd(&S.n1, 1)] = rec;
        }
        else if (subset_live<NINT, NT>(B, S, norb, part, ban)) S.u.l.L12[kChunk - 1 - atomicAdd(&S.n2, 1)] = rec;
      }
      __syncthreads();
      for (int j = 0; j < S.n0; j++) {
        const int r = S.u.l.L0[j];
        const uint64_t* Jw = rw + (size_t)r * NW;
        const double cj = rc[r];
        uint32_t X, T;
        int nx, nt;
        const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
        excitation_sets<NINT, NT>(B, S, en.y, en.x, &X, &nx, &T, &nt);
        for (int cc = tid; cc < B.nct; cc += kThreads) {
          if ((ban[cc >> 5] >> (cc & 31)) & 1u) continue;
          int ro, so, x, y;
          cell_orbitals<NINT, NT>(B, S, B.clo + cc, &ro, &so, &x, &y);
          element_grad<NINT>(p.g_dh, p.g_deri, norb, Jw, X, nx, T, nt, B.sa * norb + ro, (B.h == 2) ? B.sb * norb + so : -1, cj * A[cc]);
        }
      }
      {  // row-reaching J (a warp each), then subset-reaching J (32 per draw), drawn dynamically
        const int n1 = S.n1, n2 = S.n2;
        for (;;) {
          int jd = 0;
          if (lane == 0) jd = atomicAdd(&S.cnext, 1);
          jd = __shfl_sync(kFull, jd, 0);
          if (jd < n1) {
            const int j = jd;
            const int r = S.u.l.L12[j];
            const uint64_t* Jw = rw + (size_t)r * NW;
            const double cj = rc[r];
            const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
          const uint64_t part = en.y;
            uint32_t X, T;
            int nx, nt;
            excitation_sets<NINT, NT>(B, S, part, en.x, &X, &nx, &T, &nt);
            for_row_cells<NINT, NT>(B, S, norb, part, lane, [&](int c, int pc, int zc) {
              const int cc = c - B.clo;
              if ((unsigned)cc >= (unsigned)B.nct || ((ban[cc >> 5] >> (cc & 31)) & 1u)) return;
              element_grad<NINT>(p.g_dh, p.g_deri, norb, Jw, X, nx, T, nt, pc, zc, cj * A[cc]);
            });
          } else {
            const int j0 = (jd - n1) * 32;
            if (j0 >= n2) break;
            const int j = j0 + lane;
            if (j < n2) {
              const int r = S.u.l.L12[kChunk - 1 - j];
              const uint64_t* Jw = rw + (size_t)r * NW;
              const double cj = rc[r];
              const ulonglong2 en = make_ulonglong2(rhm[r], rpt[r]);
          const uint64_t part = en.y;
              uint32_t X, T;
              int nx, nt;
              excitation_sets<NINT, NT>(B, S, part, en.x, &X, &nx, &T, &nt);
              for_subset_cells<NINT, NT>(B, S, norb, part, [&](int c) {
                const int cc = c - B.clo;
                if ((unsigned)cc >= (unsigned)B.nct || ((ban[cc >> 5] >> (cc & 31)) & 1u)) return;
                int ro, so, x, y;
                cell_orbitals<NINT, NT>(B, S, c, &ro, &so, &x, &y);
                element_grad<NINT>(p.g_dh, p.g_deri, norb, Jw, X, nx, T, nt, B.sa * norb + ro, (B.h == 2) ? B.sb * norb + so : -1,
                                   cj * A[cc]);
              });
            }
          }
        }
      }
      __syncthreads();
    }
    // ---- diagonal: H_aa = H_II - F(a) [- F(b) + W(a,b)] + F(r) [+ F(s)]
    //      - W(r,a) [- W(r,b) - W(s,a) - W(s,b) + W(r,s)]; the W(r,s) terms
    //      were scattered per cell, the rest goes by row sums ----
    double* wF = p.g_wF + (size_t)g * 2 * norb;
    const int s1 = B.sa, s2 = (B.h == 2) ? B.sb : B.sa;
    for (int x = tid; x < S.nv[s1]; x += kThreads) {
      const double wr = S.v.w.rowW2[x];
      if (wr == 0.0) continue;
      const int r = S.vir[s1][x];
      atomicAdd(&wF[s1 * norb + r], wr);
      w_grad(p, r, s1, B.qa, B.sa, -wr);
      if (B.h == 2) w_grad(p, r, s1, B.qb, B.sb, -wr);
    }
    if (B.kind == 2)
      for (int y = tid; y < S.nv[s2]; y += kThreads) {
        const double wc = S.v.w.colW2[y];
        if (wc == 0.0) continue;
        const int sv = S.vir[s2][y];
        atomicAdd(&wF[s2 * norb + sv], wc);
        w_grad(p, sv, s2, B.qa, B.sa, -wc);
        w_grad(p, sv, s2, B.qb, B.sb, -wc);
      }
    if (tid == 0 && S.sw2 != 0.0) {
      const double sw = S.sw2;
      atomicAdd(&p.g_wH[g], sw);
      atomicAdd(&wF[B.sa * norb + B.qa], -sw);
      if (B.h == 2) {
        atomicAdd(&wF[B.sb * norb + B.qb], -sw);
        w_grad(p, B.qa, B.sa, B.qb, B.sb, sw);
      }
    }
  }
}

// Three CTAs per SM for one word per spin; two words per spin come with
// larger accumulators (at most two CTAs fit in shared memory), so those
// kernels take the registers of two CTAs and do not spill.
//
// MS = true: the multi-state form (several states at once, FP64 only).
// Each state s has its own accumulator A_s (dynamic shared memory, one
// stride of max_cells each); a (J, cell) element is formed once and added
// with c_Js to every A_s.  The cells pass forms e_s = A_s^2/(E0_s - H_aa)
// for every state, sums each into its own eps and s2, and offers the
// determinant to the selection with the criterion sum_s w_s e_s,
// w_s = 1/max_I c_Is^2 (Sec. "Selected CI", the criterion of Angeli et al.).
template <int NINT, typename NT, bool GRAD = false, bool MS = false, bool E4 = true>
__global__ void __launch_bounds__(kThreads, (NINT == 1) ? 3 : 2) batch_kernel(const __grid_constant__ SweepParams p) {
  static_assert(!(MS && GRAD), "the gradient is a one-state form");
  static_assert(!MS || sizeof(NT) == 8, "the multi-state form is FP64");
  constexpr int NW = 2 * NINT;
  __shared__ BatchShared<NINT, NT> S;
  const int tid = threadIdx.x;
  const long long nitems = (long long)p.wave_slots * p.nper;
  double* te = p.tk_e + (size_t)blockIdx.x * (size_t)p.cap;
  double* ta = p.tk_a + (size_t)blockIdx.x * (size_t)p.cap;
  uint64_t* tk = p.tk_key + (size_t)blockIdx.x * (size_t)p.cap * NW;
  const ItemEnv E = item_env<MS>(p);
  const NT* eri_n = numer_eri<NT, E4>(p);
  const NT* h_n = numer_h<NT>(p);

  if (tid == 0) {
    S.tkcnt = p.tk_cnt[blockIdx.x];
    S.tau = p.tk_tau[blockIdx.x];
    S.slot = -1;
    S.inext = S.iend = 0;
    if (p.timeout_ns) atomicCAS(p.t_start, 0ull, global_ns());
  }
  const int F = MS ? 0 : fix_scale(p);  // fixed-point scale of A_alpha (units of 2^-F)

  for (;;) {
    __syncthreads();
    if (tid == 0) {  // the next work item: p.chunk of them per draw from the queue
      if (S.inext >= S.iend) {
        const long long b0 = atomicAdd(p.queue, p.chunk);
        S.inext = b0;
        S.iend = b0 + p.chunk;
      }
      S.item = S.inext++;
      if (p.timeout_ns && global_ns() - *((volatile unsigned long long*)p.t_start) > p.timeout_ns) {
        atomicOr(p.err, 128);  // watchdog: stop taking work, report the timeout
        S.item = nitems;
      }
    }
    __syncthreads();
    const long long item = S.item;
    if (item >= nitems) break;
    batch_item<NINT, NT, GRAD, MS, E4>(p, S, item, F, te, ta, tk, E, eri_n, h_n);
  }
  if (p.k > 0 && p.last_wave) compact_selection<NINT, NT>(p, S, te, ta, tk);
  __syncthreads();
  if (tid == 0) {
    p.tk_cnt[blockIdx.x] = S.tkcnt;
    p.tk_tau[blockIdx.x] = S.tau;
  }
}

// The work items of one wave of several instances' sweeps (one word count
// and precision): the wave's pieces (instance, run of generator slots) one
// after another, each piece's items from its own queue, `m.chunk` per draw.
// A CTA moves to the next piece when the current one's queue is empty; it
// stores its selection state (candidate count and threshold) for the
// instance it leaves and loads the state of the one it enters.  The dynamic
// shared memory is sized for the largest accumulator of the instances.
// Every instance has its own candidate buffers for each CTA of the launch;
// they are compacted to k entries by compact_multi_kernel after the last
// wave.
template <int NINT, typename NT>
__global__ void __launch_bounds__(kThreads, (NINT == 1) ? 3 : 2) batch_multi_kernel(const __grid_constant__ MultiWaveInline m) {
  constexpr int NW = 2 * NINT;
  __shared__ BatchShared<NINT, NT> S;
  const int tid = threadIdx.x;
  if (tid == 0 && m.timeout_ns) atomicCAS(m.t_start, 0ull, global_ns());
  bool stop = false;
  // the pieces one after another, each from its own queue: the piece index
  // is the same in every thread, so its parameters are read like a single
  // sweep's
#pragma unroll 1
  for (int pc = 0; pc < m.n && !stop; pc++) {
    const SweepParams& p = m.ps[pc];
    const long long nitems = m.item_ofs[pc + 1] - m.item_ofs[pc];
    __syncthreads();
    if (tid == 0) {
      S.tkcnt = p.tk_cnt[blockIdx.x];
      S.tau = p.tk_tau[blockIdx.x];
      S.slot = -1;
      S.inext = S.iend = 0;
    }
    const int F = fix_scale(p);
    const ItemEnv E = item_env<false>(p);
    double* te = p.tk_e + (size_t)blockIdx.x * (size_t)p.cap;
    double* ta = p.tk_a + (size_t)blockIdx.x * (size_t)p.cap;
    uint64_t* tk = p.tk_key + (size_t)blockIdx.x * (size_t)p.cap * NW;
    for (;;) {
      __syncthreads();
      if (tid == 0) {
        if (S.inext >= S.iend) {
          const long long b0 = (long long)atomicAdd(m.queue + pc, (unsigned long long)m.chunk);
          S.inext = b0;
          S.iend = b0 + m.chunk;
        }
        S.item = S.inext++;
        if (m.timeout_ns && global_ns() - *((volatile unsigned long long*)m.t_start) > m.timeout_ns) {
          atomicOr(m.err, 128);  // watchdog: stop taking work, report the timeout
          S.item = -1;
        }
      }
      __syncthreads();
      const long long item = S.item;
      if (item < 0) stop = true;
      if (item < 0 || item >= nitems) break;
      batch_item<NINT, NT, false, false, true>(p, S, item, F, te, ta, tk, E, numer_eri<NT, true>(p), numer_h<NT>(p));
    }
    __syncthreads();
    if (tid == 0) {
      p.tk_cnt[blockIdx.x] = S.tkcnt;
      p.tk_tau[blockIdx.x] = S.tau;
    }
  }
}

// After the last wave: CTA buffer blockIdx.x of instance blockIdx.y keeps its
// k best candidates (as the last wave of a single sweep does).
template <int NINT, typename NT>
__global__ void __launch_bounds__(kThreads) compact_multi_kernel(const SweepParams* __restrict__ ps) {
  constexpr int NW = 2 * NINT;
  __shared__ BatchShared<NINT, NT> S;
  const SweepParams& p = ps[blockIdx.y];
  if (p.k <= 0) return;
  if (threadIdx.x == 0) {
    S.tkcnt = p.tk_cnt[blockIdx.x];
    S.tau = p.tk_tau[blockIdx.x];
  }
  compact_selection<NINT, NT>(p, S, p.tk_e + (size_t)blockIdx.x * (size_t)p.cap,
                              p.tk_a + (size_t)blockIdx.x * (size_t)p.cap,
                              p.tk_key + (size_t)blockIdx.x * (size_t)p.cap * NW);
  __syncthreads();
  if (threadIdx.x == 0) {
    p.tk_cnt[blockIdx.x] = S.tkcnt;
    p.tk_tau[blockIdx.x] = S.tau;
  }
}

// Launch helpers of the multi-instance batch kernels, instantiated for FP64
// in sweep.cu and for the mixed form in sweep_mixed.cu (the prep kernel is
// launched from sweep.cu only).
template <typename NT>
static cudaError_t multi_wave_launch(int nint, const MultiWaveInline& m, int total_slots, int grid, size_t smem,
                                     cudaStream_t st) {
  if (total_slots <= 0) return cudaSuccess;
  if (nint == 1) {
    cudaFuncSetAttribute(batch_multi_kernel<1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_multi_kernel<1, NT><<<grid, kThreads, smem, st>>>(m);
  } else {
    cudaFuncSetAttribute(batch_multi_kernel<2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    batch_multi_kernel<2, NT><<<grid, kThreads, smem, st>>>(m);
  }
  return cudaGetLastError();
}

template <typename NT>
static cudaError_t multi_compact_launch(int nint, const SweepParams* ps, int n, int grid, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  if (nint == 1) compact_multi_kernel<1, NT><<<dim3(grid, n), kThreads, 0, st>>>(ps);
  else compact_multi_kernel<2, NT><<<dim3(grid, n), kThreads, 0, st>>>(ps);
  return cudaGetLastError();
}

template <typename NT>
static int multi_blocks_per_sm(int nint, size_t smem) {
  int n = 0;
  if (nint == 1) {
    cudaFuncSetAttribute(batch_multi_kernel<1, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_multi_kernel<1, NT>, kThreads, smem);
  } else {
    cudaFuncSetAttribute(batch_multi_kernel<2, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, batch_multi_kernel<2, NT>, kThreads, smem);
  }
  return n;
}

// Per generator: wH * dH_II + sum_{s,x} wF[s][x] * dF^I_s(x), with
// F^I_s(x) = h_xx + sum_{j in I} W(x, j) and H_II = sum_i h_ii + sum_{i<j} W(i, j).
template <int NINT>
__global__ void __launch_bounds__(kThreads) grad_gen_kernel(const __grid_constant__ SweepParams p) {
  constexpr int NW = 2 * NINT;
  __shared__ int s_occ[kMaxElec];
  const int g = blockIdx.x, tid = threadIdx.x, norb = p.norb, nel = p.nel;
  const double wH = p.g_wH[g];
  const double* wF = p.g_wF + (size_t)g * 2 * norb;
  const uint64_t* I = p.dets + (size_t)p.order[g] * NW;
  if (tid == 0) {
    int n = 0;
    for (int s = 0; s < 2; s++)
      for (int q = 0; q < norb; q++)
        if ((I[s * NINT + (q >> 6)] >> (q & 63)) & 1ull) s_occ[n++] = s * norb + q;
  }
  __syncthreads();
  if (wH != 0.0)
    for (int ij = tid; ij < nel * nel; ij += kThreads) {
      const int i = ij / nel, j = ij - i * nel;
      const int ci = s_occ[i], si = ci >= norb, qi = ci - si * norb;
      if (i == j) atomicAdd(&p.g_dh[qi * norb + qi], wH);
      else if (i < j) {
        const int cj = s_occ[j], sj = cj >= norb, qj = cj - sj * norb;
        w_grad(p, qi, si, qj, sj, wH);
      }
    }
  for (int x = tid; x < 2 * norb; x += kThreads) {
    const double w = wF[x];
    if (w == 0.0) continue;
    const int s = x / norb, q = x - s * norb;
    atomicAdd(&p.g_dh[q * norb + q], w);
    for (int i = 0; i < nel; i++) {
      const int c = s_occ[i], sj = c >= norb, j = c - sj * norb;
      atomicAdd(&p.g_deri[eri_index(q, q, j, j)], w);
      if (sj == s) atomicAdd(&p.g_deri[eri_index(q, j, j, q)], -w);
    }
  }
}

}  // namespace qp
