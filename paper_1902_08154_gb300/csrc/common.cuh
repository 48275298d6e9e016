// common.cuh -- device helpers and launch parameters of the sm_103a EN-PT2
// sweep (Quantum Package 2.0, arXiv:1902.08154).  Internal to the library.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

struct qp_pt2_ctx;

namespace qp {

constexpr int kMaxOrb = 128;
constexpr int kMaxElec = 64;   // per determinant (both spins); hole masks are uint64
constexpr int kMaxBatch = kMaxElec + kMaxElec * (kMaxElec - 1) / 2;
constexpr int kSelBins = 1024;  // |e| histogram: 128 binary exponents (2^-100 .. 2^27) x 8 sub-bins
constexpr int kMaxStates = 4;   // states of one multi-state sweep

// Fold of splitmix64 over the key words: the digest hash of a determinant.
// splitmix64 is the generator of Steele, Lea & Flood (2014); its finaliser
// constants are those of Vigna's public reference implementation.
__host__ __device__ inline uint64_t splitmix64(uint64_t x) {
  x += 0x9E3779B97F4A7C15ull;
  x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
  x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
  return x ^ (x >> 31);
}

// Compound triangular index of Algorithm hash (0-based).
__device__ __forceinline__ int tri(int a, int b) {
  int hi = a > b ? a : b, lo = a > b ? b : a;
  return hi * (hi + 1) / 2 + lo;
}

__device__ __forceinline__ int eri_index(int p, int q, int r, int s) {
  return tri(tri(p, q), tri(r, s));
}

// Four-index layout of the integrals for the sweep's numerator gathers:
// (pq|rs) at ((p * norb + r) * norb + q) * norb + s, so that the integrals
// (pq|rs) of a fixed pair (p, r) form one norb x norb slab, row q, column s.
// The cells of a batch vary q and s over the virtual orbitals with (p, r)
// fixed (two holes, or a J's two particles), so a warp reads consecutive s
// of one row.  norb^4 entries (below 2^31 for norb <= 128).
__device__ __forceinline__ int eri4_index(int p, int q, int r, int s, int norb) {
  return ((p * norb + r) * norb + q) * norb + s;
}

// Number of set bits of the spin string sw (NINT words) strictly between
// orbitals lo < hi: the masked popcount that gives a single substitution's
// phase (Sec. "Internal representation of determinants").
template <int NINT>
__device__ __forceinline__ int count_between(const uint64_t* sw, int lo, int hi) {
  int a = lo + 1, b = hi, n = 0;
#pragma unroll
  for (int w = 0; w < NINT; w++) {
    int l = a - 64 * w, u = b - 64 * w;
    l = l < 0 ? 0 : l;
    u = u > 64 ? 64 : u;
    if (l < u) {
      uint64_t m = (u == 64 ? ~0ull : ((1ull << u) - 1)) & ~((1ull << l) - 1);
      n += __popcll(sw[w] & m);
    }
  }
  return n;
}

// What the Hamiltonian/Davidson unit needs of a context (filled by
// qp_pt2.cu, which owns the context), and the library's error reporter.
struct CtxView {
  int norb, nalpha, nbeta, nint, nel, device;
  const double *h, *eri, *Jm, *Km;  // device copies, [norb*norb] and packed
  cudaStream_t st;
};
int ctx_view(const struct ::qp_pt2_ctx* x, CtxView* v);
int report(int code, const char* msg);

// Bucket entries per coarse-filter record: a record with holes Q of I
// (d = |Q|) is listed once in the shared bucket (d <= 2), once per hole
// (d = 3) or once per pair of holes (d = 4).
__host__ __device__ inline long long bucket_entries_per_record(int nel) {
  return nel >= 4 ? 6 : (nel == 3 ? 3 : 1);
}

// Dynamic shared memory of the one-state batch kernel for mc cells: A_alpha
// as a 96-bit integer per cell (a 64-bit low word and a 32-bit high word; the
// exact accumulation in sweep_impl.cuh) and one ban bit per cell.
__host__ __device__ inline size_t sweep_smem(int mc) {
  const size_t m = (size_t)(mc < 1 ? 1 : mc);
  return 8 * m + 4 * ((m + 1) & ~(size_t)1) + 4 * ((m + 31) / 32);
}

struct GenMeta;
// Device bytes per generator slot of a wave: metadata, nd coarse-filter
// records (words, nst coefficients, hole mask, particles, flag), bucket
// offsets, ent_cap self-contained entries (20 bytes), the dead-batch bits and
// the nper items' FP64 sums (2 per state).
inline size_t wave_slot_bytes(size_t meta_bytes, int nel, int nbat, int nw, size_t nd, int nst, int nper) {
  const size_t ent_cap = nd * (size_t)bucket_entries_per_record(nel);
  return meta_bytes + nd * (8 * (size_t)nw + 8 * (size_t)nst + 8 + 8 + 4) + 4 * (size_t)(nbat + 2) + 20 * ent_cap +
         4 * (size_t)((nbat + 31) / 32) + 16 * (size_t)nper * (size_t)nst;
}

// Per-generator data built by the prep kernel and read by the batch kernel.
struct GenMeta {
  uint64_t I[4];            // generator determinant (2*NINT words used)
  int g;                    // rank of the generator (-1: empty slot)
  int nrec;                 // coarse-filter records
  double hii;               // <I|H|I>
  double cI;                // c_I
  int occ[kMaxElec];        // spin-orbital codes s*norb+q of I, ordered
  double F[2][kMaxOrb];     // Fock diagonal of I
};

struct SweepParams {
  int norb, nalpha, nbeta, nel, nbat;
  // ntile > 1: every opposite-spin two-hole batch is split into ntile work
  // items over consecutive blocks of ceil(nv_up / ntile) rows (so that its
  // accumulator fits, or fits more than once, in an SM's shared memory);
  // nper = work items per generator = nbat + (ntile - 1) n_alpha n_beta
  int ntile, nper;
  // work items taken from the queue per draw (>= 1)
  int chunk;
  // watchdog: with timeout_ns > 0 a CTA stops taking work items once
  // timeout_ns nanoseconds (device global timer) have passed since *t_start,
  // the time the first CTA of the call started, and sets error flag 128
  unsigned long long timeout_ns;
  unsigned long long* t_start;
  int64_t ndet;
  const uint64_t* dets;   // [ndet][2][NINT]
  const double* coefs;    // [ndet]
  const int32_t* order;   // det index by rank
  const int32_t* rank_of; // rank by det index
  const double* h;        // [norb*norb]
  const double* eri;      // packed
  const float* h32;       // FP32 copies for the mixed-precision numerator (NULL in FP64 mode)
  const float* eri32;
  const double* eri4;     // [norb^4] four-index layout (eri4_index) of the batch kernel's gathers
  const float* eri4_32;   // its FP32 copy (mixed precision; NULL in FP64 mode)
  int mixed;              // 1: numerator gathers and products in FP32
  const double* Jm;       // [norb*norb] (pp|qq)
  const double* Km;       // [norb*norb] (pq|qp)
  double e0;
  int shard_index, shard_count;   // generators of rank shard_index + t*shard_count
  const int32_t* gen_list;        // if set: the generator of slot t has rank gen_list[t]
  // target space: alpha must hold every core spin orbital, no deleted one,
  // and (tgt_max_exc >= 0) at most tgt_max_exc electrons moved from tgt_ref
  int tgt_on, tgt_max_exc;
  uint64_t tgt_ref[4], tgt_core[4], tgt_del[4];
  // several states (nst > 1, multi-state batch kernel only): state s has its
  // coefficients at coefs + s*ndet, its records' coefficients at
  // r_coef + s*rc_stride, its E0 in st_e0[s], its per-generator sums at
  // eps + s*ndet and s2 + s*ndet; st_cmax[s] holds the bits of max_I |c_Is|
  int nst;
  int64_t rc_stride;
  double st_e0[kMaxStates];
  const unsigned long long* st_cmax;

  // wave of generator slots
  int wave_start;                 // first generator position (t) of this wave
  int wave_slots;                 // slots in this wave
  int last_wave;                  // 1 on the last wave: final selection compaction
  int* queue;                     // per-wave item counter

  // per-slot data (capacity ndet records, ent_cap bucket entries)
  GenMeta* meta;                  // [slots]
  uint64_t* r_words;              // [slots][ndet][2*NINT]
  double* r_coef;                 // [slots][ndet]
  uint64_t* r_hmask;              // [slots][ndet]  holes of I missing from J (occupied index bits)
  uint64_t* r_part;               // [slots][ndet]  up to 4 particle codes of J outside I, 16 bits each
  uint32_t* r_flag;               // [slots][ndet]  bit 0: rank(J) < rank(I)
  int* b_ofs;                     // [slots][nbat + 2]  bucket offsets (bucket nbat: J within degree 2)
  // bucket entries, self-contained so that the batch kernel classifies a
  // bucket by streaming it: the record's hole mask and particle codes, and
  // its index with the rank flag (rank(J) < rank(I)) in bit 31
  ulonglong2* e_hp;               // [slots][ent_cap]: hole mask, particles (one 16-byte load)
  uint32_t* e_rec;                // [slots][ent_cap]
  uint32_t* b_dead;               // [slots][(nbat + 31) / 32]  batches banned as a whole
  int64_t ent_cap;

  // exact accumulation of A_alpha: bits of max_I |c_I| (written by the
  // validation) and of max |h_pq| and max |(pq|rs)| (the context's), from
  // which every CTA derives the same fixed-point scale
  const unsigned long long* cmax_bits;
  const unsigned long long* hmax_bits;  // [2]: max |h|, max |eri|

  // per-item sums of the wave, reduced per generator in a fixed order:
  // it_sum[(slot * nper + item) * it_stride + 2 s + {0, 1}] = (e, A^2/D^2)
  // of state s
  double* it_sum;
  int it_stride;

  // per-generator outputs, by rank
  double* eps;
  double* s2;
  unsigned long long* na;
  unsigned long long* ncon;
  // global accumulators
  unsigned long long* digest;       // [2]
  unsigned long long* min_den_bits; // bits of min |D| (non-negative double)
  unsigned long long* n_tiny;

  // selection
  int64_t k;
  int64_t cap;                   // per-CTA candidate capacity (>= k + max cells)
  double* tk_e;                  // [grid][cap]
  double* tk_a;                  // [grid][cap]
  uint64_t* tk_key;              // [grid][cap][2*NINT]
  int* tk_cnt;                   // [grid]
  unsigned long long* tk_tau;    // [grid] CTA thresholds (bits of |e|)
  unsigned long long* tau_bits;  // global selection threshold (bits of |e|)
  unsigned int* sel_hist;        // [kSelBins] counts of candidates offered to the buffers, by |e| bin

  int max_cells;
  int* err;                      // device error flags (0 = fine)

  // gradient of E_PT2 (Psi0 and E0 fixed); used by the GRAD batch kernel
  double* g_dh;                  // [norb*norb]  symmetric halves off the diagonal
  double* g_deri;                // [P]          packed integrals
  double* g_wF;                  // [ndet][2][norb]  weights of dF^I_s(x) per generator rank
  double* g_wH;                  // [ndet]           weight of dH_II per generator rank
};

// The batch kernel's view of one wave of several instances: the pieces'
// parameters travel inside the kernel's parameters (constant bank, read-only
// and uncontended like a single sweep's), at most kMaxPieces per wave.
constexpr int kMaxPieces = 16;
struct MultiWaveInline {
  SweepParams ps[kMaxPieces];
  long long item_ofs[kMaxPieces + 1];
  int n;
  int chunk;                   // work items per draw from a piece's queue
  unsigned long long* queue;   // [n] the pieces' item counters
  unsigned long long timeout_ns;
  unsigned long long* t_start;
  int* err;                    // flag 128: the watchdog stopped the launch
};

// One wave of several instances' sweeps in one launch: ps[i] holds instance
// i's parameters for the wave; slot_ofs / item_ofs number the instances'
// generator slots / work items one instance after the other.
struct MultiWave {
  const SweepParams* ps;       // [n]
  const int* slot_ofs;         // [n + 1]
  const long long* item_ofs;   // [n + 1]
  int n;
  int chunk;                   // work items per draw (batch kernel)
  unsigned long long* queue;   // the pieces' item counters (batch kernel)
  unsigned long long timeout_ns;
  unsigned long long* t_start;
  int* err;                    // flag 128: the watchdog stopped the launch
};

}  // namespace qp
