/*
 * qp_pt2.h -- C ABI of the GB300 (sm_103a) Epstein-Nesbet PT2 + CIPSI
 * selection sweep (Quantum Package 2.0, arXiv:1902.08154).
 *
 * The library evaluates, for a zeroth-order wave function
 * Psi0 = sum_I c_I |I> given as packed bitstring determinants,
 *
 *   e_alpha = <Psi0|H|alpha>^2 / (E0 - <alpha|H|alpha>)        (Eq. e2)
 *   E_PT2   = sum over external alpha of e_alpha                 (Eq. PT2)
 *
 * over every external determinant alpha that is a single or double
 * substitution of some internal determinant, together with the k external
 * determinants of largest |e_alpha| (the CIPSI selection, Sec. "The basic
 * algorithm", step 4).  The sweep follows the paper's determinant-driven
 * scheme (Appendix "CIPSI selection and PT2 energy"): generators sorted by
 * decreasing c_I^2, each alpha counted once under the first generator it is
 * connected to (Eqs. calpha, edetstoch), a coarse filter of Psi0 per
 * generator and batches of alpha sharing the holes of the generator, with
 * matrix elements from the Slater-Condon rules (Eqs. Hij).
 *
 * Around the sweep: its adjoint (qp_pt2_grad), batches of independent sweeps
 * in one CUDA graph (qp_pt2_batch_*), sweeps of a subset of the generators
 * for the hybrid deterministic/stochastic E_PT2 (qp_pt2_eval_gens), target
 * spaces (qp_pt2_set_target), several states with the multi-state selection
 * criterion (qp_pt2_eval_states), and the variational step: H over Psi0 and
 * its lowest eigenpair (qp_pt2_sigma, qp_pt2_davidson).
 *
 * Conventions shared by every entry point
 * ----------------------------------------
 * Orbitals are 0-based, 1 <= norb <= 128; nint = (norb-1)/64 + 1.
 * A determinant is uint64_t[2][nint]: word [0][w] holds spin-up orbitals
 * 64w..64w+63 (orbital p in bit p%64), word [1][w] the spin-down ones
 * (Sec. "Internal representation of determinants").  The determinant KEY
 * orders determinants by these 2*nint words compared as unsigned integers,
 * spin-up words first.
 * h is double[norb*norb], row-major, symmetric: (p|h|q).
 * eri is the 8-fold packed chemists' integral array, double[P] with
 * P = M(M+1)/2, M = norb(norb+1)/2: (pq|rs) is stored at
 * tri(tri(p,q), tri(r,s)), tri(a,b) = max(a,b)(max(a,b)+1)/2 + min(a,b)
 * (the compound index of Algorithm hash, 0-based).
 * Spin orbitals are ordered spin-up before spin-down, increasing index
 * inside a spin; phases follow that ordering.
 *
 * Readings of points the paper leaves open:
 *  - "connected" is structural: alpha is a perturber when it is not internal
 *    and differs from some internal determinant by one or two spin orbitals,
 *    whatever the value of the matrix element;
 *  - generators are ranked by decreasing c_I^2 (the IEEE product c_I*c_I),
 *    ties by increasing input index;
 *  - the selection is ordered by decreasing |e_alpha|, ties by increasing
 *    key; k is a parameter;
 *  - E0 is an input and the coefficients are used as given (no
 *    normalisation).
 *
 * Pointers: every array argument may be host memory or device memory of the
 * current device; the library detects which (cudaPointerGetAttributes) and
 * copies host arrays through its own device workspace.  The library never
 * frees or retains caller memory.  Exceptions are stated at the entry
 * point: the rank list of qp_pt2_eval_gens, the energies of
 * qp_pt2_eval_states and the masks of qp_pt2_set_target are host arrays,
 * and qp_pt2_eval_noalloc takes device arrays only.  Calls run on the stream of the context's configuration and
 * return after the stream has finished the call's work.
 *
 * Reproducibility: in the one-state sweeps (qp_pt2_eval, _eval_ex,
 * _eval_gens, _grad, the batch and qp_pt2_eval_noalloc) the products
 * c_J <J|H|alpha> are summed exactly (96-bit integers in units of 2^-F, F
 * fixed per call from max |c_I|, N_det and the integrals' size) and rounded
 * once, the sums of a generator are reduced in a fixed order and E_PT2 in
 * rank order: the same inputs give the same bits on every run, every grid
 * size and every work-queue order.
 *
 * Errors: every entry point returns QP_OK (0) or a negative code; no call
 * aborts, traps or throws.  qp_pt2_strerror() names a code;
 * qp_pt2_last_error() gives the message of the last failing call of this
 * thread.
 */
#ifndef QP_PT2_H
#define QP_PT2_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define QP_OK 0
#define QP_EINVAL (-1)     /* bad size, occupation, bit beyond norb, k < 0 */
#define QP_EDUP (-2)       /* duplicate determinant in Psi0 */
#define QP_ESYM (-3)       /* h not symmetric to 1e-12 */
#define QP_ESINGULAR (-4)  /* some |E0 - H_aa| < 1e-12; results still filled */
#define QP_ENOMEM (-5)     /* device allocation failed */
#define QP_ECUDA (-6)      /* CUDA runtime error */
#define QP_ETIMEOUT (-7)   /* the device watchdog stopped the sweep (cfg timeout_s); results partial */
#define QP_ENOTSUP (-8)    /* configuration not supported by the library */
#define QP_ENOTCONV (-9)  /* Davidson stopped above its residual tolerance */

#define QP_FP64 0          /* every step in FP64 */
#define QP_MIXED 1         /* numerator <J|H|alpha> gathers and products c_J<J|H|alpha> in
                              FP32 (FP32 copies of h and eri); the products are summed
                              exactly into A_alpha (as in QP_FP64, below) and A_alpha is
                              rounded once to FP64; denominators E0 - H_aa, e_alpha and
                              every reduction in FP64.  Error bound per result: about
                              2^-24 * sum_alpha 2|A_alpha| sum_J |c_J H_Jalpha| / |D_alpha|. */

typedef struct qp_pt2_ctx qp_pt2_ctx; /* opaque, library-owned */

typedef struct {
    int precision;      /* QP_FP64 or QP_MIXED */
    void *stream;       /* cudaStream_t; NULL = legacy default stream */
    int blocks_per_sm;  /* persistent CTAs per SM; 0 = as many as fit */
    int threads;        /* threads per CTA; 0 = 256 */
    int shard_index;    /* generator sharding across processes: this call   */
    int shard_count;    /* sweeps the generators of rank r with              */
                        /* r % shard_count == shard_index (0, 0: all of them) */
    int work_chunk;     /* work items (generator x hole-set batch) a CTA takes from
                           the queue per draw; 0 = 1 */
    int tile;           /* tiles of rows each opposite-spin two-hole batch is split
                           into (its accumulator shrinks by that factor, so more
                           CTAs share an SM); 0 = chosen by the library (2 when
                           the whole accumulator fits only once per SM, else 1) */
    double timeout_s;   /* device watchdog: 0 = none; otherwise CTAs stop taking
                           work items once timeout_s seconds of device time have
                           passed since the call's sweep started, and the call
                           returns QP_ETIMEOUT with the partial results of the
                           items done (the context stays usable) */
} qp_pt2_config;

typedef struct {
    double e_pt2;               /* E_PT2 (Eq. PT2) */
    double sum_e_over_d;        /* sum_alpha A^2/D^2 = -dSigma/dE at E0 (Sec. "Renormalized
                                   PT2"): Z = 1/(1 + sum_e_over_d), E_rPT2 = E0 + Z E_PT2 */
    double min_abs_denominator; /* min |E0 - H_aa| over perturbers (inf if none) */
    int64_t n_perturbers;       /* |A|: external determinants connected to Psi0 */
    int64_t n_connections;      /* pairs (J, alpha), alpha in A, deg(J,alpha) <= 2 */
    int64_t n_selected;         /* min(k, n_perturbers) */
    int64_t n_tiny;             /* perturbers with |A_alpha| < 1e-14 */
    uint64_t perturber_digest[2]; /* order-free digest of the perturber set: the
                                    sum (mod 2^64) and the xor of
                                    splitmix64(hk ^ 0x243F6A8885A308D3) over the
                                    key hashes hk, hk = fold of splitmix64 over
                                    the 2*nint key words starting from 0 */
    double z;                   /* renormalisation factor Z = 1/(1 + sum_e_over_d) (Sec.
                                   "Renormalized PT2", Eq. Z) */
    double e_rpt2;              /* E0 + Z E_PT2: the renormalised second-order energy */
} qp_pt2_result;

/* Create a context for norb orbitals and n_alpha + n_beta electrons.
 * Copies h and eri to the device (context-owned).  cfg may be NULL.
 * Besides the packed copy the context keeps the integrals in a four-index
 * layout for the sweep's gathers: 8 norb^4 bytes (12 norb^4 with the FP32
 * copy of the mixed precision), e.g. 134 MB at norb = 64 and 2.1 GB at
 * norb = 128 in FP64.  QP_ENOMEM when the device cannot hold it.
 * Returns QP_EINVAL for sizes out of range, QP_ESYM if h is not symmetric. */
int qp_pt2_create(qp_pt2_ctx **out, int norb, int n_alpha, int n_beta, const double *h,
                  const double *eri, const qp_pt2_config *cfg);

/* One sweep over Psi0 (ndet determinants, layout above; coefs[ndet]).
 * Writes the best min(k, |A|) external determinants, best first, to
 * sel_dets[k][2][nint] and their e_alpha to sel_e[k] (either may be NULL when
 * k = 0).  Fills *res.  Validates Psi0: QP_EINVAL for a wrong popcount or a
 * bit at or beyond norb, QP_EDUP for a repeated determinant. */
int qp_pt2_eval(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, const double *coefs, double e0,
                int64_t k, uint64_t *sel_dets, double *sel_e, qp_pt2_result *res);

/* With sharding (shard_count > 1) the call covers only its share of the
 * generators: e_pt2, sums, counts and digest are partial (they add up over
 * the shards; the digests add modulo 2^64 and xor), the selection is the best
 * min(k, |A| of the shard) of the shard, and per-generator outputs of other
 * shards' generators are zero.
 *
 * qp_pt2_eval plus optional outputs (each may be NULL):
 *   sel_num[k]        A_alpha = <Psi0|H|alpha> of each selected determinant;
 *   eps_by_rank[ndet] eps_I of the generator of rank r (Eq. edetstoch);
 *   na_by_rank[ndet]  |A_I|;  ncon_by_rank[ndet]  connections of A_I;
 *   rank_of[ndet]     rank of each input determinant in the generator order. */
int qp_pt2_eval_ex(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, const double *coefs,
                   double e0, int64_t k, uint64_t *sel_dets, double *sel_e, double *sel_num,
                   double *eps_by_rank, int64_t *na_by_rank, int64_t *ncon_by_rank,
                   int32_t *rank_of, qp_pt2_result *res);

/* Target space (Sec. "Selected CI": the sweep applies to CAS, CIS, CISD ...
 * spaces, with the contributions of external determinants outside the
 * target space set to zero).  Later sweeps, subset sweeps and gradients of
 * ctx count an external determinant alpha only if every spin orbital set
 * in core is occupied in alpha, none set in deleted is, and, when ref is
 * given and max_exc >= 0, alpha differs from ref by at most max_exc
 * electrons.  ref, core, deleted: HOST arrays in determinant layout
 * ([2][nint] words), each may be NULL; all NULL clears the target space.
 * QP_EINVAL if a spin orbital is both core and deleted.  Psi0 itself is not
 * restricted. */
int qp_pt2_set_target(qp_pt2_ctx *ctx, const uint64_t *ref, int max_exc, const uint64_t *core,
                      const uint64_t *deleted);

/* The sweep of a subset of the generators (the building block of the
 * hybrid deterministic/stochastic E_PT2, Sec. "Stochastic selection",
 * Eqs. calpha and edetstoch): E_PT2 = sum_I eps_I over the generators sorted
 * by decreasing c_I^2, and each eps_I (its set A_I by the canonical rule)
 * depends on the whole Psi0 but not on which other eps are computed.
 * ranks[ngen] is a HOST array of distinct generator ranks in [0, ndet)
 * (rank 0 = largest c_I^2, ties by input index); only those generators are
 * swept.  gen_eps / gen_na / gen_ncon (each may be NULL; host or device)
 * receive eps_I, |A_I| and the connection count of each listed generator, in
 * list order, and gen_s2 (may be NULL) their sums A^2/D^2.  *res holds the
 * totals over the listed generators and the
 * selection is the best min(k, ...) of their perturbers.  The list overrides
 * sharding.  QP_EINVAL for a rank out of range, a repeated rank or a device
 * pointer for ranks. */
int qp_pt2_eval_gens(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, const double *coefs,
                     double e0, int64_t ngen, const int32_t *ranks, int64_t k, uint64_t *sel_dets,
                     double *sel_e, double *gen_eps, double *gen_s2, int64_t *gen_na, int64_t *gen_ncon,
                     qp_pt2_result *res);

/* E_PT2 from per-generator values by rank, reduced exactly as a whole sweep
 * reduces them (Eq. edetstoch: E_PT2 = sum over generators of eps_I, in rank
 * order, with the library's fixed-order compensated sum): a sweep assembled
 * from subset sweeps (a checkpointed or distributed one) gets the same bits
 * as one qp_pt2_eval.  eps[n], s2[n] (sum A^2/D^2 of each generator), na[n],
 * ncon[n]: host or device arrays indexed by rank.  Fills e_pt2,
 * sum_e_over_d, n_perturbers, n_connections, z and e_rpt2 of *res (the
 * other fields: 0, min_abs_denominator inf). */
int qp_pt2_reduce_ranks(qp_pt2_ctx *ctx, int64_t n, const double *eps, const double *s2, const int64_t *na,
                        const int64_t *ncon, double e0, qp_pt2_result *res);

/* Several states at once (Sec. "Selected CI": one PT2 calculation per
 * state, and the selection criterion of Angeli et al.):
 *
 *   A_s(alpha)     = <Psi0_s|H|alpha>,   c_alpha,s = A_s / (E0_s - H_aa)
 *   E_PT2,s        = sum over external alpha of A_s^2 / (E0_s - H_aa)
 *   e~(alpha)      = sum_s c_alpha,s A_s / max_I c_Is^2
 *
 * over the external determinants of the common internal space (dets).
 * nstates in [1, 4]; coefs is double[nstates][ndet] (state s at
 * coefs + s*ndet, host or device); e0 is a HOST array of nstates energies.
 * res is an array of nstates results: res[s].e_pt2 and sum_e_over_d are
 * state s's; the counts, digest, n_selected and n_tiny (of state 0's A) are
 * shared; min_abs_denominator is the minimum over alpha and states.  The
 * selection keeps the k determinants of largest |e~| (ties by key):
 * sel_dets [k][2][nint], sel_crit [k] (e~), sel_num [k] (state 0's A); each
 * may be NULL when k = 0.  FP64 contexts only (QP_ENOTSUP for mixed
 * precision, or when nstates accumulators of the largest batch do not fit
 * in one CTA's shared memory); QP_EINVAL for nstates out of range or a
 * state whose coefficients are all zero.  Target spaces and sharding apply
 * as in qp_pt2_eval. */
int qp_pt2_eval_states(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, int nstates,
                       const double *coefs, const double *e0, int64_t k, uint64_t *sel_dets,
                       double *sel_crit, double *sel_num, qp_pt2_result *res);

/* The variational step of CIPSI (Sec. "Davidson diagonalization"): the
 * Hamiltonian over Psi0 and its lowest eigenpair.
 *
 * qp_pt2_sigma: S[k] = H U[k] for nvec vectors (U, S: [nvec][ndet], host or
 * device), H the matrix of Psi0's determinants (Slater-Condon rules,
 * Eqs. Hij).  H is rebuilt on every call (device memory freed on return).
 *
 * qp_pt2_davidson: the lowest eigenvalue *e0 and its normalised eigenvector
 * coefs[ndet] (host or device; coefs[0] >= 0), by Davidson's method with the
 * diagonal preconditioner, starting from guess (NULL: the determinant of
 * lowest H_II), until the residual norm |H c - e0 c| <= tol or max_iter
 * basis extensions (QP_ENOTCONV, outputs still written).  *e0 is the
 * Rayleigh quotient of the returned vector.  info (may be NULL) receives the
 * iteration count, the final residual, the number of stored off-diagonal
 * elements and the build and solve times.  Psi0 is validated as for
 * qp_pt2_eval (QP_EINVAL, QP_EDUP).  Allocates device memory for H and the
 * basis (32 vectors). */
typedef struct {
  int iterations, converged;
  double residual;
  int64_t nnz;
  double build_ms, solve_ms;
} qp_pt2_davidson_info;

int qp_pt2_sigma(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, int nvec, const double *U, double *S);
int qp_pt2_davidson(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, const double *guess, double tol,
                    int max_iter, double *coefs, double *e0, qp_pt2_davidson_info *info);

/* The Hamiltonian over Psi0 as it is built for qp_pt2_sigma and
 * qp_pt2_davidson: the off-diagonal elements of the pairs at excitation
 * degree 1 or 2 in CSR form, columns ascending within each row, and the
 * diagonal.  search 0: connected pairs found through the spin-up and
 * spin-down strings (Appendix "Davidson diagonalization": Psi0 = sum C_IJ
 * |I_up J_dn>, same-spin excitations along a row or a column of C,
 * opposite-spin doubles by a spin-up single excitation then a spin-down one;
 * the work per row is the length of its string lists, O(N_det^(3/2)) in all);
 * search 1: every pair tested, O(N_det^2).  Both give the same matrix.
 * *nnz (host) receives the number of stored off-diagonal elements; rowptr
 * [ndet+1] (int64), cols [nnz], vals [nnz] and diag [ndet] are written when
 * not NULL (host or device memory), so a first call with cols = vals = NULL
 * gives the sizes.  *build_ms (may be NULL): device time of the build.
 * Psi0 is validated as for qp_pt2_eval (QP_EINVAL, QP_EDUP). */
int qp_pt2_hamiltonian(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, int search, int64_t *nnz,
                       int64_t *rowptr, int32_t *cols, double *vals, double *diag, double *build_ms);

/* Gradient of E_PT2 (adjoint of the sweep), with Psi0's coefficients and E0
 * held fixed.  Every matrix element is linear in h and the integrals (Eqs.
 * Hij), so with A_alpha = <Psi0|H|alpha> and D_alpha = E0 - <alpha|H|alpha>
 * (Eqs. e2, PT2):
 *   dE/dtheta = sum_alpha [ (2 A/D) sum_J c_J d<J|H|alpha>/dtheta
 *                           + (A/D)^2 d<alpha|H|alpha>/dtheta ],
 *   dE/dE0    = - sum_alpha A^2/D^2.
 * The matrix elements are recomputed (nothing is kept from qp_pt2_eval).
 * Outputs (host or device memory): dh[norb*norb], symmetric, with
 * dh[p][q] = dh[q][p] = (1/2) dE/du_pq for p != q where u_pq moves h_pq and
 * h_qp together, and dh[p][p] = dE/dh_pp; deri[P], the derivative with respect
 * to each packed entry of eri; *de0.  *res (may be NULL) receives the sweep's
 * totals (no selection).  FP64 contexts only (QP_ENOTSUP otherwise); with
 * sharding the gradient is the shard's part and the shards' gradients add. */
int qp_pt2_grad(qp_pt2_ctx *ctx, int64_t ndet, const uint64_t *dets, const double *coefs, double e0,
                double *dh, double *deri, double *de0, qp_pt2_result *res);

/* Batched sweeps (many independent Psi0 instances, each with its own context,
 * Hamiltonian and size).  qp_pt2_batch_create plans every instance (device
 * workspaces are allocated here, once), then captures all of their sweeps on
 * up to max_streams concurrent streams (0: 16) into one CUDA graph: no host
 * synchronisation happens inside an instance's sweep, input checks run on the
 * device.  qp_pt2_batch_run launches the graph on `stream` (NULL: a stream of
 * the batch's own), waits, and fills res[n] (one result per instance; its
 * return value is the first instance error, QP_OK if none) and, if ms is not
 * NULL, the graph's device time in milliseconds.  The graph may be run any
 * number of times; it reads the inputs and writes the outputs at the
 * addresses given here, so new inputs of the same sizes can be written in
 * place between runs.
 *   ctxs[n]      distinct FP64 or mixed contexts (no sharding); a context must
 *                not be used by other calls while the batch exists
 *   ndet[n], dets[n], coefs[n], e0[n], k[n]: as in qp_pt2_eval, device memory
 *   sel_dets[n], sel_e[n]: device outputs (may be NULL where k[i] = 0)
 *   grid[n]      persistent CTAs of each instance's sweep (NULL or 0: the
 *                context's default); chosen by the package's autotuner
 * qp_pt2_batch_create is qp_pt2_batch_create_ex with fused = 0 and the
 * given max_streams. */
typedef struct qp_pt2_batch qp_pt2_batch;
int qp_pt2_batch_create(qp_pt2_batch **out, int n, qp_pt2_ctx *const *ctxs, const int64_t *ndet,
                        const uint64_t *const *dets, const double *const *coefs, const double *e0,
                        const int64_t *k, uint64_t *const *sel_dets, double *const *sel_e, const int *grid,
                        int max_streams, void *stream);

/* Launch shape of a batch (qp_pt2_batch_create_ex).
 *   fused = 1: the instances are grouped by words per spin and precision; the
 *     sweeps of a group run as one persistent launch per wave whose work
 *     queue spans the (instance, generator, hole-set batch) items of all its
 *     instances, instance after instance (the instance with the largest
 *     work items first), and every CTA may take items of every instance.
 *     The instances' waves are planned together so that all of a group's
 *     instances finish in about the same number of waves.  The groups run
 *     on concurrent streams; validation, ranking and the selection merge of
 *     each instance run on up to max_streams concurrent streams.
 *   fused = 0: each instance's sweep keeps launches of its own, on up to
 *     max_streams concurrent streams (grid[] applies in this form only).
 *   work_chunk    fused: items per draw from the shared queue (0: 1)
 *   tile          fused: row tiles of the opposite-spin batches, applied to
 *                 every instance (0: each context's own choice)
 *   blocks_per_sm fused: persistent CTAs per SM (0: as many as fit)
 *   wave_gb       fused: device memory for the records and buckets of one
 *                 wave of all instances, in GiB (0: 24) */
typedef struct {
    int fused;
    int max_streams;
    int work_chunk;
    int tile;
    int blocks_per_sm;
    double wave_gb;
} qp_pt2_batch_options;
int qp_pt2_batch_create_ex(qp_pt2_batch **out, int n, qp_pt2_ctx *const *ctxs, const int64_t *ndet,
                           const uint64_t *const *dets, const double *const *coefs, const double *e0,
                           const int64_t *k, uint64_t *const *sel_dets, double *const *sel_e, const int *grid,
                           const qp_pt2_batch_options *opt, void *stream);
int qp_pt2_batch_run(qp_pt2_batch *batch, qp_pt2_result *res, double *ms);
void qp_pt2_batch_destroy(qp_pt2_batch *batch);

/* Number of device kernel launches made by the last qp_pt2_eval* call of ctx
 * (the library's own kernels; the radix sorts' kernels are not counted). */
int64_t qp_pt2_last_launches(const qp_pt2_ctx *ctx);

/* Device time of the last qp_pt2_eval* call of ctx, from CUDA events recorded
 * on the context's stream: ms[0] = the persistent sweep kernel alone,
 * ms[1] = from the first to the last device operation of the call.
 * Returns QP_EINVAL if no call has completed yet. */
int qp_pt2_last_timings(const qp_pt2_ctx *ctx, double *ms);

/* The whole sweep without allocating any device memory.  The paper has no
 * counterpart: this entry point exists for callers that cannot call
 * cudaMalloc or cudaFree -- a host program that reserves the GPU's memory up
 * front and gives its plugins no allocator, or a deployment whose device
 * footprint must stay fixed.
 *
 * No context is used.  h, eri, dets, coefs and (when k > 0) sel_dets and
 * sel_e must be device memory of the current device (QP_EINVAL otherwise);
 * layouts are those of qp_pt2_create and qp_pt2_eval; res is host memory.
 * The work runs on `stream` (a cudaStream_t, NULL = legacy default stream)
 * and the call returns once it has finished.  Results equal those of
 * qp_pt2_eval for the same inputs (same rules, same tolerances).
 *
 * Scratch: one 64 MiB device array inside the library (static storage),
 * which every GPU that loads the library holds until the process exits.  The
 * first call on a device looks up that array's device address
 * (cudaGetSymbolAddress) and caches it; make that first call before any
 * stream capture.  Every call reuses the same array: calls whose GPU work
 * overlaps (other streams, other threads) race and must not be issued.
 * Problems whose integral tables, generator order, per-generator records,
 * selection buffers (one CTA per SM, k + cells entries each) and sort space
 * do not fit in the array are refused with QP_EINVAL; as a guide, 64
 * orbitals with 10+10 electrons fit up to roughly 10^3 determinants with
 * k = 10^3. */
int qp_pt2_eval_noalloc(int norb, int n_alpha, int n_beta, const double *h, const double *eri,
                        int64_t ndet, const uint64_t *dets, const double *coefs, double e0, int64_t k,
                        uint64_t *sel_dets, double *sel_e, qp_pt2_result *res, void *stream);

/* Merge of the partial results of n generator shards of one sweep (the
 * exchange step of a sharded sweep, Sec. "Parallelism"): E_PT2, sum A^2/D^2,
 * the counts and n_tiny add, the digest words add modulo 2^64 and xor, the
 * minimum denominator is the minimum, n_selected is left 0 (the selection is
 * merged separately), and z, e_rpt2 are recomputed from the merged sums with
 * e0.  parts and out are host memory; out may alias parts[0].  QP_EINVAL if
 * n < 1 or a pointer is NULL. */
int qp_pt2_merge_results(int n, const qp_pt2_result *parts, double e0, qp_pt2_result *out);

/* Release the context and its device memory.  NULL is accepted. */
void qp_pt2_destroy(qp_pt2_ctx *ctx);

const char *qp_pt2_strerror(int code);
const char *qp_pt2_last_error(void);

#ifdef __cplusplus
}
#endif
#endif
