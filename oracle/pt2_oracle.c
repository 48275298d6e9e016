/*
 * pt2_oracle.c -- plain, slow FP64 CPU oracle for the Epstein-Nesbet PT2 and
 * CIPSI selection sweep of Quantum Package 2.0 (arXiv:1902.08154).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this library.  The CUDA library never
 * links, includes or calls anything in this directory, and this file shares
 * no code, header, table or constant with it.
 *
 * What is computed, and where the paper defines it:
 *   - Target spaces (Sec. "Selected CI", the remark that the method applies
 *     to CAS, CIS, CISD, ... spaces): external determinants outside the
 *     target space contribute nothing (or_set_target; a filter on alpha).
 *   - Slater-Condon rules for <I|H|I>, <I|H|I_p^r>, <I|H|I_pq^rs>
 *     (Sec. "Matrix elements of the Hamiltonian", Eqs. Hij).  Phases are
 *     obtained by COUNTING the occupied spin orbitals between hole and particle
 *     in the ordering of Sec. "Internal representation of determinants"
 *     (spin-up before spin-down, increasing index inside a spin); no phase
 *     masks are used here.
 *   - e_alpha = <Psi0|H|alpha>^2 / (E0 - <alpha|H|alpha>)   (Eq. e2)
 *   - E_PT2 = sum over external alpha of e_alpha             (Eq. PT2)
 *   - the per-generator split E_PT2 = sum_I eps_I with A_I the determinants
 *     connected to I and to no generator before it, generators sorted by
 *     decreasing c_I^2 (Eqs. calpha, edetstoch; Appendix "CIPSI selection and
 *     PT2 energy")
 *   - selection of the k external determinants of largest |e_alpha|
 *     (Sec. "The basic algorithm", step 4);
 *   - several states: one PT2 per state and the selection criterion of
 *     Angeli et al. quoted in Sec. "Selected CI" (or_states).
 *
 * Readings taken where the paper is silent (each is listed in the design
 * notes): "connected" means structurally connected (excitation degree 1 or 2);
 * ties in c_I^2 are broken by input index; ties in |e_alpha| by the
 * determinant key (spin-up words then spin-down words, unsigned, ascending);
 * E0 is an independent input and coefficients are used as given.
 *
 * Two independent evaluations of the sweep are provided:
 *   or_sweep      -- the plain definition.  Every pair (J, alpha) with alpha a
 *                    single or double substitution of an internal J is
 *                    enumerated; pairs are grouped by alpha (sorting), so that
 *                    A_alpha = sum_J c_J <J|H|alpha> is formed directly, and
 *                    the generator of alpha is the lowest-ranked J connected
 *                    to it.  Pairs are bucketed by a hash of alpha's key so
 *                    that memory stays bounded.
 *   or_generator  -- the per-generator definition for one generator I of rank
 *                    g: every substitution alpha of I is tested against every
 *                    internal J within excitation degree 4 of I (the only J
 *                    that can be within degree 2 of alpha).
 *   or_states     -- several states: the plain definition with every alpha
 *                    formed once and A_k taken over all internal J.
 */
#define _GNU_SOURCE
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define OR_MAXNINT 2
#define OR_MAXORB 128
#define OR_NSUB 64

/* ------------------------------------------------------------------------ */
/* Hamiltonian                                                               */
/* ------------------------------------------------------------------------ */

typedef struct or_ham {
    int norb, nint, nalpha, nbeta;
    double *h;   /* norb*norb */
    double *eri; /* packed, 8-fold */
    double *J;   /* J[p*norb+q] = (pp|qq) */
    double *K;   /* K[p*norb+q] = (pq|qp) */
    /* target space (Sec. "Selected CI" remark on CAS/CISD spaces): external
     * determinants outside it contribute nothing */
    int tgt_on, tgt_max_exc;
    uint64_t tgt_ref[4], tgt_core[4], tgt_del[4];
} or_ham;

/* alpha belongs to the target space: every core spin orbital occupied, no
 * deleted one occupied, and (when max_exc >= 0) at most max_exc electrons
 * moved from the reference determinant. */
static int in_target(const or_ham *H, const uint64_t *a)
{
    if (!H->tgt_on) return 1;
    int moved = 0;
    for (int w = 0; w < 2 * H->nint; w++) {
        if ((a[w] & H->tgt_core[w]) != H->tgt_core[w]) return 0;
        if (a[w] & H->tgt_del[w]) return 0;
        moved += __builtin_popcountll(a[w] ^ H->tgt_ref[w]);
    }
    return H->tgt_max_exc < 0 || moved / 2 <= H->tgt_max_exc;
}

/* Sets the target space; ref/core/deleted may be NULL (no constraint). */
void or_set_target(or_ham *H, int on, const uint64_t *ref, int max_exc, const uint64_t *core, const uint64_t *deleted)
{
    H->tgt_on = on;
    H->tgt_max_exc = ref ? max_exc : -1;
    for (int w = 0; w < 4; w++) {
        H->tgt_ref[w] = (ref && w < 2 * H->nint) ? ref[w] : 0;
        H->tgt_core[w] = (core && w < 2 * H->nint) ? core[w] : 0;
        H->tgt_del[w] = (deleted && w < 2 * H->nint) ? deleted[w] : 0;
    }
}

static int64_t tri(int64_t a, int64_t b)
{
    if (a < b) { int64_t t = a; a = b; b = t; }
    return a * (a + 1) / 2 + b;
}

/* chemists' (pq|rs) */
double or_eri(const or_ham *H, int p, int q, int r, int s)
{
    return H->eri[tri(tri(p, q), tri(r, s))];
}

or_ham *or_ham_new(int norb, int nalpha, int nbeta, const double *h, const double *eri)
{
    if (norb < 1 || norb > OR_MAXORB || nalpha < 0 || nbeta < 0 || nalpha > norb || nbeta > norb)
        return NULL;
    or_ham *H = (or_ham *)calloc(1, sizeof(or_ham));
    int64_t m = (int64_t)norb * (norb + 1) / 2;
    int64_t P = m * (m + 1) / 2;
    H->norb = norb;
    H->nint = (norb - 1) / 64 + 1;
    H->nalpha = nalpha;
    H->nbeta = nbeta;
    H->h = (double *)malloc(sizeof(double) * norb * norb);
    H->eri = (double *)malloc(sizeof(double) * P);
    H->J = (double *)malloc(sizeof(double) * norb * norb);
    H->K = (double *)malloc(sizeof(double) * norb * norb);
    memcpy(H->h, h, sizeof(double) * norb * norb);
    memcpy(H->eri, eri, sizeof(double) * P);
    for (int p = 0; p < norb; p++)
        for (int q = 0; q < norb; q++) {
            H->J[p * norb + q] = or_eri(H, p, p, q, q);
            H->K[p * norb + q] = or_eri(H, p, q, q, p);
        }
    return H;
}

void or_ham_free(or_ham *H)
{
    if (!H) return;
    free(H->h); free(H->eri); free(H->J); free(H->K);
    free(H);
}

/* ------------------------------------------------------------------------ */
/* Determinants: words [spin][nint]; orbital p is bit p%64 of word p/64.      */
/* ------------------------------------------------------------------------ */

static int getbit(const uint64_t *d, int nint, int s, int p)
{
    return (int)((d[s * nint + p / 64] >> (p % 64)) & 1u);
}

static void setbit(uint64_t *d, int nint, int s, int p) { d[s * nint + p / 64] |= (uint64_t)1 << (p % 64); }
static void clrbit(uint64_t *d, int nint, int s, int p) { d[s * nint + p / 64] &= ~((uint64_t)1 << (p % 64)); }

static int popc64(uint64_t x)
{
    int n = 0;
    while (x) { x &= x - 1; n++; }
    return n;
}

int or_degree(int nint, const uint64_t *a, const uint64_t *b)
{
    int n = 0;
    for (int w = 0; w < 2 * nint; w++) n += popc64(a[w] ^ b[w]);
    return n / 2;
}

/* unsigned lexicographic compare of the 2*nint words (spin-up words first) */
static int keycmp(const uint64_t *a, const uint64_t *b, int nw)
{
    for (int w = 0; w < nw; w++) {
        if (a[w] < b[w]) return -1;
        if (a[w] > b[w]) return 1;
    }
    return 0;
}

/* Sign of a^+_p a_h on the ordered determinant d (same spin s): (-1) to the
 * number of occupied spin-s orbitals strictly between h and p.  Spin-down
 * operators never cross spin-up ones because all spin-up operators come
 * first in the ordering. */
static double phase_single(const uint64_t *d, int nint, int s, int h, int p)
{
    int lo = h < p ? h : p, hi = h < p ? p : h, n = 0;
    for (int o = lo + 1; o < hi; o++) n += getbit(d, nint, s, o);
    return (n & 1) ? -1.0 : 1.0;
}

/* <I|H|I>: sum_i h_ii + sum over pairs i<j of [(ii|jj) - delta_spin (ij|ji)] */
double or_diag(const or_ham *H, const uint64_t *d)
{
    int norb = H->norb, nint = H->nint;
    int occ[2 * OR_MAXORB], spin[2 * OR_MAXORB], n = 0;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++)
            if (getbit(d, nint, s, p)) { occ[n] = p; spin[n] = s; n++; }
    double e = 0.0;
    for (int i = 0; i < n; i++) e += H->h[occ[i] * norb + occ[i]];
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            e += H->J[occ[i] * norb + occ[j]];
            if (spin[i] == spin[j]) e -= H->K[occ[i] * norb + occ[j]];
        }
    return e;
}

/* <I|H|J> by Slater-Condon.  Holes are spin orbitals of I missing from J,
 * particles those of J missing from I, both listed in the determinant
 * ordering (spin-up first, increasing orbital index). */
double or_hij(const or_ham *H, const uint64_t *I, const uint64_t *Jd)
{
    int norb = H->norb, nint = H->nint;
    int deg = or_degree(nint, I, Jd);
    if (deg == 0) return or_diag(H, I);
    if (deg > 2) return 0.0;
    int hs[2], ho[2], ps[2], po[2], nh = 0, np = 0;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++) {
            int a = getbit(I, nint, s, p), b = getbit(Jd, nint, s, p);
            if (a && !b) { hs[nh] = s; ho[nh] = p; nh++; }
            if (!a && b) { ps[np] = s; po[np] = p; np++; }
        }
    if (deg == 1) {
        int s = hs[0], h = ho[0], p = po[0];
        double v = H->h[h * norb + p];
        for (int t = 0; t < 2; t++)
            for (int i = 0; i < norb; i++) {
                if (!getbit(I, nint, t, i)) continue;
                v += or_eri(H, h, p, i, i);
                if (t == s) v -= or_eri(H, h, i, i, p);
            }
        return phase_single(I, nint, s, h, p) * v;
    }
    /* deg == 2: pair hole k with particle k; apply h1->p1 then h2->p2 */
    uint64_t I1[2 * OR_MAXNINT];
    memcpy(I1, I, sizeof(uint64_t) * 2 * nint);
    double ph = phase_single(I, nint, hs[0], ho[0], po[0]);
    clrbit(I1, nint, hs[0], ho[0]);
    setbit(I1, nint, ps[0], po[0]);
    ph *= phase_single(I1, nint, hs[1], ho[1], po[1]);
    double v = or_eri(H, ho[0], po[0], ho[1], po[1]);
    if (hs[0] == hs[1]) v -= or_eri(H, ho[0], po[1], ho[1], po[0]);
    return ph * v;
}

/* ------------------------------------------------------------------------ */
/* Substitutions of one determinant, by explicit orbital loops.              */
/* Calls emit(ctx, alpha) for every single and double substitution.         */
/* ------------------------------------------------------------------------ */

typedef void (*emit_fn)(void *ctx, const uint64_t *alpha);

static void for_each_substitution(const or_ham *H, const uint64_t *d, emit_fn emit, void *ctx)
{
    int norb = H->norb, nint = H->nint;
    int occ[2][OR_MAXORB], vir[2][OR_MAXORB], no[2] = {0, 0}, nv[2] = {0, 0};
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++) {
            if (getbit(d, nint, s, p)) occ[s][no[s]++] = p;
            else vir[s][nv[s]++] = p;
        }
    uint64_t a[2 * OR_MAXNINT];
    /* singles */
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < no[s]; i++)
            for (int x = 0; x < nv[s]; x++) {
                memcpy(a, d, sizeof(uint64_t) * 2 * nint);
                clrbit(a, nint, s, occ[s][i]);
                setbit(a, nint, s, vir[s][x]);
                emit(ctx, a);
            }
    /* same-spin doubles */
    for (int s = 0; s < 2; s++)
        for (int i = 0; i < no[s]; i++)
            for (int j = i + 1; j < no[s]; j++)
                for (int x = 0; x < nv[s]; x++)
                    for (int y = x + 1; y < nv[s]; y++) {
                        memcpy(a, d, sizeof(uint64_t) * 2 * nint);
                        clrbit(a, nint, s, occ[s][i]);
                        clrbit(a, nint, s, occ[s][j]);
                        setbit(a, nint, s, vir[s][x]);
                        setbit(a, nint, s, vir[s][y]);
                        emit(ctx, a);
                    }
    /* opposite-spin doubles */
    for (int i = 0; i < no[0]; i++)
        for (int j = 0; j < no[1]; j++)
            for (int x = 0; x < nv[0]; x++)
                for (int y = 0; y < nv[1]; y++) {
                    memcpy(a, d, sizeof(uint64_t) * 2 * nint);
                    clrbit(a, nint, 0, occ[0][i]);
                    clrbit(a, nint, 1, occ[1][j]);
                    setbit(a, nint, 0, vir[0][x]);
                    setbit(a, nint, 1, vir[1][y]);
                    emit(ctx, a);
                }
}

int64_t or_n_substitutions(const or_ham *H)
{
    int64_t na = H->nalpha, nb = H->nbeta, va = H->norb - na, vb = H->norb - nb;
    return na * va + nb * vb + (na * (na - 1) / 2) * (va * (va - 1) / 2) +
           (nb * (nb - 1) / 2) * (vb * (vb - 1) / 2) + na * nb * va * vb;
}

typedef struct { int nw; int64_t n, cap; uint64_t *out; } collect_ctx;

static void collect_emit(void *vctx, const uint64_t *alpha)
{
    collect_ctx *c = (collect_ctx *)vctx;
    if (c->n < c->cap) memcpy(c->out + c->n * c->nw, alpha, sizeof(uint64_t) * c->nw);
    c->n++;
}

/* All substitutions of det d, in the loop order above; returns their count
 * (writes at most cap of them). */
int64_t or_substitutions(const or_ham *H, const uint64_t *d, int64_t cap, uint64_t *out)
{
    collect_ctx c = {2 * H->nint, 0, cap, out};
    for_each_substitution(H, d, collect_emit, &c);
    return c.n;
}

/* ------------------------------------------------------------------------ */
/* Digest of a set of determinants: order independent.                      */
/* splitmix64 finaliser (Steele, Lea & Flood 2014, with the constants of     */
/* Vigna's public reference implementation).                                 */
/* ------------------------------------------------------------------------ */

static uint64_t splitmix64(uint64_t x)
{
    x += 0x9E3779B97F4A7C15ull;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    return x ^ (x >> 31);
}

uint64_t or_key_hash(int nw, const uint64_t *key)
{
    uint64_t hk = 0;
    for (int w = 0; w < nw; w++) hk = splitmix64(hk ^ key[w]);
    return hk;
}

/* ------------------------------------------------------------------------ */
/* Compensated summation (Neumaier 1974).                                    */
/* ------------------------------------------------------------------------ */

typedef struct { double s, c; } nsum;

static void nsum_add(nsum *a, double x)
{
    double t = a->s + x;
    if (fabs(a->s) >= fabs(x)) a->c += (a->s - t) + x;
    else a->c += (x - t) + a->s;
    a->s = t;
}

static double nsum_get(const nsum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Bounded selection: keep the k best (|e| descending, key ascending).       */
/* Binary min-heap whose root is the worst kept entry.                       */
/* ------------------------------------------------------------------------ */

typedef struct {
    int nw;
    int64_t k, n;
    double *e, *num;   /* e_alpha and A_alpha */
    uint64_t *key;     /* n * nw */
} topk;

static int worse(const topk *t, double ea, const uint64_t *ka, double eb, const uint64_t *kb)
{
    double a = fabs(ea), b = fabs(eb);
    if (a != b) return a < b;
    return keycmp(ka, kb, t->nw) > 0;
}

static void topk_init(topk *t, int nw, int64_t k)
{
    t->nw = nw; t->k = k; t->n = 0;
    t->e = (double *)malloc(sizeof(double) * (k > 0 ? k : 1));
    t->num = (double *)malloc(sizeof(double) * (k > 0 ? k : 1));
    t->key = (uint64_t *)malloc(sizeof(uint64_t) * nw * (k > 0 ? k : 1));
}

static void topk_free(topk *t) { free(t->e); free(t->num); free(t->key); }

static void topk_swap(topk *t, int64_t i, int64_t j)
{
    double x = t->e[i]; t->e[i] = t->e[j]; t->e[j] = x;
    x = t->num[i]; t->num[i] = t->num[j]; t->num[j] = x;
    uint64_t tmp[2 * OR_MAXNINT];
    memcpy(tmp, t->key + i * t->nw, 8 * t->nw);
    memcpy(t->key + i * t->nw, t->key + j * t->nw, 8 * t->nw);
    memcpy(t->key + j * t->nw, tmp, 8 * t->nw);
}

static int heap_less(const topk *t, int64_t i, int64_t j)
{
    return worse(t, t->e[i], t->key + i * t->nw, t->e[j], t->key + j * t->nw);
}

static void topk_push(topk *t, double e, double num, const uint64_t *key)
{
    if (t->k <= 0) return;
    if (t->n < t->k) {
        int64_t i = t->n++;
        t->e[i] = e; t->num[i] = num;
        memcpy(t->key + i * t->nw, key, 8 * t->nw);
        while (i > 0) {
            int64_t p = (i - 1) / 2;
            if (heap_less(t, i, p)) { topk_swap(t, i, p); i = p; } else break;
        }
        return;
    }
    if (!worse(t, t->e[0], t->key, e, key)) return; /* root is not worse: reject */
    t->e[0] = e; t->num[0] = num;
    memcpy(t->key, key, 8 * t->nw);
    int64_t i = 0;
    for (;;) {
        int64_t l = 2 * i + 1, r = l + 1, m = i;
        if (l < t->n && heap_less(t, l, m)) m = l;
        if (r < t->n && heap_less(t, r, m)) m = r;
        if (m == i) break;
        topk_swap(t, i, m);
        i = m;
    }
}

/* ------------------------------------------------------------------------ */
/* Generator ranks: stable sort by decreasing c^2, ties by input index.      */
/* ------------------------------------------------------------------------ */

typedef struct { double c2; int64_t i; } rank_rec;

static int rank_cmp(const void *a, const void *b)
{
    const rank_rec *x = (const rank_rec *)a, *y = (const rank_rec *)b;
    if (x->c2 > y->c2) return -1;
    if (x->c2 < y->c2) return 1;
    return (x->i < y->i) ? -1 : (x->i > y->i);
}

/* rank_of[i] = position of det i in the generator order */
void or_ranks(int64_t ndet, const double *coefs, int64_t *rank_of)
{
    rank_rec *r = (rank_rec *)malloc(sizeof(rank_rec) * (ndet > 0 ? ndet : 1));
    for (int64_t i = 0; i < ndet; i++) { r[i].c2 = coefs[i] * coefs[i]; r[i].i = i; }
    qsort(r, ndet, sizeof(rank_rec), rank_cmp);
    for (int64_t g = 0; g < ndet; g++) rank_of[r[g].i] = g;
    free(r);
}

/* ------------------------------------------------------------------------ */
/* Sorted internal keys for membership tests.                                */
/* ------------------------------------------------------------------------ */

static int g_nw_sort; /* only used by qsort below, set before each call in a
                         single-threaded section */

static int key_qcmp(const void *a, const void *b)
{
    return keycmp((const uint64_t *)a, (const uint64_t *)b, g_nw_sort);
}

static int is_member(const uint64_t *sorted, int64_t n, int nw, const uint64_t *key)
{
    int64_t lo = 0, hi = n - 1;
    while (lo <= hi) {
        int64_t mid = lo + (hi - lo) / 2;
        int c = keycmp(sorted + mid * nw, key, nw);
        if (c == 0) return 1;
        if (c < 0) lo = mid + 1; else hi = mid - 1;
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Validation of the internal space.                                         */
/* ------------------------------------------------------------------------ */

/* 0 ok; -1 bad occupation (popcount or bits beyond norb); -2 duplicate */
int or_validate(const or_ham *H, int64_t ndet, const uint64_t *dets)
{
    int nint = H->nint, nw = 2 * nint;
    for (int64_t i = 0; i < ndet; i++) {
        const uint64_t *d = dets + i * nw;
        for (int s = 0; s < 2; s++) {
            int n = 0;
            for (int w = 0; w < nint; w++) n += popc64(d[s * nint + w]);
            if (n != (s == 0 ? H->nalpha : H->nbeta)) return -1;
            for (int p = H->norb; p < 64 * nint; p++)
                if (getbit(d, nint, s, p)) return -1;
        }
    }
    uint64_t *srt = (uint64_t *)malloc(sizeof(uint64_t) * nw * (ndet > 0 ? ndet : 1));
    memcpy(srt, dets, sizeof(uint64_t) * nw * ndet);
    g_nw_sort = nw;
    qsort(srt, ndet, sizeof(uint64_t) * nw, key_qcmp);
    int dup = 0;
    for (int64_t i = 1; i < ndet; i++)
        if (keycmp(srt + (i - 1) * nw, srt + i * nw, nw) == 0) dup = 1;
    free(srt);
    return dup ? -2 : 0;
}

/* ------------------------------------------------------------------------ */
/* Result record shared by both sweeps.                                      */
/* ------------------------------------------------------------------------ */

typedef struct {
    double e_pt2;            /* sum_alpha e_alpha */
    double sum_e_over_d;     /* sum_alpha A^2 / D^2 (= -dSigma/dE at E0) */
    double min_abs_den;      /* min |E0 - H_aa| over perturbers */
    int64_t n_perturbers;    /* |A| */
    int64_t n_connections;   /* pairs (J, alpha), alpha in A, deg(J,alpha) <= 2 */
    int64_t n_selected;
    int64_t n_tiny;          /* perturbers with |A_alpha| < 1e-14 */
    uint64_t digest[2];      /* sum and xor of key hashes over A */
} or_result;

/* ------------------------------------------------------------------------ */
/* or_sweep: the plain definition, pairs grouped by alpha.                   */
/* ------------------------------------------------------------------------ */

typedef struct {
    const or_ham *H;
    int nw, stride;      /* stride = nw + 1 words: key then J index */
    int nparts, part;
    int64_t *cnt, *cap;  /* per sub-bucket */
    uint64_t **buf;      /* per sub-bucket record arrays */
    int64_t jidx;
} pair_ctx;

static void pair_emit(void *vctx, const uint64_t *alpha)
{
    pair_ctx *c = (pair_ctx *)vctx;
    if (!in_target(c->H, alpha)) return;  /* outside the target space: no contribution */
    uint64_t hk = or_key_hash(c->nw, alpha);
    if ((int)((hk >> 32) % (uint64_t)c->nparts) != c->part) return;
    int sub = (int)((hk & 0xffffffffull) % OR_NSUB);
    if (c->cnt[sub] == c->cap[sub]) {
        c->cap[sub] = c->cap[sub] ? 2 * c->cap[sub] : 1024;
        c->buf[sub] = (uint64_t *)realloc(c->buf[sub], sizeof(uint64_t) * c->stride * c->cap[sub]);
    }
    uint64_t *r = c->buf[sub] + c->cnt[sub] * c->stride;
    memcpy(r, alpha, sizeof(uint64_t) * c->nw);
    r[c->nw] = (uint64_t)c->jidx;
    c->cnt[sub]++;
}

static int rec_cmp(const void *a, const void *b, void *arg)
{
    int nw = *(const int *)arg;
    const uint64_t *x = (const uint64_t *)a, *y = (const uint64_t *)b;
    for (int w = 0; w <= nw; w++) { /* key words, then J index */
        if (x[w] < y[w]) return -1;
        if (x[w] > y[w]) return 1;
    }
    return 0;
}

typedef struct {
    nsum e, s2;
    double min_den;
    int64_t na, ncon, ntiny;
    uint64_t d0, d1;
} sub_acc;

static int topk_entry_cmp(const void *a, const void *b, void *arg)
{
    /* entries are indices into a topk; best first */
    const topk *t = (const topk *)arg;
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    if (worse(t, t->e[i], t->key + i * t->nw, t->e[j], t->key + j * t->nw)) return 1;
    if (worse(t, t->e[j], t->key + j * t->nw, t->e[i], t->key + i * t->nw)) return -1;
    return 0;
}

/*
 * Full sweep.  Outputs (any pointer may be NULL):
 *   sel_dets [k][2][nint], sel_e [k], sel_num [k]: the selection, best first;
 *   eps_by_rank, na_by_rank, ncon_by_rank [ndet]: per-generator eps_I, |A_I|,
 *     connections, indexed by generator rank;
 *   rank_of [ndet]: generator rank of each input determinant.
 * mem_budget_bytes bounds the pair records held at once (0: 4 GiB).
 * Returns 0, or a negative validation code.
 */
int or_sweep(const or_ham *H, int64_t ndet, const uint64_t *dets, const double *coefs, double e0,
             int64_t k, uint64_t *sel_dets, double *sel_e, double *sel_num, double *eps_by_rank,
             int64_t *na_by_rank, int64_t *ncon_by_rank, int64_t *rank_of_out, or_result *res,
             int nthreads, int64_t mem_budget_bytes)
{
    int nint = H->nint, nw = 2 * nint, stride = nw + 1;
    int rc = or_validate(H, ndet, dets);
    memset(res, 0, sizeof(*res));
    res->min_abs_den = INFINITY;
    if (rc) return rc;
    if (k < 0) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int64_t *rank_of = (int64_t *)malloc(sizeof(int64_t) * (ndet > 0 ? ndet : 1));
    or_ranks(ndet, coefs, rank_of);
    if (rank_of_out) memcpy(rank_of_out, rank_of, sizeof(int64_t) * ndet);

    uint64_t *srt = (uint64_t *)malloc(sizeof(uint64_t) * nw * (ndet > 0 ? ndet : 1));
    memcpy(srt, dets, sizeof(uint64_t) * nw * ndet);
    g_nw_sort = nw;
    qsort(srt, ndet, sizeof(uint64_t) * nw, key_qcmp);

    if (mem_budget_bytes <= 0) mem_budget_bytes = (int64_t)4 << 30;
    double total = (double)ndet * (double)or_n_substitutions(H) * stride * 8.0;
    int nparts = (int)ceil(total / (double)mem_budget_bytes);
    if (nparts < 1) nparts = 1;

    /* per sub-bucket accumulators (fixed count, so the result does not
     * depend on the number of threads) */
    sub_acc *acc = (sub_acc *)calloc(OR_NSUB, sizeof(sub_acc));
    for (int s = 0; s < OR_NSUB; s++) acc[s].min_den = INFINITY;
    double *eps_sub = (double *)calloc((size_t)OR_NSUB * (ndet > 0 ? ndet : 1), sizeof(double));
    int64_t *na_sub = (int64_t *)calloc((size_t)OR_NSUB * (ndet > 0 ? ndet : 1), sizeof(int64_t));
    int64_t *nc_sub = (int64_t *)calloc((size_t)OR_NSUB * (ndet > 0 ? ndet : 1), sizeof(int64_t));
    topk *tk = (topk *)malloc(sizeof(topk) * OR_NSUB);
    for (int s = 0; s < OR_NSUB; s++) topk_init(&tk[s], nw, k);

    /* per-thread, per-sub-bucket record buffers */
    pair_ctx *ctx = (pair_ctx *)calloc(nthreads, sizeof(pair_ctx));
    for (int t = 0; t < nthreads; t++) {
        ctx[t].H = H; ctx[t].nw = nw; ctx[t].stride = stride; ctx[t].nparts = nparts;
        ctx[t].cnt = (int64_t *)calloc(OR_NSUB, sizeof(int64_t));
        ctx[t].cap = (int64_t *)calloc(OR_NSUB, sizeof(int64_t));
        ctx[t].buf = (uint64_t **)calloc(OR_NSUB, sizeof(uint64_t *));
    }

    for (int part = 0; part < nparts; part++) {
        for (int t = 0; t < nthreads; t++) {
            ctx[t].part = part;
            for (int s = 0; s < OR_NSUB; s++) ctx[t].cnt[s] = 0;
        }
        /* 1. enumerate every (J, alpha) pair whose alpha falls in this part */
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
        for (int64_t j = 0; j < ndet; j++) {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            ctx[t].jidx = j;
            for_each_substitution(H, dets + j * nw, pair_emit, &ctx[t]);
        }
        /* 2. per sub-bucket: gather, sort by (alpha, J), evaluate groups */
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
        for (int s = 0; s < OR_NSUB; s++) {
            int64_t n = 0;
            for (int t = 0; t < nthreads; t++) n += ctx[t].cnt[s];
            if (n == 0) continue;
            uint64_t *rec = (uint64_t *)malloc(sizeof(uint64_t) * stride * n);
            int64_t off = 0;
            for (int t = 0; t < nthreads; t++) {
                memcpy(rec + off * stride, ctx[t].buf[s], sizeof(uint64_t) * stride * ctx[t].cnt[s]);
                off += ctx[t].cnt[s];
            }
            int nwl = nw;
            qsort_r(rec, n, sizeof(uint64_t) * stride, rec_cmp, &nwl);
            sub_acc *a = &acc[s];
            for (int64_t g0 = 0; g0 < n;) {
                int64_t g1 = g0 + 1;
                while (g1 < n && keycmp(rec + g1 * stride, rec + g0 * stride, nw) == 0) g1++;
                const uint64_t *alpha = rec + g0 * stride;
                if (!is_member(srt, ndet, nw, alpha)) {
                    nsum A = {0.0, 0.0};
                    int64_t gen = ndet;
                    for (int64_t r = g0; r < g1; r++) {
                        int64_t j = (int64_t)rec[r * stride + nw];
                        nsum_add(&A, coefs[j] * or_hij(H, dets + j * nw, alpha));
                        if (rank_of[j] < gen) gen = rank_of[j];
                    }
                    double Av = nsum_get(&A);
                    double haa = or_diag(H, alpha);
                    double D = e0 - haa;
                    double e = Av * Av / D;
                    nsum_add(&a->e, e);
                    nsum_add(&a->s2, (Av / D) * (Av / D));
                    if (fabs(D) < a->min_den) a->min_den = fabs(D);
                    a->na++;
                    a->ncon += g1 - g0;
                    if (fabs(Av) < 1e-14) a->ntiny++;
                    uint64_t hk = or_key_hash(nw, alpha);
                    a->d0 += hk;
                    a->d1 ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
                    eps_sub[(size_t)s * ndet + gen] += e;
                    na_sub[(size_t)s * ndet + gen] += 1;
                    nc_sub[(size_t)s * ndet + gen] += g1 - g0;
                    topk_push(&tk[s], e, Av, alpha);
                }
                g0 = g1;
            }
            free(rec);
        }
    }

    /* combine in sub-bucket order */
    nsum E = {0, 0}, S2 = {0, 0};
    for (int s = 0; s < OR_NSUB; s++) {
        nsum_add(&E, nsum_get(&acc[s].e));
        nsum_add(&S2, nsum_get(&acc[s].s2));
        if (acc[s].min_den < res->min_abs_den) res->min_abs_den = acc[s].min_den;
        res->n_perturbers += acc[s].na;
        res->n_connections += acc[s].ncon;
        res->n_tiny += acc[s].ntiny;
        res->digest[0] += acc[s].d0;
        res->digest[1] ^= acc[s].d1;
    }
    res->e_pt2 = nsum_get(&E);
    res->sum_e_over_d = nsum_get(&S2);
    for (int64_t g = 0; g < ndet; g++) {
        double v = 0.0;
        int64_t x = 0, y = 0;
        for (int s = 0; s < OR_NSUB; s++) {
            v += eps_sub[(size_t)s * ndet + g];
            x += na_sub[(size_t)s * ndet + g];
            y += nc_sub[(size_t)s * ndet + g];
        }
        if (eps_by_rank) eps_by_rank[g] = v;
        if (na_by_rank) na_by_rank[g] = x;
        if (ncon_by_rank) ncon_by_rank[g] = y;
    }

    /* merge the bounded selections */
    topk all;
    int64_t ntot = 0;
    for (int s = 0; s < OR_NSUB; s++) ntot += tk[s].n;
    topk_init(&all, nw, ntot > 0 ? ntot : 1);
    for (int s = 0; s < OR_NSUB; s++)
        for (int64_t i = 0; i < tk[s].n; i++) {
            all.e[all.n] = tk[s].e[i];
            all.num[all.n] = tk[s].num[i];
            memcpy(all.key + all.n * nw, tk[s].key + i * nw, 8 * nw);
            all.n++;
        }
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (all.n > 0 ? all.n : 1));
    for (int64_t i = 0; i < all.n; i++) ord[i] = i;
    qsort_r(ord, all.n, sizeof(int64_t), topk_entry_cmp, &all);
    int64_t nsel = all.n < k ? all.n : k;
    for (int64_t i = 0; i < nsel; i++) {
        if (sel_dets) memcpy(sel_dets + i * nw, all.key + ord[i] * nw, 8 * nw);
        if (sel_e) sel_e[i] = all.e[ord[i]];
        if (sel_num) sel_num[i] = all.num[ord[i]];
    }
    res->n_selected = nsel;

    free(ord);
    topk_free(&all);
    for (int s = 0; s < OR_NSUB; s++) topk_free(&tk[s]);
    free(tk);
    for (int t = 0; t < nthreads; t++) {
        for (int s = 0; s < OR_NSUB; s++) free(ctx[t].buf[s]);
        free(ctx[t].buf); free(ctx[t].cnt); free(ctx[t].cap);
    }
    free(ctx);
    free(eps_sub); free(na_sub); free(nc_sub); free(acc);
    free(srt); free(rank_of);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* or_generator: the per-generator definition, for one generator.            */
/* ------------------------------------------------------------------------ */

/*
 * Generator of rank g (in the order of or_ranks).  Outputs eps_I, |A_I|,
 * connections of I, the sum of A^2/D^2 and the digest of A_I.  If cap > 0,
 * the first cap perturbers of I (in substitution order) are written to
 * out_dets / out_e.  Returns 0 or a negative code.
 */
int or_generator(const or_ham *H, int64_t ndet, const uint64_t *dets, const double *coefs, double e0,
                 int64_t g, double *eps, int64_t *na, int64_t *ncon, double *s2, uint64_t *digest,
                 int64_t cap, uint64_t *out_dets, double *out_e, int nthreads)
{
    int nint = H->nint, nw = 2 * nint;
    if (g < 0 || g >= ndet) return -1;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int64_t *rank_of = (int64_t *)malloc(sizeof(int64_t) * ndet);
    or_ranks(ndet, coefs, rank_of);
    int64_t gi = -1;
    for (int64_t i = 0; i < ndet; i++)
        if (rank_of[i] == g) gi = i;
    const uint64_t *I = dets + gi * nw;
    /* internal determinants within degree 4 of I */
    int64_t nf = 0;
    int64_t *F = (int64_t *)malloc(sizeof(int64_t) * ndet);
    for (int64_t j = 0; j < ndet; j++)
        if (or_degree(nint, I, dets + j * nw) <= 4) F[nf++] = j;
    int64_t nc = or_n_substitutions(H);
    uint64_t *cand = (uint64_t *)malloc(sizeof(uint64_t) * nw * (nc > 0 ? nc : 1));
    or_substitutions(H, I, nc, cand);
    double *ev = (double *)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    double *qv = (double *)malloc(sizeof(double) * (nc > 0 ? nc : 1));
    int64_t *cv = (int64_t *)malloc(sizeof(int64_t) * (nc > 0 ? nc : 1));
    char *keep = (char *)calloc(nc > 0 ? nc : 1, 1);
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
    for (int64_t c = 0; c < nc; c++) {
        const uint64_t *alpha = cand + c * nw;
        int skip = !in_target(H, alpha);
        int64_t con = 0;
        nsum A = {0.0, 0.0};
        for (int64_t f = 0; f < nf && !skip; f++) {
            const uint64_t *J = dets + F[f] * nw;
            int d = or_degree(nint, J, alpha);
            if (d == 0) skip = 1;                         /* alpha is internal */
            else if (d <= 2) {
                if (rank_of[F[f]] < g) skip = 1;          /* belongs to an earlier generator */
                else { nsum_add(&A, coefs[F[f]] * or_hij(H, J, alpha)); con++; }
            }
        }
        if (!skip) {
            double Av = nsum_get(&A);
            double D = e0 - or_diag(H, alpha);
            ev[c] = Av * Av / D;
            qv[c] = (Av / D) * (Av / D);
            cv[c] = con;
            keep[c] = 1;
        }
    }
    nsum E = {0, 0}, S = {0, 0};
    int64_t n = 0, conn = 0, nout = 0;
    uint64_t d0 = 0, d1 = 0;
    for (int64_t c = 0; c < nc; c++) {
        if (!keep[c]) continue;
        nsum_add(&E, ev[c]);
        nsum_add(&S, qv[c]);
        n++;
        conn += cv[c];
        uint64_t hk = or_key_hash(nw, cand + c * nw);
        d0 += hk;
        d1 ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
        if (nout < cap) {
            if (out_dets) memcpy(out_dets + nout * nw, cand + c * nw, 8 * nw);
            if (out_e) out_e[nout] = ev[c];
            nout++;
        }
    }
    if (eps) *eps = nsum_get(&E);
    if (s2) *s2 = nsum_get(&S);
    if (na) *na = n;
    if (ncon) *ncon = conn;
    if (digest) { digest[0] = d0; digest[1] = d1; }
    free(keep); free(cv); free(qv); free(ev); free(cand); free(F); free(rank_of);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* One perturber at a time: A_alpha, H_aa, and whether alpha is external.    */
/* ------------------------------------------------------------------------ */

/* A_alpha = sum_J c_J <J|H|alpha> over all internal J (direct sum);
 * returns 1 if alpha is internal, else 0.  Also reports the lowest rank of a
 * connected J (-1 if none) and the number of connected J. */
int or_alpha(const or_ham *H, int64_t ndet, const uint64_t *dets, const double *coefs,
             const uint64_t *alpha, double *A, double *haa, int64_t *gen_rank, int64_t *ncon)
{
    int nint = H->nint, nw = 2 * nint;
    int64_t *rank_of = (int64_t *)malloc(sizeof(int64_t) * (ndet > 0 ? ndet : 1));
    or_ranks(ndet, coefs, rank_of);
    nsum s = {0, 0};
    int internal = 0;
    int64_t gen = -1, con = 0;
    for (int64_t j = 0; j < ndet; j++) {
        int d = or_degree(nint, dets + j * nw, alpha);
        if (d == 0) internal = 1;
        else if (d <= 2) {
            nsum_add(&s, coefs[j] * or_hij(H, dets + j * nw, alpha));
            con++;
            if (gen < 0 || rank_of[j] < gen) gen = rank_of[j];
        }
    }
    *A = nsum_get(&s);
    *haa = or_diag(H, alpha);
    *gen_rank = gen;
    *ncon = con;
    free(rank_of);
    return internal;
}

/* ------------------------------------------------------------------------ */
/* Several states at once (Sec. "Selected CI", the multi-state criterion of  */
/* Angeli et al.).  One PT2 per state k,                                     */
/*   E_PT2,k = sum_alpha A_k^2 / (E0_k - H_aa),  A_k = <Psi0_k|H|alpha>,     */
/* and the selection criterion                                               */
/*   e~_alpha = sum_k c_alpha,k A_k / max_I c_Ik^2,                          */
/*   c_alpha,k = A_k / (E0_k - H_aa).                                        */
/* Plain definition: the external space is the sorted, de-duplicated set of  */
/* the single and double substitutions of every internal determinant, less   */
/* the internal ones (and those outside the target space); for each alpha    */
/* every internal J is tested and A_k = sum_J c_Jk <J|H|alpha> is formed     */
/* directly.  No generator order enters.                                     */
/* ------------------------------------------------------------------------ */

#define OR_MAXST 8

/*
 * coefs: [nst][ndet] (state k's coefficients at coefs + k*ndet); e0: [nst].
 * Outputs: e_pt2[nst], sum_e_over_d[nst]; res holds the counts, the digest,
 * min |E0_k - H_aa| over alpha and k, n_tiny (|A_0| < 1e-14), and e_pt2 /
 * sum_e_over_d of state 0.  The selection (k entries, best first by |e~|,
 * ties by key) goes to sel_dets, sel_crit (e~) and sel_num (A_0).
 * shard_count > 0 keeps only the alpha whose generator (the lowest-ranked
 * connected J, ranks by state 0's c^2: the canonical rule of Eqs. calpha and
 * edetstoch) has a rank equal to shard_index modulo shard_count.
 * Returns 0, -1 (bad sizes, a state with no nonzero coefficient) or a
 * validation code of or_validate.
 */
int or_states(const or_ham *H, int64_t ndet, const uint64_t *dets, int nst, const double *coefs,
              const double *e0, int64_t k, uint64_t *sel_dets, double *sel_crit, double *sel_num,
              double *e_pt2, double *sum_e_over_d, or_result *res, int nthreads, int shard_index,
              int shard_count)
{
    int nint = H->nint, nw = 2 * nint;
    memset(res, 0, sizeof(*res));
    res->min_abs_den = INFINITY;
    if (nst < 1 || nst > OR_MAXST || k < 0) return -1;
    if (shard_count < 0 || (shard_count > 0 && (shard_index < 0 || shard_index >= shard_count))) return -1;
    int rc = or_validate(H, ndet, dets);
    if (rc) return rc;
    for (int s = 0; s < nst; s++) { e_pt2[s] = 0.0; sum_e_over_d[s] = 0.0; }
    if (ndet == 0) return 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    /* weights 1 / max_I c_Ik^2 */
    double w[OR_MAXST];
    for (int s = 0; s < nst; s++) {
        double m = 0.0;
        for (int64_t i = 0; i < ndet; i++) {
            double c = coefs[(size_t)s * ndet + i];
            if (c * c > m) m = c * c;
        }
        if (!(m > 0.0)) return -1;
        w[s] = 1.0 / m;
    }
    /* every substitution of every internal determinant, sorted */
    int64_t nsub = or_n_substitutions(H), ncand = ndet * nsub;
    uint64_t *cand = (uint64_t *)malloc(sizeof(uint64_t) * nw * (ncand > 0 ? ncand : 1));
    for (int64_t i = 0; i < ndet; i++) or_substitutions(H, dets + i * nw, nsub, cand + i * nsub * nw);
    uint64_t *srt = (uint64_t *)malloc(sizeof(uint64_t) * nw * ndet);
    memcpy(srt, dets, sizeof(uint64_t) * nw * ndet);
    g_nw_sort = nw;
    qsort(cand, ncand, sizeof(uint64_t) * nw, key_qcmp);
    qsort(srt, ndet, sizeof(uint64_t) * nw, key_qcmp);
    /* distinct, external, inside the target space */
    int64_t m = 0;
    for (int64_t i = 0; i < ncand; i++) {
        const uint64_t *a = cand + i * nw;
        if (i > 0 && keycmp(a, cand + (i - 1) * nw, nw) == 0) continue;
        if (is_member(srt, ndet, nw, a) || !in_target(H, a)) continue;
        if (m != i) memcpy(cand + m * nw, a, sizeof(uint64_t) * nw);
        m++;
    }
    /* A_k, H_aa and the generator rank per alpha */
    double *A = (double *)calloc((size_t)(m > 0 ? m : 1) * nst, sizeof(double));
    double *haa = (double *)malloc(sizeof(double) * (m > 0 ? m : 1));
    int64_t *nc = (int64_t *)calloc((size_t)(m > 0 ? m : 1), sizeof(int64_t));
    int64_t *gen = (int64_t *)malloc(sizeof(int64_t) * (m > 0 ? m : 1));
    int64_t *rank_of = (int64_t *)malloc(sizeof(int64_t) * ndet);
    or_ranks(ndet, coefs, rank_of);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nthreads)
#endif
    for (int64_t a = 0; a < m; a++) {
        const uint64_t *al = cand + a * nw;
        nsum acc[OR_MAXST];
        for (int s = 0; s < nst; s++) { acc[s].s = 0.0; acc[s].c = 0.0; }
        int64_t n = 0, g = -1;
        for (int64_t j = 0; j < ndet; j++) {
            const uint64_t *J = dets + j * nw;
            if (or_degree(nint, J, al) > 2) continue;
            double v = or_hij(H, J, al);
            for (int s = 0; s < nst; s++) nsum_add(&acc[s], coefs[(size_t)s * ndet + j] * v);
            n++;
            if (g < 0 || rank_of[j] < g) g = rank_of[j];
        }
        for (int s = 0; s < nst; s++) A[(size_t)a * nst + s] = nsum_get(&acc[s]);
        haa[a] = or_diag(H, al);
        nc[a] = n;
        gen[a] = g;
    }
    /* totals and the selection, in alpha order */
    nsum E[OR_MAXST], S2[OR_MAXST];
    for (int s = 0; s < nst; s++) { E[s].s = E[s].c = 0.0; S2[s].s = S2[s].c = 0.0; }
    topk tk;
    topk_init(&tk, nw, k > 0 ? k : 1);
    tk.k = k;
    for (int64_t a = 0; a < m; a++) {
        const uint64_t *al = cand + a * nw;
        if (shard_count > 0 && gen[a] % shard_count != shard_index) continue;
        double crit = 0.0;
        for (int s = 0; s < nst; s++) {
            double Av = A[(size_t)a * nst + s], D = e0[s] - haa[a];
            double e = Av * Av / D, q = Av / D;
            nsum_add(&E[s], e);
            nsum_add(&S2[s], q * q);
            crit += w[s] * e;   /* c_alpha,k A_k / max_I c_Ik^2 */
            if (fabs(D) < res->min_abs_den) res->min_abs_den = fabs(D);
        }
        res->n_perturbers++;
        res->n_connections += nc[a];
        if (fabs(A[(size_t)a * nst]) < 1e-14) res->n_tiny++;
        uint64_t hk = or_key_hash(nw, al);
        res->digest[0] += hk;
        res->digest[1] ^= splitmix64(hk ^ 0x243F6A8885A308D3ull);
        topk_push(&tk, crit, A[(size_t)a * nst], al);
    }
    for (int s = 0; s < nst; s++) { e_pt2[s] = nsum_get(&E[s]); sum_e_over_d[s] = nsum_get(&S2[s]); }
    res->e_pt2 = e_pt2[0];
    res->sum_e_over_d = sum_e_over_d[0];
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (tk.n > 0 ? tk.n : 1));
    for (int64_t i = 0; i < tk.n; i++) ord[i] = i;
    qsort_r(ord, tk.n, sizeof(int64_t), topk_entry_cmp, &tk);
    for (int64_t i = 0; i < tk.n; i++) {
        if (sel_dets) memcpy(sel_dets + i * nw, tk.key + ord[i] * nw, 8 * nw);
        if (sel_crit) sel_crit[i] = tk.e[ord[i]];
        if (sel_num) sel_num[i] = tk.num[ord[i]];
    }
    res->n_selected = tk.n;
    free(ord);
    topk_free(&tk);
    free(A); free(haa); free(nc); free(gen); free(rank_of); free(cand); free(srt);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Sparse Hamiltonian over the internal space (upper triangle, diagonal      */
/* included), for the diagonalisation that produces Psi0.                    */
/* ------------------------------------------------------------------------ */

/* count pass (out == NULL) or fill pass; returns nnz */
int64_t or_hamiltonian(const or_ham *H, int64_t ndet, const uint64_t *dets, int64_t cap,
                       int64_t *rows, int64_t *cols, double *vals, int nthreads)
{
    int nint = H->nint, nw = 2 * nint;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int64_t *cnt = (int64_t *)calloc(ndet + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
    for (int64_t i = 0; i < ndet; i++) {
        int64_t c = 0;
        for (int64_t j = i; j < ndet; j++)
            if (or_degree(nint, dets + i * nw, dets + j * nw) <= 2) c++;
        cnt[i + 1] = c;
    }
    for (int64_t i = 0; i < ndet; i++) cnt[i + 1] += cnt[i];
    int64_t nnz = cnt[ndet];
    if (rows && nnz <= cap) {
#pragma omp parallel for schedule(dynamic, 16) num_threads(nthreads)
        for (int64_t i = 0; i < ndet; i++) {
            int64_t o = cnt[i];
            for (int64_t j = i; j < ndet; j++)
                if (or_degree(nint, dets + i * nw, dets + j * nw) <= 2) {
                    rows[o] = i;
                    cols[o] = j;
                    vals[o] = or_hij(H, dets + i * nw, dets + j * nw);
                    o++;
                }
        }
    }
    free(cnt);
    return nnz;
}

int or_max_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* ------------------------------------------------------------------------ */
/* Gradient of E_PT2 with respect to the integrals (Psi0 and E0 fixed).      */
/*                                                                           */
/* E_PT2 = sum_alpha A_alpha^2 / D_alpha, A_alpha = sum_J c_J <J|H|alpha>,   */
/* D_alpha = E0 - <alpha|H|alpha> (Eqs. e2, PT2).  Every matrix element is   */
/* linear in h and in the integrals (Eqs. Hij), so                           */
/*   dE/dtheta = sum_alpha [ (2 A/D) sum_J c_J d<J|H|alpha>/dtheta           */
/*                           + (A/D)^2 d<alpha|H|alpha>/dtheta ],            */
/*   dE/dE0    = - sum_alpha A^2/D^2.                                        */
/* Conventions: deri[i] is the derivative with respect to packed entry i;    */
/* dh is symmetric with dh[p][q] = dh[q][p] = 1/2 dE/du_pq for p != q, where */
/* u_pq moves h_pq and h_qp together, and dh[p][p] = dE/dh_pp.               */
/* ------------------------------------------------------------------------ */

/* add w * d<I|H|I>/dtheta */
static void diag_grad(const or_ham *H, const uint64_t *d, double w, double *dh, double *deri)
{
    int norb = H->norb, nint = H->nint;
    int occ[2 * OR_MAXORB], spin[2 * OR_MAXORB], n = 0;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++)
            if (getbit(d, nint, s, p)) { occ[n] = p; spin[n] = s; n++; }
    for (int i = 0; i < n; i++) dh[occ[i] * norb + occ[i]] += w;
    for (int i = 0; i < n; i++)
        for (int j = i + 1; j < n; j++) {
            deri[tri(tri(occ[i], occ[i]), tri(occ[j], occ[j]))] += w;
            if (spin[i] == spin[j]) deri[tri(tri(occ[i], occ[j]), tri(occ[j], occ[i]))] -= w;
        }
}

/* add w * d<I|H|J>/dtheta (same case analysis as or_hij) */
static void hij_grad(const or_ham *H, const uint64_t *I, const uint64_t *Jd, double w, double *dh, double *deri)
{
    int norb = H->norb, nint = H->nint;
    int deg = or_degree(nint, I, Jd);
    if (deg == 0) { diag_grad(H, I, w, dh, deri); return; }
    if (deg > 2) return;
    int hs[2], ho[2], ps[2], po[2], nh = 0, np = 0;
    for (int s = 0; s < 2; s++)
        for (int p = 0; p < norb; p++) {
            int a = getbit(I, nint, s, p), b = getbit(Jd, nint, s, p);
            if (a && !b) { hs[nh] = s; ho[nh] = p; nh++; }
            if (!a && b) { ps[np] = s; po[np] = p; np++; }
        }
    if (deg == 1) {
        int s = hs[0], h = ho[0], p = po[0];
        double ws = w * phase_single(I, nint, s, h, p);
        dh[h * norb + p] += 0.5 * ws;
        dh[p * norb + h] += 0.5 * ws;
        for (int t = 0; t < 2; t++)
            for (int i = 0; i < norb; i++) {
                if (!getbit(I, nint, t, i)) continue;
                deri[tri(tri(h, p), tri(i, i))] += ws;
                if (t == s) deri[tri(tri(h, i), tri(i, p))] -= ws;
            }
        return;
    }
    uint64_t I1[2 * OR_MAXNINT];
    memcpy(I1, I, sizeof(uint64_t) * 2 * nint);
    double ph = phase_single(I, nint, hs[0], ho[0], po[0]);
    clrbit(I1, nint, hs[0], ho[0]);
    setbit(I1, nint, ps[0], po[0]);
    ph *= phase_single(I1, nint, hs[1], ho[1], po[1]);
    deri[tri(tri(ho[0], po[0]), tri(ho[1], po[1]))] += w * ph;
    if (hs[0] == hs[1]) deri[tri(tri(ho[0], po[1]), tri(ho[1], po[0]))] -= w * ph;
}

/* Plain-definition gradient (pairs grouped by alpha, as in or_sweep).
 * dh[norb*norb], deri[P], *de0 and *e_pt2 are overwritten. */
int or_gradient(const or_ham *H, int64_t ndet, const uint64_t *dets, const double *coefs, double e0,
                double *dh, double *deri, double *de0, double *e_pt2, int nthreads, int64_t mem_budget_bytes)
{
    int nint = H->nint, nw = 2 * nint, stride = nw + 1, norb = H->norb;
    int rc = or_validate(H, ndet, dets);
    if (rc) return rc;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#else
    nthreads = 1;
#endif
    int64_t m = (int64_t)norb * (norb + 1) / 2, P = m * (m + 1) / 2;
    uint64_t *srt = (uint64_t *)malloc(sizeof(uint64_t) * nw * (ndet > 0 ? ndet : 1));
    memcpy(srt, dets, sizeof(uint64_t) * nw * ndet);
    g_nw_sort = nw;
    qsort(srt, ndet, sizeof(uint64_t) * nw, key_qcmp);
    if (mem_budget_bytes <= 0) mem_budget_bytes = (int64_t)4 << 30;
    double total = (double)ndet * (double)or_n_substitutions(H) * stride * 8.0;
    int nparts = (int)ceil(total / (double)mem_budget_bytes);
    if (nparts < 1) nparts = 1;
    /* per sub-bucket gradient arrays, summed in sub-bucket order at the end */
    double *gh = (double *)calloc((size_t)OR_NSUB * norb * norb, sizeof(double));
    double *ge = (double *)calloc((size_t)OR_NSUB * P, sizeof(double));
    nsum *ee = (nsum *)calloc(OR_NSUB, sizeof(nsum));
    nsum *e0s = (nsum *)calloc(OR_NSUB, sizeof(nsum));
    pair_ctx *ctx = (pair_ctx *)calloc(nthreads, sizeof(pair_ctx));
    for (int t = 0; t < nthreads; t++) {
        ctx[t].H = H; ctx[t].nw = nw; ctx[t].stride = stride; ctx[t].nparts = nparts;
        ctx[t].cnt = (int64_t *)calloc(OR_NSUB, sizeof(int64_t));
        ctx[t].cap = (int64_t *)calloc(OR_NSUB, sizeof(int64_t));
        ctx[t].buf = (uint64_t **)calloc(OR_NSUB, sizeof(uint64_t *));
    }
    for (int part = 0; part < nparts; part++) {
        for (int t = 0; t < nthreads; t++) {
            ctx[t].part = part;
            for (int s = 0; s < OR_NSUB; s++) ctx[t].cnt[s] = 0;
        }
#pragma omp parallel for schedule(dynamic, 4) num_threads(nthreads)
        for (int64_t j = 0; j < ndet; j++) {
            int t = 0;
#ifdef _OPENMP
            t = omp_get_thread_num();
#endif
            ctx[t].jidx = j;
            for_each_substitution(H, dets + j * nw, pair_emit, &ctx[t]);
        }
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
        for (int s = 0; s < OR_NSUB; s++) {
            int64_t n = 0;
            for (int t = 0; t < nthreads; t++) n += ctx[t].cnt[s];
            if (n == 0) continue;
            uint64_t *rec = (uint64_t *)malloc(sizeof(uint64_t) * stride * n);
            int64_t off = 0;
            for (int t = 0; t < nthreads; t++) {
                memcpy(rec + off * stride, ctx[t].buf[s], sizeof(uint64_t) * stride * ctx[t].cnt[s]);
                off += ctx[t].cnt[s];
            }
            int nwl = nw;
            qsort_r(rec, n, sizeof(uint64_t) * stride, rec_cmp, &nwl);
            double *dhs = gh + (size_t)s * norb * norb;
            double *des = ge + (size_t)s * P;
            for (int64_t g0 = 0; g0 < n;) {
                int64_t g1 = g0 + 1;
                while (g1 < n && keycmp(rec + g1 * stride, rec + g0 * stride, nw) == 0) g1++;
                const uint64_t *alpha = rec + g0 * stride;
                if (!is_member(srt, ndet, nw, alpha)) {
                    nsum A = {0.0, 0.0};
                    for (int64_t r = g0; r < g1; r++) {
                        int64_t j = (int64_t)rec[r * stride + nw];
                        nsum_add(&A, coefs[j] * or_hij(H, dets + j * nw, alpha));
                    }
                    double Av = nsum_get(&A);
                    double D = e0 - or_diag(H, alpha);
                    double q = Av / D;
                    nsum_add(&ee[s], Av * Av / D);
                    nsum_add(&e0s[s], -q * q);
                    for (int64_t r = g0; r < g1; r++) {
                        int64_t j = (int64_t)rec[r * stride + nw];
                        /* d<J|H|alpha> = d<alpha|H|J> for real symmetric integrals */
                        hij_grad(H, dets + j * nw, alpha, 2.0 * q * coefs[j], dhs, des);
                    }
                    diag_grad(H, alpha, q * q, dhs, des);
                }
                g0 = g1;
            }
            free(rec);
        }
    }
    nsum E = {0, 0}, E0 = {0, 0};
    for (int s = 0; s < OR_NSUB; s++) {
        nsum_add(&E, nsum_get(&ee[s]));
        nsum_add(&E0, nsum_get(&e0s[s]));
    }
    *e_pt2 = nsum_get(&E);
    *de0 = nsum_get(&E0);
    for (int64_t i = 0; i < (int64_t)norb * norb; i++) {
        double v = 0.0;
        for (int s = 0; s < OR_NSUB; s++) v += gh[(size_t)s * norb * norb + i];
        dh[i] = v;
    }
    for (int64_t i = 0; i < P; i++) {
        double v = 0.0;
        for (int s = 0; s < OR_NSUB; s++) v += ge[(size_t)s * P + i];
        deri[i] = v;
    }
    for (int t = 0; t < nthreads; t++) {
        for (int s = 0; s < OR_NSUB; s++) free(ctx[t].buf[s]);
        free(ctx[t].buf); free(ctx[t].cnt); free(ctx[t].cap);
    }
    free(ctx); free(gh); free(ge); free(ee); free(e0s); free(srt);
    return 0;
}
