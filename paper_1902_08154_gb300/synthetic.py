"""Seeded synthetic inputs: Hamiltonians, determinant sets and coefficient vectors.

This module only draws random numbers and lays them out in the library's data
format. It holds none of the perturbation method's arithmetic (no matrix
elements, no energies, no selection), so both the CUDA path and the CPU oracle
can take their inputs from it.

Data format (shared by every consumer):

* ``h``: ``float64[norb, norb]``, symmetric one-electron integrals (p|h|q).
* ``eri``: ``float64[P]``, chemists' two-electron integrals (pq|rs) with the
  8-fold permutational symmetry of real orbitals, stored once per orbit.  With
  0-based orbitals, ``PQ = max(p,q)(max(p,q)+1)/2 + min(p,q)``, likewise ``RS``,
  and ``(pq|rs)`` sits at ``max(PQ,RS)(max(PQ,RS)+1)/2 + min(PQ,RS)``.  This is
  the compound triangular index of the paper's integral hash (Algorithm hash,
  Sec. "Storage of the two-electron integrals"), shifted to 0-based indices.
  ``P = M(M+1)/2`` with ``M = norb(norb+1)/2``.
* determinants: ``uint64[ndet, 2, nint]``; ``[:, 0]`` holds the spin-up string,
  ``[:, 1]`` the spin-down string; orbital p (0-based) is bit ``p % 64`` of word
  ``p // 64`` (Sec. "Internal representation of determinants");
  ``nint = (norb - 1) // 64 + 1``.

Recipe of the synthetic Hamiltonian (stands in for the paper's molecular
integrals, which are not available): numpy PCG64 generator seeded with
``seed``; draws in this order

1. the strict upper triangle of h, row-major, from N(0, 0.05^2);
2. h_pp = -2.0 + 0.15 p (no draw);
3. for each Cholesky vector L < rank: the upper triangle (diagonal included)
   of a symmetric B^L, row-major, from N(0,1) scaled by 0.3 r^(p+q), where
   r = exp(-0.1) rounded to a double and its powers are formed by repeated
   multiplication (so every platform gets the same bits);
4. (pq|rs) = sum_L B^L_pq B^L_rs, accumulated in L order with separate
   IEEE multiplies and adds.
"""
from __future__ import annotations

import hashlib
import math

import numpy as np

# exp(-0.1) rounded to the nearest double; written out so that no platform's
# libm enters the inputs.
DECAY = 0.9048374180359595


def nint_of(norb: int) -> int:
    return (norb - 1) // 64 + 1


def pair_count(norb: int) -> int:
    return norb * (norb + 1) // 2


def packed_len(norb: int) -> int:
    m = pair_count(norb)
    return m * (m + 1) // 2


def hamiltonian(norb: int, rank: int, seed: int):
    """Return (h, eri) for the seeded synthetic Hamiltonian described above."""
    rng = np.random.default_rng(seed)
    h = np.zeros((norb, norb), dtype=np.float64)
    iu = np.triu_indices(norb, 1)
    h[iu] = rng.normal(0.0, 0.05, size=iu[0].size)
    h = h + h.T
    h[np.arange(norb), np.arange(norb)] = -2.0 + 0.15 * np.arange(norb, dtype=np.float64)

    powers = np.empty(2 * norb, dtype=np.float64)
    acc = 1.0
    for k in range(2 * norb):
        powers[k] = acc
        acc = acc * DECAY
    # pair list in packed order: PQ = p(p+1)/2 + q, q <= p
    pp, qq = np.tril_indices(norb)
    scale = 0.3 * powers[pp + qq]
    iu0 = np.triu_indices(norb, 0)
    m = pp.size
    V = np.zeros((m, m), dtype=np.float64)
    for _ in range(rank):
        B = np.zeros((norb, norb), dtype=np.float64)
        B[iu0] = rng.standard_normal(iu0[0].size)
        B = np.triu(B) + np.triu(B, 1).T
        b = B[pp, qq] * scale
        V += np.multiply.outer(b, b)
    rows, cols = np.tril_indices(m)
    eri = np.ascontiguousarray(V[rows, cols])
    return h, eri


def hamiltonian_digest(h: np.ndarray, eri: np.ndarray) -> str:
    s = hashlib.sha256()
    s.update(np.ascontiguousarray(h, dtype=np.float64).tobytes())
    s.update(np.ascontiguousarray(eri, dtype=np.float64).tobytes())
    return s.hexdigest()


def occ_to_det(occ_up, occ_dn, norb: int) -> np.ndarray:
    """Pack two orbital lists into one determinant ``uint64[2, nint]``."""
    nint = nint_of(norb)
    d = np.zeros((2, nint), dtype=np.uint64)
    for s, occ in enumerate((occ_up, occ_dn)):
        for p in occ:
            d[s, p // 64] |= np.uint64(1) << np.uint64(p % 64)
    return d


def det_to_occ(det: np.ndarray, norb: int):
    out = []
    for s in range(2):
        occ = []
        for p in range(norb):
            if (int(det[s, p // 64]) >> (p % 64)) & 1:
                occ.append(p)
        out.append(occ)
    return out


def hf_det(norb: int, nalpha: int, nbeta: int) -> np.ndarray:
    """Lowest orbitals filled in each spin (the synthetic stand-in for HF)."""
    return occ_to_det(range(nalpha), range(nbeta), norb)


def random_excited_dets(norb, nalpha, nbeta, ndet, seed, max_level=4, include_hf=True):
    """Distinct determinants made by moving up to ``max_level`` electrons of
    the HF determinant to random virtual orbitals (a CIPSI-like shape: all
    determinants lie near HF).  Returns ``uint64[ndet, 2, nint]``."""
    rng = np.random.default_rng(seed)
    seen = set()
    dets = []
    if include_hf:
        d = hf_det(norb, nalpha, nbeta)
        seen.add(d.tobytes())
        dets.append(d)
    occ0 = [list(range(nalpha)), list(range(nbeta))]
    virt0 = [list(range(nalpha, norb)), list(range(nbeta, norb))]
    tries = 0
    while len(dets) < ndet:
        tries += 1
        if tries > 200 * ndet + 10000:
            raise ValueError("space too small for the requested number of determinants")
        level = int(rng.integers(1, max_level + 1))
        occ = [list(occ0[0]), list(occ0[1])]
        for _ in range(level):
            s = int(rng.integers(0, 2))
            if not occ[s] or len(occ[s]) == 0:
                continue
            h = occ[s][int(rng.integers(0, len(occ[s])))]
            free = [p for p in range(norb) if p not in occ[s]]
            if not free:
                continue
            p = free[int(rng.integers(0, len(free)))]
            occ[s].remove(h)
            occ[s].append(p)
        d = occ_to_det(sorted(occ[0]), sorted(occ[1]), norb)
        b = d.tobytes()
        if b in seen:
            continue
        seen.add(b)
        dets.append(d)
    return np.ascontiguousarray(np.stack(dets), dtype=np.uint64)


def random_coefs(ndet: int, seed: int, decay: float = 0.0) -> np.ndarray:
    """Unit-norm coefficient vector; entry i drawn from N(0,1) times
    ``exp(-decay * i)`` (a large first coefficient mimics a CI vector)."""
    rng = np.random.default_rng(seed)
    c = rng.standard_normal(ndet)
    if decay:
        c = c * np.exp(-decay * np.arange(ndet))
        c[0] = abs(c[0]) + 1.0
    return c / np.linalg.norm(c)


def all_dets(norb: int, nalpha: int, nbeta: int) -> np.ndarray:
    """Every determinant of the (nalpha, nbeta) space, in lexicographic order
    of (spin-up orbital tuple, spin-down orbital tuple)."""
    from itertools import combinations

    ups = list(combinations(range(norb), nalpha))
    dns = list(combinations(range(norb), nbeta))
    out = np.zeros((len(ups) * len(dns), 2, nint_of(norb)), dtype=np.uint64)
    i = 0
    for u in ups:
        du = occ_to_det(u, (), norb)[0]
        for d in dns:
            out[i, 0] = du
            out[i, 1] = occ_to_det((), d, norb)[1]
            i += 1
    return out


def n_singles_doubles(norb: int, nalpha: int, nbeta: int) -> int:
    """Number of single and double substitutions of one determinant."""
    va, vb = norb - nalpha, norb - nbeta
    singles = nalpha * va + nbeta * vb
    same = math.comb(nalpha, 2) * math.comb(va, 2) + math.comb(nbeta, 2) * math.comb(vb, 2)
    opp = nalpha * nbeta * va * vb
    return singles + same + opp


# ---------------------------------------------------------------------------
# The batched workload: many independent instances of uneven size.
# ---------------------------------------------------------------------------
def batch_specs(n=64, seed0=1000):
    """Instance i (seed seed0 + i): norb uniform in {24, 32, 48, 64, 96},
    n_alpha = n_beta uniform in 6..12, N_det = exp(U(ln 1e3, ln 5e4))
    rounded to a multiple of 8, Cholesky rank ceil(1.5 norb)."""
    out = []
    for i in range(n):
        rng = np.random.default_rng(seed0 + i)
        norb = int(rng.choice([24, 32, 48, 64, 96]))
        ne = int(rng.integers(6, 13))
        ndet = max(8, int(round(math.exp(rng.uniform(math.log(1e3), math.log(5e4))) / 8)) * 8)
        out.append(dict(norb=norb, nalpha=ne, nbeta=ne, ndet=ndet, rank=math.ceil(1.5 * norb), seed=seed0 + i))
    return out


def hamiltonian_fast(norb: int, rank: int, seed: int):
    """Same draws as ``hamiltonian`` but (pq|rs) formed by one matrix
    product; the last bits may depend on the BLAS of the machine, so inputs
    made this way are consumed on the machine that made them."""
    rng = np.random.default_rng(seed)
    h = np.zeros((norb, norb), dtype=np.float64)
    iu = np.triu_indices(norb, 1)
    h[iu] = rng.normal(0.0, 0.05, size=iu[0].size)
    h = h + h.T
    h[np.arange(norb), np.arange(norb)] = -2.0 + 0.15 * np.arange(norb, dtype=np.float64)
    powers = np.empty(2 * norb, dtype=np.float64)
    acc = 1.0
    for k in range(2 * norb):
        powers[k] = acc
        acc = acc * DECAY
    pp, qq = np.tril_indices(norb)
    scale = 0.3 * powers[pp + qq]
    iu0 = np.triu_indices(norb, 0)
    Bm = np.zeros((rank, pp.size))
    for L in range(rank):
        B = np.zeros((norb, norb), dtype=np.float64)
        B[iu0] = rng.standard_normal(iu0[0].size)
        B = np.triu(B) + np.triu(B, 1).T
        Bm[L] = B[pp, qq] * scale
    V = Bm.T @ Bm
    rows, cols = np.tril_indices(pp.size)
    return h, np.ascontiguousarray(V[rows, cols])


def excited_dets_fast(norb, nalpha, nbeta, ndet, seed, max_level=4):
    """Vectorised form of ``random_excited_dets`` for large spaces: HF first,
    then distinct determinants with 1..max_level electrons moved from the HF
    occupation to random virtual orbitals (order: first occurrence)."""
    rng = np.random.default_rng(seed)
    nint = nint_of(norb)
    hf = hf_det(norb, nalpha, nbeta)
    seen = {hf.tobytes()}
    dets = [hf]
    while len(dets) < ndet:
        m = 4 * (ndet - len(dets)) + 64
        level = rng.integers(1, max_level + 1, size=m)
        up = rng.binomial(level, 0.5)
        words = np.zeros((m, 2, nint), dtype=np.uint64)
        for s, (nocc, moves) in enumerate(((nalpha, up), (nbeta, level - up))):
            moves = np.minimum(moves, min(nocc, norb - nocc))
            occ = np.zeros((m, norb), dtype=bool)
            occ[:, :nocc] = True
            if nocc and norb - nocc:
                hole = np.argsort(rng.random((m, nocc)), axis=1)
                part = nocc + np.argsort(rng.random((m, norb - nocc)), axis=1)
                kmax = int(moves.max()) if m else 0
                for j in range(kmax):
                    sel = moves > j
                    r = np.nonzero(sel)[0]
                    occ[r, hole[r, j]] = False
                    occ[r, part[r, j]] = True
            for w in range(nint):
                block = occ[:, 64 * w: 64 * (w + 1)]
                bits = (block.astype(np.uint64) << np.arange(block.shape[1], dtype=np.uint64)).sum(axis=1)
                words[:, s, w] = bits.astype(np.uint64)
        for row in words:
            b = row.tobytes()
            if b not in seen:
                seen.add(b)
                dets.append(row.copy())
                if len(dets) == ndet:
                    break
    return np.ascontiguousarray(np.stack(dets), dtype=np.uint64)


def diagonal_lower_bound(h, eri, nel):
    """A number below <D|H|D> for every determinant D with nel electrons:
    nel * min h_pp + C(nel, 2) * min(0, min_pq ((pp|qq) - (pq|qp)))."""
    norb = h.shape[0]
    i = np.arange(norb)

    def tri(a, b):
        hi, lo = np.maximum(a, b), np.minimum(a, b)
        return hi * (hi + 1) // 2 + lo

    pq = tri(i[:, None], i[None, :])
    pp = tri(i, i)
    J = eri[tri(pp[:, None], pp[None, :])]
    K = eri[tri(pq, pq)]
    pair = min(0.0, float((J - K).min()), float(J.min()))
    return nel * float(np.diag(h).min()) + nel * (nel - 1) / 2 * pair


def batch_instance(spec):
    """Inputs of one batched instance: (h, eri, dets, coefs, e0).  E0 lies
    below every diagonal energy of the space (no singular denominators)."""
    h, eri = hamiltonian_fast(spec["norb"], spec["rank"], spec["seed"])
    dets = excited_dets_fast(spec["norb"], spec["nalpha"], spec["nbeta"], spec["ndet"], spec["seed"] + 1)
    coefs = random_coefs(len(dets), spec["seed"] + 2, decay=4.0 / len(dets))
    e0 = diagonal_lower_bound(h, eri, spec["nalpha"] + spec["nbeta"]) - 1.0
    return h, eri, dets, coefs, e0


# ---------------------------------------------------------------------------
# The 128-orbital workload (two words per spin) for the mixed-precision
# comparison: 14 + 14 electrons, Cholesky rank 192, 10^5 determinants.
# ---------------------------------------------------------------------------
CFG3 = dict(norb=128, nalpha=14, nbeta=14, rank=192, ndet=100000, seed=2)


def cfg3_instance(ndet=None, spec=CFG3):
    """Inputs (h, eri, dets, coefs, e0) of the 128-orbital workload.  Psi0 is
    HF plus distinct determinants with 1..4 electrons moved to random virtual
    orbitals, with coefficients decaying along the list (a stand-in for a
    CIPSI-grown Psi0, which is out of reach of the CPU oracle at this size);
    E0 lies below every diagonal energy of the space.  ``ndet`` keeps the
    first ndet determinants of the same list, with a coefficient vector of
    that length."""
    h, eri = hamiltonian_fast(spec["norb"], spec["rank"], spec["seed"])
    n = spec["ndet"] if ndet is None else min(int(ndet), spec["ndet"])
    dets = excited_dets_fast(spec["norb"], spec["nalpha"], spec["nbeta"], spec["ndet"], spec["seed"] + 1)[:n]
    coefs = random_coefs(n, spec["seed"] + 2, decay=4.0 / n)
    e0 = diagonal_lower_bound(h, eri, spec["nalpha"] + spec["nbeta"]) - 1.0
    return h, eri, dets, coefs, e0
