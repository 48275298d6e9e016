"""Pins of the CPU oracle to facts fixed by the paper and by mathematics.

None of these compares the oracle with itself: each compares it with an
independent construction (explicit second quantisation, a dense-matrix sum
over the whole external space, closed forms, brute-force bit counting) or
with an invariant of the definition.
"""
import itertools
import math

import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.sq_hamiltonian import dense_h, eri_full

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _ham(oracle_mod, norb, na, nb, rank, seed):
    h, eri = S.hamiltonian(norb, rank, seed)
    return oracle_mod.Hamiltonian(norb, na, nb, h, eri), h, eri


# ---------------------------------------------------------------------------
# P1: Slater-Condon rules vs explicit second quantisation (Eqs. Hij)
# ---------------------------------------------------------------------------
@pytest.mark.parametrize("norb,na,nb", [(6, 2, 2), (6, 3, 3), (7, 3, 2), (8, 2, 2)])
def test_slater_condon_matches_second_quantisation(oracle_mod, norb, na, nb):
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=norb + 2, seed=11 + norb + na)
    dets = S.all_dets(norb, na, nb)
    ref = dense_h(dets, h, eri, norb)
    got = np.array([[ham.hij(a, b) for b in dets] for a in dets])
    assert np.max(np.abs(got - ref)) < 1e-13
    # Hermiticity (Sec. "Matrix elements of the Hamiltonian": real MOs)
    assert np.max(np.abs(got - got.T)) < 1e-14
    # elements beyond double substitutions vanish
    deg = np.array([[ham.degree(a, b) for b in dets] for a in dets])
    assert np.all(got[deg > 2] == 0.0)


def test_slater_condon_across_word_boundary(oracle_mod):
    """Two 64-bit words per spin: orbitals straddling bit 63/64."""
    norb, na, nb = 68, 2, 2
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=6, seed=5)
    rng = np.random.default_rng(0)
    near = [0, 1, 61, 62, 63, 64, 65, 66, 67]
    dets, seen = [], set()
    while len(dets) < 40:
        up = tuple(sorted(rng.choice(near, na, replace=False)))
        dn = tuple(sorted(rng.choice(near, nb, replace=False)))
        if (up, dn) in seen:
            continue
        seen.add((up, dn))
        dets.append(S.occ_to_det(up, dn, norb))
    dets = np.stack(dets)
    ref = dense_h(dets, h, eri, norb)
    got = np.array([[ham.hij(a, b) for b in dets] for a in dets])
    assert np.max(np.abs(got - ref)) < 1e-13


# ---------------------------------------------------------------------------
# P2: E_PT2 against a dense-H sum over the whole external space (Eq. PT2)
# ---------------------------------------------------------------------------
def _dense_pt2(Hm, internal_idx, c, e0):
    n = Hm.shape[0]
    mask = np.ones(n, bool)
    mask[internal_idx] = False
    ext = np.nonzero(mask)[0]
    A = Hm[np.ix_(ext, internal_idx)] @ c
    D = e0 - np.diag(Hm)[ext]
    return ext, A, D


@pytest.mark.parametrize("norb,na,nb,nint_,seed", [(6, 2, 2, 30, 1), (7, 3, 2, 45, 2), (8, 2, 2, 60, 3)])
def test_pt2_matches_dense_external_sum(oracle_mod, norb, na, nb, nint_, seed):
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=norb + 3, seed=100 + seed)
    fci = S.all_dets(norb, na, nb)
    Hm = dense_h(fci, h, eri, norb)
    # CIPSI-like internal space: the lowest-diagonal determinants plus a few
    # random ones, so that E0 lies below the external diagonal energies
    rng = np.random.default_rng(seed)
    low = list(np.argsort(np.diag(Hm), kind="stable")[: nint_ - 5])
    rest = [i for i in range(len(fci)) if i not in set(low)]
    idx = np.sort(np.array(low + list(rng.choice(rest, 5, replace=False))))
    w, v = np.linalg.eigh(Hm[np.ix_(idx, idx)])
    c, e0 = v[:, 0], w[0]
    ext, A, D = _dense_pt2(Hm, idx, c, e0)
    e_dense = A * A / D
    connected = np.any(Hm[np.ix_(ext, idx)] != 0.0, axis=1)
    n_ext = int(connected.sum())

    dets = fci[idx]
    out = ham.sweep(dets, c, e0, k=len(fci))
    assert abs(out["e_pt2"] - e_dense.sum()) < 1e-12
    assert out["sum_e_over_d"] == pytest.approx(np.sum((A / D) ** 2), rel=1e-12)
    assert out["n_perturbers"] == n_ext
    # per-determinant values and the perturber set
    sel = {d.tobytes(): e for d, e in zip(out["sel_dets"], out["sel_e"])}
    assert len(sel) == n_ext
    for j, i in enumerate(ext):
        key = fci[i].tobytes()
        if connected[j]:
            assert abs(sel[key] - e_dense[j]) < 1e-13
        else:
            assert key not in sel
    # selection order: |e| descending, determinant key ascending
    order = sorted(
        [i for j, i in enumerate(ext) if connected[j]],
        key=lambda i: (-abs(e_dense[list(ext).index(i)]), tuple(int(x) for x in fci[i].reshape(-1))),
    )
    k = 10
    top = ham.sweep(dets, c, e0, k=k)
    assert [d.tobytes() for d in top["sel_dets"]] == [fci[i].tobytes() for i in order[:k]]
    # the per-generator definition adds up to the same total
    gens = [ham.generator(dets, c, e0, g) for g in range(len(dets))]
    assert abs(sum(r["eps"] for r in gens) - e_dense.sum()) < 1e-12
    assert sum(r["n_perturbers"] for r in gens) == n_ext
    assert all(r["eps"] == pytest.approx(out["eps_by_rank"][g], abs=1e-13) for g, r in enumerate(gens))


# ---------------------------------------------------------------------------
# P3: Psi0 = full CI space -> no perturbers (Sec. "Extrapolation": E_PT2 = 0
#     at the FCI limit)
# ---------------------------------------------------------------------------
def test_full_ci_space_has_no_perturbers(oracle_mod):
    norb, na, nb = 6, 2, 2
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=8, seed=9)
    fci = S.all_dets(norb, na, nb)
    c = S.random_coefs(len(fci), 1)
    out = ham.sweep(fci, c, -10.0, k=5)
    assert out["e_pt2"] == 0.0 and out["n_perturbers"] == 0 and out["n_selected"] == 0
    assert out["n_connections"] == 0


# ---------------------------------------------------------------------------
# P6: single-determinant Psi0: closed form over (i, j, a, b)
# ---------------------------------------------------------------------------
def test_hf_only_closed_form(oracle_mod):
    norb, n = 9, 3  # closed shell, n electrons per spin
    ham, h, eri = _ham(oracle_mod, norb, n, n, rank=10, seed=21)
    g = eri_full(eri, norb)
    occ, vir = range(n), range(n, norb)

    def energy(up, dn):
        so = [(0, p) for p in up] + [(1, p) for p in dn]
        e = sum(h[p, p] for _, p in so)
        for (s1, p), (s2, q) in itertools.combinations(so, 2):
            e += g[p, p, q, q] - (g[p, q, q, p] if s1 == s2 else 0.0)
        return e

    ehf = energy(occ, occ)
    e0 = ehf
    tot = 0.0
    count = 0
    for i in occ:  # singles, both spins (closed shell: identical)
        for a in vir:
            f = h[i, a] + sum(2 * g[i, a, j, j] - g[i, j, j, a] for j in occ)
            up = [x for x in occ if x != i] + [a]
            tot += 2 * f * f / (e0 - energy(up, occ))
            count += 2
    for i, j in itertools.combinations(occ, 2):  # same-spin doubles
        for a, b in itertools.combinations(vir, 2):
            v = g[i, a, j, b] - g[i, b, j, a]
            up = [x for x in occ if x not in (i, j)] + [a, b]
            tot += 2 * v * v / (e0 - energy(up, occ))
            count += 2
    for i in occ:  # opposite-spin doubles
        for j in occ:
            for a in vir:
                for b in vir:
                    v = g[i, a, j, b]
                    up = [x for x in occ if x != i] + [a]
                    dn = [x for x in occ if x != j] + [b]
                    tot += v * v / (e0 - energy(up, dn))
                    count += 1
    hf = S.hf_det(norb, n, n)
    out = ham.sweep(hf[None], np.array([1.0]), e0, k=3)
    assert out["n_perturbers"] == count == S.n_singles_doubles(norb, n, n)
    assert abs(out["e_pt2"] - tot) < 1e-12
    assert abs(ham.diag(hf) - ehf) < 1e-13


# ---------------------------------------------------------------------------
# P5: phase mask (Sec. "Internal representation of determinants", Algorithm
#     PhasemaskOfDet) -- the reading used by the CUDA path
# ---------------------------------------------------------------------------
M64 = (1 << 64) - 1


def _phasemask_corrected(words):
    """P <- I, then P ^= P << 2^d for d = 0..5, then xor the carry r of the
    preceding words (all ones when their popcount is odd)."""
    out, r = [], 0
    for w in words:
        p = w
        for d in range(6):
            p ^= (p << (1 << d)) & M64
        out.append(p ^ r)
        if bin(w).count("1") & 1:
            r = ~r & M64
    return out


def _phasemask_as_printed(words):
    out, r = [], 0
    for w in words:
        p = w ^ ((w << 1) & M64)
        for d in range(6):
            p ^= (p << (1 << d)) & M64
        out.append(p ^ r)
        if bin(w).count("1") & 1:
            r = ~r & M64
    return out


def test_phase_mask_reading():
    rng = np.random.default_rng(3)
    for _ in range(500):
        words = [int(x) for x in rng.integers(0, 2**63, size=2, dtype=np.int64)]
        words = [w | (int(rng.integers(0, 2)) << 63) for w in words]
        bits = [(words[b // 64] >> (b % 64)) & 1 for b in range(128)]
        brute = [sum(bits[: i + 1]) & 1 for i in range(128)]
        pm = _phasemask_corrected(words)
        assert [(pm[i // 64] >> (i % 64)) & 1 for i in range(128)] == brute
    # the listing as printed applies the one-bit shift twice and returns I
    w = int(rng.integers(0, 2**63))
    assert _phasemask_as_printed([w]) == [w]


def test_phase_formula_matches_counting(oracle_mod):
    """+-(-1)^(P[h] xor P[p]) equals (-1)^(occupied strictly between h, p)."""
    rng = np.random.default_rng(4)
    for _ in range(2000):
        w = int(rng.integers(0, 2**62))
        occ = [i for i in range(62) if (w >> i) & 1]
        vir = [i for i in range(62) if not (w >> i) & 1]
        if not occ or not vir:
            continue
        h = occ[int(rng.integers(len(occ)))]
        p = vir[int(rng.integers(len(vir)))]
        P = _phasemask_corrected([w])[0]
        sgn = (-1) ** (((P >> h) & 1) ^ ((P >> p) & 1))
        if h > p:
            sgn = -sgn
        between = sum(1 for i in occ if min(h, p) < i < max(h, p))
        assert sgn == (-1) ** between


# ---------------------------------------------------------------------------
# P7: invariants of the definition
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def small_case(oracle_mod):
    norb, na, nb = 12, 3, 3
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=14, seed=31)
    dets = S.random_excited_dets(norb, na, nb, 60, seed=32)
    c = S.random_coefs(60, 33, decay=0.04)
    e0 = min(ham.diag(d) for d in dets) - 0.3
    return ham, h, eri, dets, c, e0


def test_invariant_input_order(small_case):
    ham, h, eri, dets, c, e0 = small_case
    a = ham.sweep(dets, c, e0, k=20)
    perm = np.random.default_rng(1).permutation(len(dets))
    b = ham.sweep(dets[perm], c[perm], e0, k=20)
    assert a["e_pt2"] == pytest.approx(b["e_pt2"], abs=1e-12)
    assert a["digest"] == b["digest"]
    assert a["n_perturbers"] == b["n_perturbers"]
    assert a["n_connections"] == b["n_connections"]
    assert np.array_equal(a["sel_dets"], b["sel_dets"])


def test_invariant_sum_of_generators(small_case):
    ham, h, eri, dets, c, e0 = small_case
    a = ham.sweep(dets, c, e0, k=0)
    assert math.fsum(a["eps_by_rank"]) == pytest.approx(a["e_pt2"], abs=1e-12)
    assert int(a["na_by_rank"].sum()) == a["n_perturbers"]
    assert int(a["ncon_by_rank"].sum()) == a["n_connections"]


def test_invariant_coefficient_scaling(small_case):
    ham, h, eri, dets, c, e0 = small_case
    a = ham.sweep(dets, c, e0, k=0)
    b = ham.sweep(dets, -c, e0, k=0)
    assert b["e_pt2"] == pytest.approx(a["e_pt2"], abs=1e-13)
    lam = 1.7
    d = ham.sweep(dets, lam * c, e0, k=0)
    assert d["e_pt2"] == pytest.approx(lam * lam * a["e_pt2"], rel=1e-12)


def test_invariant_homogeneity(oracle_mod, small_case):
    ham, h, eri, dets, c, e0 = small_case
    lam = 1.3
    ham2 = oracle_mod.Hamiltonian(ham.norb, ham.nalpha, ham.nbeta, lam * h, lam * eri)
    a = ham.sweep(dets, c, e0, k=0)
    b = ham2.sweep(dets, c, lam * e0, k=0)
    assert b["e_pt2"] == pytest.approx(lam * a["e_pt2"], rel=1e-12)


def test_invariant_spin_flip(oracle_mod):
    norb, n = 10, 3
    ham, h, eri = _ham(oracle_mod, norb, n, n, rank=12, seed=41)
    base = S.random_excited_dets(norb, n, n, 30, seed=42)
    flipped = base[:, ::-1, :]
    allk = {d.tobytes(): d for d in np.concatenate([base, flipped])}
    dets = np.stack(list(allk.values()))
    # spin-flip-symmetric coefficients: c(flip(D)) = c(D)
    rng = np.random.default_rng(5)
    cmap = {}
    c = np.zeros(len(dets))
    for i, d in enumerate(dets):
        f = d[::-1].tobytes()
        if f in cmap:
            c[i] = cmap[f]
        else:
            c[i] = rng.standard_normal()
            cmap[d.tobytes()] = c[i]
    e0 = min(ham.diag(d) for d in dets) - 0.4
    a = ham.sweep(dets, c, e0, k=0)
    b = ham.sweep(dets[:, ::-1, :].copy(), c, e0, k=0)
    assert b["e_pt2"] == pytest.approx(a["e_pt2"], abs=1e-12)
    assert b["n_perturbers"] == a["n_perturbers"]


def test_per_generator_definition_matches_plain_definition(small_case):
    ham, h, eri, dets, c, e0 = small_case
    a = ham.sweep(dets, c, e0, k=0)
    for g in [0, 1, 7, 30, 59]:
        r = ham.generator(dets, c, e0, g)
        assert r["n_perturbers"] == a["na_by_rank"][g]
        assert r["n_connections"] == a["ncon_by_rank"][g]
        assert r["eps"] == pytest.approx(a["eps_by_rank"][g], abs=1e-13)


def test_single_alpha_query(small_case):
    ham, h, eri, dets, c, e0 = small_case
    a = ham.sweep(dets, c, e0, k=15)
    for d, e in zip(a["sel_dets"], a["sel_e"]):
        q = ham.alpha(dets, c, d)
        assert not q["internal"]
        assert q["A"] ** 2 / (e0 - q["haa"]) == pytest.approx(e, rel=1e-12)


def test_validation_rejects_bad_spaces(small_case):
    ham, h, eri, dets, c, e0 = small_case
    assert ham.validate(dets) == 0
    dup = np.concatenate([dets, dets[:1]])
    assert ham.validate(dup) == -2
    bad = dets.copy()
    bad[0, 0, 0] |= np.uint64(1) << np.uint64(20)  # bit beyond norb / wrong count
    assert ham.validate(bad) == -1


def test_packed_integral_symmetry(oracle_mod):
    """The compound index (Algorithm hash) is invariant under the 8
    permutations of real chemists' integrals."""
    norb = 7
    ham, h, eri = _ham(oracle_mod, norb, 2, 2, rank=9, seed=51)
    rng = np.random.default_rng(0)
    for _ in range(200):
        p, q, r, s = (int(x) for x in rng.integers(0, norb, 4))
        v = ham.eri_value(p, q, r, s)
        for perm in [(q, p, r, s), (p, q, s, r), (q, p, s, r), (r, s, p, q), (s, r, p, q), (r, s, q, p), (s, r, q, p)]:
            assert ham.eri_value(*perm) == v


# ---------------------------------------------------------------------------
# P8: gradient of E_PT2 with respect to the integrals (Psi0 and E0 fixed)
# ---------------------------------------------------------------------------
@pytest.fixture(scope="module")
def grad_case(oracle_mod):
    norb, na, nb = 9, 3, 3
    ham, h, eri = _ham(oracle_mod, norb, na, nb, rank=11, seed=91)
    dets = S.random_excited_dets(norb, na, nb, 40, seed=92)
    c = S.random_coefs(40, 93, decay=0.05)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    g = ham.gradient(dets, c, e0)
    return oracle_mod, ham, h, eri, dets, c, e0, g


def _energy(oracle_mod, norb, na, nb, h, eri, dets, c, e0):
    return oracle_mod.Hamiltonian(norb, na, nb, h, eri).sweep(dets, c, e0, k=0, per_generator=False)["e_pt2"]


def test_gradient_energy_and_de0(grad_case):
    oracle_mod, ham, h, eri, dets, c, e0, g = grad_case
    s = ham.sweep(dets, c, e0, k=0)
    assert g["e_pt2"] == pytest.approx(s["e_pt2"], abs=1e-12)
    assert g["de0"] == pytest.approx(-s["sum_e_over_d"], rel=1e-12)


def test_gradient_euler_identity(grad_case):
    """E_PT2 is homogeneous of degree 1 in (h, eri, E0): the sum of
    theta * dE/dtheta over all parameters equals E_PT2."""
    oracle_mod, ham, h, eri, dets, c, e0, g = grad_case
    lhs = np.sum(h * g["dh"]) + np.dot(eri, g["deri"]) + e0 * g["de0"]
    assert lhs == pytest.approx(g["e_pt2"], abs=1e-10)


def test_gradient_matches_central_differences(grad_case):
    oracle_mod, ham, h, eri, dets, c, e0, g = grad_case
    norb, na, nb = ham.norb, ham.nalpha, ham.nbeta
    step = 1e-5
    rng = np.random.default_rng(94)
    for idx in rng.choice(len(eri), 25, replace=False):
        ep, em = eri.copy(), eri.copy()
        ep[idx] += step
        em[idx] -= step
        fd = (_energy(oracle_mod, norb, na, nb, h, ep, dets, c, e0) -
              _energy(oracle_mod, norb, na, nb, h, em, dets, c, e0)) / (2 * step)
        assert abs(fd - g["deri"][idx]) <= 1e-6 * abs(fd) + 1e-8, (idx, fd, g["deri"][idx])
    for p, q in [(0, 0), (4, 4), (0, 3), (2, 7), (5, 8)]:
        hp, hm = h.copy(), h.copy()
        hp[p, q] += step
        hm[p, q] -= step
        if p != q:
            hp[q, p] += step
            hm[q, p] -= step
        fd = (_energy(oracle_mod, norb, na, nb, hp, eri, dets, c, e0) -
              _energy(oracle_mod, norb, na, nb, hm, eri, dets, c, e0)) / (2 * step)
        an = g["dh"][p, p] if p == q else g["dh"][p, q] + g["dh"][q, p]
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-8, (p, q, fd, an)
    assert np.allclose(g["dh"], g["dh"].T, atol=0, rtol=0)


# ---------------------------------------------------------------------------
# Renormalised PT2 (Sec. "Renormalized PT2", Eqs. E2-w, Z)
# ---------------------------------------------------------------------------
def test_rpt2_self_energy_derivative_and_z(small_case):
    """Sigma(E) = sum A^2/(E - H_aa): Sigma(E0) = E_PT2, dSigma/dE at E0 =
    -sum A^2/D^2 (central difference), and Z = 1/(1 + sum A^2/D^2) in (0, 1].
    Z and E_rPT2 are the library's (qp_pt2_merge_results of the oracle's
    totals, no GPU needed), checked against the definition."""
    from paper_1902_08154_gb300 import build

    build.build()
    import paper_1902_08154_gb300 as qp

    ham, h, eri, dets, c, e0 = small_case
    base = ham.sweep(dets, c, e0, k=0)
    d = 1e-5
    sp = ham.sweep(dets, c, e0 + d, k=0)["e_pt2"]
    sm = ham.sweep(dets, c, e0 - d, k=0)["e_pt2"]
    assert (sp - sm) / (2 * d) == pytest.approx(-base["sum_e_over_d"], rel=1e-7)
    r = qp.merge_results([base], e0)
    assert 0.0 < r["z"] <= 1.0
    assert r["z"] == pytest.approx(1.0 / (1.0 + base["sum_e_over_d"]), rel=1e-15)
    assert r["e_rpt2"] == pytest.approx(e0 + r["z"] * base["e_pt2"], abs=1e-14)
    assert abs(r["e_rpt2"] - e0) <= abs(base["e_pt2"])  # rPT2 damps the correction
    # merging shards: sums and counts add, digests add modulo 2^64 and xor
    half = [dict(base, e_pt2=base["e_pt2"] / 2, sum_e_over_d=base["sum_e_over_d"] / 2,
                 n_perturbers=base["n_perturbers"] // 2, n_connections=base["n_connections"] // 2,
                 digest=(base["digest"][0], 0)),
            dict(base, e_pt2=base["e_pt2"] / 2, sum_e_over_d=base["sum_e_over_d"] / 2,
                 n_perturbers=base["n_perturbers"] - base["n_perturbers"] // 2,
                 n_connections=base["n_connections"] - base["n_connections"] // 2,
                 digest=((1 << 64) - 1, base["digest"][1]))]
    m = qp.merge_results(half, e0)
    assert m["n_perturbers"] == base["n_perturbers"] and m["n_connections"] == base["n_connections"]
    assert m["digest"] == ((base["digest"][0] - 1) % (1 << 64), base["digest"][1])
    assert m["e_pt2"] == pytest.approx(base["e_pt2"], abs=1e-15) and m["z"] == pytest.approx(r["z"], rel=1e-15)
