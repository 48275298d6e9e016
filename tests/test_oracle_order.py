"""Pins of the oracle's generator order and of its eigen-solver.

The generator order (Sec. "New stochastic selection" and the Appendix on the
CIPSI selection: generators sorted by decreasing c_I^2; ties by increasing
input index, the reading this library takes) decides which generator owns
each perturber (Eqs. calpha, edetstoch).  Every per-generator value the
oracle reports rests on it, so it is pinned here against constructions that
share nothing with the oracle's C code:

* the rank of every determinant against numpy's stable lexsort on
  (-c*c, index), on vectors built with exact ties in c^2 (repeated values,
  sign flips +c/-c, zeros);
* the per-generator energies eps_I against a dense-H sum over the whole
  external space in which each alpha is given to the first connected
  internal determinant in the numpy order, so that a wrong order (ascending
  c^2, ties by key, ties by descending index) moves energy between
  generators and fails;
* the Davidson solver used to make the stored workloads against
  numpy's dense eigh above the size (64) where it hands over to eigh.
"""
import numpy as np
import pytest
import scipy.sparse as sp

from paper_1902_08154_gb300 import synthetic as S
from tests.sq_hamiltonian import dense_h


def _numpy_ranks(c):
    """rank_of[i] = position of i when sorted by decreasing c^2, then index."""
    c = np.asarray(c, dtype=np.float64)
    c2 = c * c
    order = np.lexsort((np.arange(len(c)), -c2))
    rank_of = np.empty(len(c), dtype=np.int64)
    rank_of[order] = np.arange(len(c))
    return rank_of


def _tied_vector(n, seed):
    rng = np.random.default_rng(seed)
    base = rng.normal(size=max(2, n // 4))
    c = rng.choice(base, size=n)                 # exact repeats
    c *= rng.choice([-1.0, 1.0], size=n)         # +c and -c tie in c^2
    c[rng.choice(n, size=max(1, n // 10), replace=False)] = 0.0
    return c


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (17, 2), (256, 3), (5000, 4)])
def test_ranks_match_numpy_lexsort(oracle_mod, n, seed):
    c = _tied_vector(n, seed)
    got = oracle_mod.ranks(c)
    assert np.array_equal(got, _numpy_ranks(c))
    # the construction really has ties, including across a sign flip
    if n >= 17:
        c2 = c * c
        assert len(np.unique(c2)) < n
        assert np.any((c > 0)[:, None] & (c[None, :] == -c[:, None]))


def test_ranks_small_cases_by_hand(oracle_mod):
    # c = [0.5, -0.5, 0.7, 0.0, 0.5]: c^2 = [.25, .25, .49, 0, .25]
    # order: index 2, then the tie {0, 1, 4} by index, then 3
    got = oracle_mod.ranks(np.array([0.5, -0.5, 0.7, 0.0, 0.5]))
    assert list(got) == [1, 2, 0, 4, 3]
    # the square is the IEEE product c*c: 0.1*0.1 and (-0.1)*(-0.1) tie exactly
    got = oracle_mod.ranks(np.array([-0.1, 0.1, 0.3]))
    assert list(got) == [1, 2, 0]


@pytest.mark.parametrize("norb,na,nb,nint_,seed", [(6, 2, 2, 30, 7), (7, 3, 2, 40, 8)])
def test_generator_ownership_matches_dense_assignment(oracle_mod, norb, na, nb, nint_, seed):
    """eps_I of every generator against the dense external sum, with each
    alpha owned by the first (numpy order) internal J connected to it."""
    h, eri = S.hamiltonian(norb, norb + 3, 300 + seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    fci = S.all_dets(norb, na, nb)
    Hm = dense_h(fci, h, eri, norb)
    rng = np.random.default_rng(seed)
    low = list(np.argsort(np.diag(Hm), kind="stable")[:nint_])
    # input order differs from key order, so that "ties by index" and "ties
    # by key" are different rules
    idx = rng.permutation(np.array(low))
    w, v = np.linalg.eigh(Hm[np.ix_(idx, idx)])
    e0 = w[0]
    # coefficients with exact ties in c^2 (the eigenvector's values, with
    # some of them copied, sign-flipped, onto others), so that the tie rule
    # decides the owner of some perturbers
    c = v[:, 0].copy()
    pick = rng.choice(len(c), size=2 * (len(c) // 4), replace=False)
    src, dst = pick[: len(pick) // 2], pick[len(pick) // 2:]
    c[dst] = -c[src]
    rank_of = _numpy_ranks(c)
    assert len(np.unique(c * c)) < len(c)

    mask = np.ones(len(fci), bool)
    mask[idx] = False
    ext = np.nonzero(mask)[0]
    Hx = Hm[np.ix_(ext, idx)]
    A = Hx @ c
    D = e0 - np.diag(Hm)[ext]
    e = A * A / D
    # structural connection: excitation degree 1 or 2 (whatever the value)
    def deg(a, b):
        return int(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a.ravel(), b.ravel()))) // 2

    eps_ref = np.zeros(len(idx))
    na_ref = np.zeros(len(idx), dtype=np.int64)
    for j, a in enumerate(ext):
        conn = [i for i in range(len(idx)) if deg(fci[a], fci[idx[i]]) <= 2]
        if not conn:
            continue
        owner = min(conn, key=lambda i: rank_of[i])
        eps_ref[rank_of[owner]] += e[j]
        na_ref[rank_of[owner]] += 1

    dets = fci[idx]
    out = ham.sweep(dets, c, e0, k=0)
    assert np.array_equal(out["rank_of"], rank_of)
    assert np.max(np.abs(out["eps_by_rank"] - eps_ref)) < 1e-13
    assert np.array_equal(np.asarray(out["na_by_rank"]), na_ref)
    for g in range(len(idx)):
        r = ham.generator(dets, c, e0, g)
        assert r["eps"] == pytest.approx(eps_ref[g], abs=1e-13)
        assert r["n_perturbers"] == na_ref[g]
    # a plausible mistake is visible: ascending order moves perturbers
    wrong = _numpy_ranks(1.0 / np.where(c == 0, 1e-300, c))
    assert not np.array_equal(wrong, rank_of)


def _sparse_symmetric(n, seed, density):
    rng = np.random.default_rng(seed)
    m = sp.random(n, n, density=density, random_state=np.random.RandomState(seed), data_rvs=rng.standard_normal)
    m = 0.1 * (m + m.T)
    diag = np.sort(rng.uniform(-5.0, 5.0, size=n))
    diag[0] -= 0.5  # a separated lowest level, as in a CI matrix near HF
    return (m + sp.diags(diag)).tocsr()


@pytest.mark.parametrize("n,seed,density", [(65, 1, 0.05), (200, 2, 0.02), (800, 3, 0.01)])
def test_davidson_matches_dense_eigh(n, seed, density):
    from oracle import psi0

    Hm = _sparse_symmetric(n, seed, density)
    e, x, res = psi0.davidson(Hm, tol=1e-10)
    w, v = np.linalg.eigh(Hm.toarray())
    assert res < 1e-10
    assert abs(e - w[0]) < 1e-10
    ov = abs(float(x @ v[:, 0]))
    assert ov == pytest.approx(1.0, abs=1e-10)
    # a guess close to the answer converges to the same pair
    e2, x2, _ = psi0.davidson(Hm, guess=v[:, 0] + 1e-3, tol=1e-10)
    assert abs(e2 - w[0]) < 1e-10


def test_ground_state_on_cipsi_like_space_matches_eigh(oracle_mod):
    """The path the stored workloads take: H over a determinant space of
    more than 64 determinants, Davidson, c_0 > 0, E0 as Rayleigh quotient."""
    from oracle import psi0

    norb, na, nb = 8, 2, 2
    h, eri = S.hamiltonian(norb, 10, 41)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    fci = S.all_dets(norb, na, nb)
    Hm = dense_h(fci, h, eri, norb)
    idx = np.sort(np.argsort(np.diag(Hm), kind="stable")[:150])
    dets = fci[idx]
    e0, c, res = psi0.ground_state(ham, dets, tol=1e-11)
    w, v = np.linalg.eigh(Hm[np.ix_(idx, idx)])
    assert len(dets) > 64
    assert abs(e0 - w[0]) < 1e-10
    ref = v[:, 0] * np.sign(v[0, 0])
    assert c[0] > 0
    assert np.max(np.abs(c - ref)) < 1e-8
