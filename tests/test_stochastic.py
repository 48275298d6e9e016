"""The hybrid deterministic/stochastic estimator of E_PT2 (Sec. "Stochastic
selection", Eq. edetstoch), with the per-generator eps_I of the oracle: the
estimate is unbiased, its error bar is calibrated, and a run that reaches
the end of the ranks returns the deterministic value."""
import numpy as np
import pytest

from paper_1902_08154_gb300 import stochastic as ST
from paper_1902_08154_gb300 import synthetic as S


@pytest.fixture(scope="module")
def case(oracle_mod):
    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 41)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 80, 42)
    c = S.random_coefs(len(dets), 43, decay=0.05)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    ref = ham.sweep(dets, c, e0, k=0)
    return c, ref["eps_by_rank"], ref["e_pt2"], oracle_mod.ranks(c)


def test_order_matches_oracle_ranks(case):
    c, eps, e_ref, rank_of = case
    order = ST.generator_order(c)
    assert np.array_equal(rank_of[order], np.arange(len(c)))


def test_terms_expectation_is_the_tail_sum(case):
    c, eps, _, _ = case
    p = ST.draw_probabilities(c)
    assert abs(p.sum() - 1.0) < 1e-15
    every = np.arange(len(p))
    for d in (0, 7, 40, len(p)):
        expect = float(np.dot(p, ST.terms(every, d, eps, p)))
        assert expect == pytest.approx(float(eps[d:].sum()), abs=1e-14)


def test_exact_when_the_prefix_covers_every_rank(case):
    c, eps, e_ref, _ = case
    asked = []

    def eval_fn(ranks):
        assert len(np.unique(ranks)) == len(ranks)
        asked.extend(ranks.tolist())
        return eps[ranks]

    res = ST.run(eval_fn, c, rel_err=0.0, det_per_iter=9, draws_per_iter=20, seed=3)
    assert res["exact"] and res["prefix"] == len(c)
    assert sorted(asked) == list(range(len(c)))  # each eps_I computed once
    assert res["e_pt2"] == pytest.approx(e_ref, abs=1e-12)


def test_unbiased_and_error_bar(case):
    c, eps, e_ref, _ = case
    est, errs = [], []
    for seed in range(400):
        r = ST.run(lambda rk: eps[rk], c, rel_err=0.0, det_per_iter=5, draws_per_iter=60, seed=seed, max_iters=1,
                   min_tail=1)
        est.append(r["e_pt2"])
        errs.append(r["error"])
    est, errs = np.array(est), np.array(errs)
    se = est.std(ddof=1) / np.sqrt(len(est))
    assert abs(est.mean() - e_ref) <= 5 * se + 1e-15
    assert np.mean(np.abs(est - e_ref) <= 2 * errs) >= 0.85


def test_merge_top_k():
    e = np.array([0.1, -0.5, 0.3, -0.3, 0.05])
    d = np.array([[5], [1], [9], [2], [7]], dtype=np.uint64).reshape(5, 1, 1)
    se, sd = ST.merge_top_k(e, d, 3)
    assert np.array_equal(se, [-0.5, -0.3, 0.3])  # tie |e| = 0.3 ordered by key
    assert np.array_equal(sd.ravel(), [1, 2, 9])
