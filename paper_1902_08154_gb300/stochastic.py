"""Hybrid deterministic/stochastic E_PT2 with on-the-fly selection
(Sec. "Stochastic selection", Eqs. calpha and edetstoch), driven over the
per-generator sweep of the CUDA library.

E_PT2 = sum_I eps_I, the generators I sorted by decreasing c_I^2 (rank 0
first) and eps_I the contribution of the perturbers assigned to I by the
canonical rule.  Two processes feed the sum, as in the paper:

* a deterministic one computes eps_I for the lowest ranks not computed yet,
  so that the deterministic set D is always a prefix 0..d-1 of the ranks;
* a stochastic one draws ranks with probability p_I = c_I^2 / sum_J c_J^2.
  A computed eps_I is kept: a rank drawn again costs nothing.

With M draws I_1..I_M so far the estimate is

    E = sum_{I < d} eps_I + (1/M) sum_m t(I_m),   t(I) = [I >= d] eps_I / p_I.

For any d the expectation of t over the draws is sum_{I >= d} eps_I, so E is
unbiased; its statistical error is the standard error of the mean of the M
terms.  The run stops when |dE / E| <= rel_err (the paper's default is
0.002), with at least ``min_tail`` draws beyond the prefix, or when the
prefix holds every rank, where E is the deterministic value.  The selection
is the best k perturbers of every generator computed so far.

Only the draws and the arithmetic of the estimate run on the host (a few
operations per draw); every eps_I comes from the GPU sweep
(``PT2.eval_generators``).  Draws use numpy's PCG64 generator with ``seed``.
"""
from __future__ import annotations

import numpy as np


def generator_order(coefs):
    """Input index of the generator of each rank: decreasing c^2, ties by
    input index (the library's order)."""
    c = np.asarray(coefs, dtype=np.float64)
    return np.argsort(-(c * c), kind="stable")


def draw_probabilities(coefs):
    """p_r = c^2 / sum c^2 of the generator of rank r."""
    c = np.asarray(coefs, dtype=np.float64)[generator_order(coefs)]
    w = c * c
    return w / w.sum()


def terms(draws, d, eps_by_rank, p):
    """t(I_m) = [I_m >= d] eps_{I_m} / p_{I_m} for each draw."""
    draws = np.asarray(draws, dtype=np.int64)
    out = np.zeros(len(draws))
    tail = draws >= d
    out[tail] = eps_by_rank[draws[tail]] / p[draws[tail]]
    return out


def estimate(d, eps_by_rank, draws, p):
    """(E, statistical error, number of draws beyond the prefix) for the
    prefix 0..d-1 and the draws so far; eps_by_rank must hold every rank
    below d and every drawn rank."""
    det = float(np.sum(eps_by_rank[:d]))
    n = len(draws)
    if n == 0:
        return det, (0.0 if d == len(p) else np.inf), 0
    t = terms(draws, d, eps_by_rank, p)
    mean = float(t.mean())
    err = float(t.std(ddof=1) / np.sqrt(n)) if n > 1 else np.inf
    return det + mean, err, int(np.count_nonzero(np.asarray(draws) >= d))


def run(eval_fn, coefs, rel_err=0.002, det_per_iter=None, draws_per_iter=None, seed=0, min_tail=64,
        max_iters=None):
    """The two processes, one block of ranks per iteration.

    eval_fn(ranks) -> eps of those ranks (an int32 array of new, distinct
    ranks each time).  Returns a dict: e_pt2, error, prefix (d), computed
    (distinct ranks evaluated), draws, iterations, exact (d covers all)."""
    p = draw_probabilities(coefs)
    n = len(p)
    # draws are cheap (a drawn rank is computed once), so each iteration
    # draws ten times more ranks than the deterministic block it adds
    det_per_iter = det_per_iter or max(1, n // 200)
    draws_per_iter = draws_per_iter or max(256, n // 20)
    rng = np.random.Generator(np.random.PCG64(seed))
    eps = np.zeros(n)
    known = np.zeros(n, dtype=bool)
    draws = np.zeros(0, dtype=np.int64)
    d = 0
    it = 0
    while True:
        it += 1
        block = np.arange(d, min(n, d + det_per_iter), dtype=np.int64)
        new_draws = rng.choice(n, size=draws_per_iter, p=p) if d + len(block) < n else np.zeros(0, np.int64)
        want = np.union1d(block, new_draws)
        want = want[~known[want]]
        if len(want):
            eps[want] = eval_fn(want.astype(np.int32))
            known[want] = True
        d += len(block)
        draws = np.concatenate([draws, new_draws])
        e, err, ntail = estimate(d, eps, draws, p)
        exact = d == n
        if exact:
            e, err = float(np.sum(eps)), 0.0
        done = exact or (ntail >= min_tail and err <= rel_err * abs(e))
        if done or (max_iters is not None and it >= max_iters):
            return {"e_pt2": e, "error": err, "prefix": d, "computed": int(known.sum()), "draws": len(draws),
                    "iterations": it, "exact": exact, "converged": done}


def merge_top_k(sel_e, sel_dets, k):
    """Best k of concatenated selections: |e| descending, then the key words
    ascending (the library's order)."""
    if k <= 0 or len(sel_e) == 0:
        return sel_e[:0], sel_dets[:0]
    keys = sel_dets.reshape(len(sel_e), -1)
    order = np.lexsort(tuple(keys[:, w] for w in range(keys.shape[1] - 1, -1, -1)) + (-np.abs(sel_e),))
    order = order[:k]
    return sel_e[order], sel_dets[order]


def stochastic_pt2(pt2, dets, coefs, e0, rel_err=0.002, k=0, **kw):
    """Hybrid E_PT2 over a PT2 context; dets and coefs as for PT2.eval (the
    coefficients are also needed on the host for the draws).  With k > 0
    the result holds the best k perturbers of the computed generators
    (host arrays)."""
    c_host = coefs.detach().cpu().numpy() if hasattr(coefs, "detach") else np.asarray(coefs)
    sel = {"e": np.zeros(0), "dets": np.zeros((0, 2, pt2.nint), dtype=np.uint64)}

    def eval_fn(ranks):
        out = pt2.eval_generators(dets, coefs, e0, ranks, k=k)
        if k > 0 and len(out["sel_e"]):
            se = out["sel_e"].detach().cpu().numpy() if hasattr(out["sel_e"], "detach") else out["sel_e"]
            sd = out["sel_dets"].detach().cpu().numpy() if hasattr(out["sel_dets"], "detach") else out["sel_dets"]
            e_all = np.concatenate([sel["e"], se])
            d_all = np.concatenate([sel["dets"], sd.view(np.uint64)])
            sel["e"], sel["dets"] = merge_top_k(e_all, d_all, k)
        return out["eps"]

    res = run(eval_fn, c_host, rel_err=rel_err, **kw)
    if k > 0:
        res.update(sel_e=sel["e"], sel_dets=sel["dets"])
    return res
