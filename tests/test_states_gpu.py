"""Parity of the multi-state sweep (qp_pt2_eval_states, through the C ABI)
with the oracle's plain multi-state definition (Sec. "Selected CI": one PT2
per state and the selection criterion of Angeli et al.)."""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import E_TOL, as_np, check_selection

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qp():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1902_08154_gb300 import build

    build.build()
    import paper_1902_08154_gb300 as qp

    qp.load()
    return qp


def _dev(a):
    import torch

    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _states_case(oracle_mod, norb, na, nb, ndet, nst, seed, rank=None):
    h, eri = S.hamiltonian(norb, rank or norb + 2, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    C = np.stack([S.random_coefs(len(dets), seed + 2 + 7 * s, decay=0.05 / (1 + s)) for s in range(nst)])
    e_low = min(ham.diag(d) for d in dets)
    E0 = np.array([e_low - 1.0 - 0.2 * s for s in range(nst)])
    return h, eri, ham, dets, C, E0


def _check_states(got, ref):
    assert got["n_perturbers"] == ref["n_perturbers"]
    assert got["n_connections"] == ref["n_connections"]
    assert tuple(got["digest"]) == tuple(int(x) for x in ref["digest"])
    assert got["n_tiny"] == ref["n_tiny"]
    assert got["n_selected"] == ref["n_selected"]
    d = np.abs(got["e_pt2_states"] - ref["e_pt2_states"])
    assert d.max() <= E_TOL, d
    s = np.maximum(1.0, np.abs(ref["sum_e_over_d_states"]))
    assert np.all(np.abs(got["sum_e_over_d_states"] - ref["sum_e_over_d_states"]) <= E_TOL * s)
    if ref["n_perturbers"]:
        assert got["min_abs_den"] == pytest.approx(ref["min_abs_den"], rel=1e-12)
    check_selection(got["sel_dets"], got["sel_crit"], ref["sel_dets"], ref["sel_crit"])


@pytest.mark.parametrize("norb,na,nb,ndet,k,nst,seed,rank", [
    (10, 3, 2, 60, 50, 2, 2, None),
    (16, 4, 4, 150, 300, 3, 4, None),
    (24, 6, 5, 120, 64, 4, 6, None),
    (9, 4, 0, 30, 20, 2, 7, None),         # no spin-down electrons
    (40, 3, 3, 80, 100000, 3, 9, None),    # k above the perturber count
    (70, 3, 3, 60, 50, 2, 12, 6),          # two words per spin
    (112, 3, 3, 40, 30, 3, 15, 4),         # opposite-spin batches in two row tiles
    (64, 2, 2, 60, 50, 2, 16, 6),          # 62 x 62 cells: two accumulators of 31 KB each
])
def test_states_match_oracle(qp, oracle_mod, norb, na, nb, ndet, k, nst, seed, rank):
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, ndet, nst, seed, rank)
    ref = ham.states(dets, C, E0, k=k)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    got = pt2.eval_states(_dev(dets), _dev(C), E0, k)
    _check_states(got, ref)
    # host inputs give the same answer
    got_h = pt2.eval_states(np.ascontiguousarray(dets), C, E0, k)
    _check_states(got_h, ref)
    pt2.close()


def test_one_state_matches_the_one_state_sweep(qp, oracle_mod):
    norb, na, nb = 20, 5, 5
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, 200, 1, 21)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    one = pt2.eval(_dev(dets), _dev(C[0]), float(E0[0]), 100)
    ms = pt2.eval_states(_dev(dets), _dev(C), E0, 100)
    for key in ("n_perturbers", "n_connections", "digest", "n_tiny", "n_selected"):
        assert one[key] == ms[key], key
    assert abs(one["e_pt2"] - ms["e_pt2_states"][0]) <= E_TOL
    # one state: the criterion is e / max c^2
    check_selection(ms["sel_dets"], as_np(ms["sel_crit"]) * np.max(C[0] ** 2), one["sel_dets"], one["sel_e"])
    pt2.close()


def test_states_with_a_target_space(qp, oracle_mod):
    norb, na, nb = 16, 4, 4
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, 100, 2, 31)
    ref_det = S.occ_to_det(range(na), range(nb), norb)
    core = S.occ_to_det([0], [0], norb)
    ham.set_target(ref=ref_det, max_exc=3, core=core)
    ref = ham.states(dets, C, E0, k=80)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    pt2.set_target(ref=ref_det, max_exc=3, core=core)
    got = pt2.eval_states(_dev(dets), _dev(C), E0, 80)
    _check_states(got, ref)
    pt2.close()
    ham.set_target()


def test_states_rejects_bad_arguments(qp, oracle_mod):
    norb, na, nb = 12, 3, 3
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, 40, 2, 41)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    d = _dev(dets)
    zero = C.copy()
    zero[1] = 0.0
    assert pt2.eval_states(d, _dev(zero), E0, 10, check=False)["rc"] == qp.QP_EINVAL
    five = np.concatenate([C, C, C])[:5]
    assert pt2.eval_states(d, _dev(five), np.full(5, E0[0]), 10, check=False)["rc"] == qp.QP_EINVAL
    bad = C.copy()
    bad[1, 3] = np.nan
    assert pt2.eval_states(d, _dev(bad), E0, 10, check=False)["rc"] == qp.QP_EINVAL
    # the context still works after the rejected calls
    ref = ham.states(dets, C, E0, k=10)
    _check_states(pt2.eval_states(d, _dev(C), E0, 10), ref)
    pt2.close()
    mixed = qp.PT2(norb, na, nb, _dev(h), _dev(eri), precision=qp.QP_MIXED)
    assert mixed.eval_states(d, _dev(C), E0, 10, check=False)["rc"] == qp.QP_ENOTSUP
    mixed.close()


def test_states_largest_accumulators(qp, oracle_mod):
    """128 orbitals, 2+2 electrons: a row tile of an opposite-spin batch holds
    63 x 126 cells, so three states' accumulators (190 KB) still fit in one
    CTA's shared memory and four do not."""
    norb, na, nb = 128, 2, 2
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, 12, 4, 51, rank=3)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    d = _dev(dets)
    assert pt2.eval_states(d, _dev(C), E0, 20, check=False)["rc"] == qp.QP_ENOTSUP
    ref = ham.states(dets, C[:3], E0[:3], k=20)
    _check_states(pt2.eval_states(d, _dev(C[:3]), E0[:3], 20), ref)
    pt2.close()


def test_states_shards_on_one_gpu(qp, oracle_mod):
    """Two generator shards of a multi-state sweep (generators of rank i mod 2),
    run one after the other: each against the oracle's shard, and their merge
    against the whole sweep."""
    from paper_1902_08154_gb300.shard import merge_selections, merge_totals

    norb, na, nb = 16, 4, 4
    h, eri, ham, dets, C, E0 = _states_case(oracle_mod, norb, na, nb, 120, 2, 61)
    k = 60
    parts, es, ds = [], [], []
    for i in range(2):
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), shard_index=i, shard_count=2)
        got = pt2.eval_states(_dev(dets), _dev(C), E0, k)
        _check_states(got, ham.states(dets, C, E0, k=k, shard=(i, 2)))
        parts.append(got)
        es.append(as_np(got["sel_crit"]))
        ds.append(as_np(got["sel_dets"]).view(np.uint64).reshape(len(es[-1]), -1))
        pt2.close()
    full = ham.states(dets, C, E0, k=k)
    tot = merge_totals(parts)
    assert tot["n_perturbers"] == full["n_perturbers"]
    assert tot["n_connections"] == full["n_connections"]
    assert tuple(tot["digest"]) == tuple(full["digest"])
    assert np.abs(tot["e_pt2_states"] - full["e_pt2_states"]).max() <= E_TOL
    e, d = merge_selections(es, ds, k)
    check_selection(d, e, full["sel_dets"], full["sel_crit"])


def test_states_full_size_cfg2_sampled(qp, oracle_mod):
    """The 64-orbital, 10^4-determinant workload with two states (its stored
    Psi0, and a seeded second vector with E0 - 0.1): state 0's totals against
    the oracle's stored sweep, and sampled selected determinants recomputed by
    the oracle one by one (A_s and H_aa by the Slater-Condon rules, then the
    multi-state criterion)."""
    import json
    import os

    gold = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
    P = np.load(os.path.join(gold, "cfg2_psi0.npz"))
    E = np.load(os.path.join(gold, "cfg2_expected.npz"))
    meta = json.loads(str(P["meta"]))
    summ = json.loads(str(E["summary"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    ham = oracle_mod.Hamiltonian(meta["norb"], meta["nalpha"], meta["nbeta"], h, eri)
    dets = P["dets"]
    C = np.stack([P["coefs"], S.random_coefs(len(dets), 71, decay=0.001)])
    E0 = np.array([float(P["e0"]), float(P["e0"]) - 0.1])
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    got = pt2.eval_states(_dev(dets), _dev(C), E0, meta["k"])
    pt2.close()
    assert got["n_perturbers"] == summ["n_perturbers"]
    assert got["n_connections"] == summ["n_connections"]
    assert tuple(got["digest"]) == tuple(int(x) for x in summ["digest"])
    assert abs(got["e_pt2_states"][0] - summ["e_pt2"]) <= E_TOL
    sel, crit, num = as_np(got["sel_dets"]).view(np.uint64), as_np(got["sel_crit"]), as_np(got["sel_num"])
    assert len(crit) == meta["k"]
    assert np.all(np.abs(crit[:-1]) >= np.abs(crit[1:]))
    w = 1.0 / np.max(C * C, axis=1)
    for i in np.random.default_rng(5).choice(len(crit), 24, replace=False):
        a = [ham.alpha(dets, C[s], sel[i]) for s in range(2)]
        assert not a[0]["internal"] and a[0]["n_connections"] > 0
        ref = sum(w[s] * a[s]["A"] ** 2 / (E0[s] - a[s]["haa"]) for s in range(2))
        assert abs(crit[i] - ref) <= 1e-12 + 1e-10 * abs(ref)
        assert abs(num[i] - a[0]["A"]) <= 1e-12 + 1e-10 * abs(a[0]["A"])
