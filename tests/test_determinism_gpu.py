"""Run-to-run reproducibility of the CUDA sweep, and the error paths that
need a GPU: singular denominators, and generator shards of the one-state
sweep against the oracle's per-generator sums.

A_alpha is accumulated exactly (integer sums of the products), the item
sums of each generator are reduced in item order and E_PT2 in rank order
(Eqs. calpha and edetstoch: E_PT2 = sum_I eps_I), so the same inputs give
the same bits whatever the number of CTAs and the order in which they take
work items.
"""
import json
import os

import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import as_np, check_per_generator, check_selection, check_totals

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


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


def _bits(x):
    return np.asarray(as_np(x), dtype=np.float64).view(np.uint64)


def _same(a, b):
    assert np.float64(a["e_pt2"]).view(np.uint64) == np.float64(b["e_pt2"]).view(np.uint64)
    assert np.float64(a["sum_e_over_d"]).view(np.uint64) == np.float64(b["sum_e_over_d"]).view(np.uint64)
    assert a["n_perturbers"] == b["n_perturbers"] and a["n_connections"] == b["n_connections"]
    assert tuple(a["digest"]) == tuple(b["digest"])
    assert np.array_equal(_bits(a["eps_by_rank"]), _bits(b["eps_by_rank"]))
    assert np.array_equal(_bits(a["sel_e"]), _bits(b["sel_e"]))
    assert np.array_equal(as_np(a["sel_dets"]), as_np(b["sel_dets"]))


def _cfg2_head(n):
    P = np.load(os.path.join(GOLDEN, "cfg2_psi0.npz"))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    return meta, h, eri, P["dets"][:n].copy(), P["coefs"][:n].copy(), float(P["e0"])


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_bit_identical_runs_and_grids(qp, precision):
    """Two runs, and grids of 1 and of the default CTAs per SM, give the
    same bits for E_PT2, sum A^2/D^2, every eps_I and the selection."""
    meta, h, eri, dets, c, e0 = _cfg2_head(2500)
    prec = qp.QP_FP64 if precision == "fp64" else qp.QP_MIXED
    k = 2 * len(dets)
    outs = []
    for bps in (0, 0, 1):
        pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri), blocks_per_sm=bps,
                     precision=prec)
        outs.append(pt2.eval(_dev(dets), _dev(c), e0, k, per_generator=True))
        pt2.close()
    _same(outs[0], outs[1])
    _same(outs[0], outs[2])


def test_bit_identical_two_words(qp, oracle_mod):
    norb, na, nb = 90, 4, 4
    h, eri = S.hamiltonian(norb, 8, 61)
    dets = S.random_excited_dets(norb, na, nb, 120, 62)
    c = S.random_coefs(len(dets), 63, decay=0.05)
    c /= np.linalg.norm(c)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    outs = []
    for bps in (0, 1):
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), blocks_per_sm=bps)
        outs.append(pt2.eval(_dev(dets), _dev(c), e0, 200, per_generator=True))
        pt2.close()
    _same(outs[0], outs[1])
    ref = ham.sweep(dets, c, e0, k=200)
    check_totals(outs[0], ref)
    check_per_generator(outs[0], ref)


def test_singular_denominator_reported(qp, oracle_mod):
    """E0 equal to the diagonal energy of a perturber: QP_ESINGULAR, with the
    result still filled in and min |D| = 0 (reading: no level shift)."""
    norb, na, nb = 10, 3, 3
    h, eri = S.hamiltonian(norb, 12, 71)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    hf = S.hf_det(norb, na, nb)
    subs = ham.substitutions(hf)
    alpha = subs[len(subs) // 2]
    e0 = ham.diag(alpha)  # D_alpha = E0 - H_aa = 0 for this perturber of HF
    pt2 = qp.PT2(norb, na, nb, h, eri)
    got = pt2.eval(hf[None].copy(), np.array([1.0]), e0, 5, check=False)
    assert got["rc"] == qp.QP_ESINGULAR
    assert got["min_abs_den"] < 1e-12
    ref = ham.sweep(hf[None], np.array([1.0]), e0 + 1.0, k=0)
    assert got["n_perturbers"] == ref["n_perturbers"] and got["n_connections"] == ref["n_connections"]
    # the context stays usable
    ok = pt2.eval(hf[None].copy(), np.array([1.0]), e0 + 1.0, 5)
    assert ok["rc"] == qp.QP_OK
    assert abs(ok["e_pt2"] - ref["e_pt2"]) < 1e-10
    pt2.close()


@pytest.mark.parametrize("nshard", [2, 3])
def test_one_state_shards_match_oracle(qp, oracle_mod, nshard):
    """Generator shards of the one-state sweep (qp_pt2_eval with
    shard_index/shard_count): each shard against the oracle's per-rank sums of
    its ranks, and the merged totals against the whole sweep."""
    norb, na, nb = 16, 4, 4
    h, eri = S.hamiltonian(norb, 18, 81)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 160, 82)
    c = S.random_coefs(len(dets), 83, decay=0.05)
    c /= np.linalg.norm(c)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    k = 120
    ref = ham.sweep(dets, c, e0, k=k)
    tot_e, tot_na, tot_nc, d0, d1 = 0.0, 0, 0, 0, 0
    sel_e, sel_d = [], []
    for s in range(nshard):
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), shard_index=s, shard_count=nshard)
        got = pt2.eval(_dev(dets), _dev(c), e0, k, per_generator=True)
        pt2.close()
        mine = np.arange(len(dets)) % nshard == s
        eps = as_np(got["eps_by_rank"])
        assert np.all(eps[~mine] == 0.0)
        assert np.max(np.abs(eps[mine] - ref["eps_by_rank"][mine])) <= 1e-10
        assert np.array_equal(as_np(got["na_by_rank"])[mine], ref["na_by_rank"][mine])
        assert got["n_perturbers"] == int(ref["na_by_rank"][mine].sum())
        assert abs(got["e_pt2"] - ref["eps_by_rank"][mine].sum()) <= 1e-10
        tot_e += got["e_pt2"]
        tot_na += got["n_perturbers"]
        tot_nc += got["n_connections"]
        d0 = (d0 + got["digest"][0]) % (1 << 64)
        d1 ^= got["digest"][1]
        sel_e.append(as_np(got["sel_e"]))
        sel_d.append(as_np(got["sel_dets"]).view(np.uint64).reshape(len(got["sel_e"]), -1))
    assert tot_na == ref["n_perturbers"] and tot_nc == ref["n_connections"]
    assert (d0, d1) == tuple(int(x) for x in ref["digest"])
    assert abs(tot_e - ref["e_pt2"]) <= 1e-10
    # merged selection: the k best of the union, |e| descending then key
    e = np.concatenate(sel_e)
    d = np.concatenate(sel_d)
    keys = [tuple(int(w) for w in row) for row in d]
    order = sorted(range(len(e)), key=lambda i: (-abs(e[i]), keys[i]))[:k]
    check_selection(d[order].reshape(len(order), 2, -1), e[order], ref["sel_dets"], ref["sel_e"])


def test_work_chunk_and_row_tiles(qp, oracle_mod):
    """Runtime launch parameters: items drawn 4 per queue draw, and the
    opposite-spin batches split into 1, 2 or 3 tiles of rows; every setting
    matches the oracle, and the draw size does not change a single bit."""
    norb, na, nb = 20, 4, 4
    h, eri = S.hamiltonian(norb, 22, 91)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 140, 92)
    c = S.random_coefs(len(dets), 93, decay=0.05)
    c /= np.linalg.norm(c)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    ref = ham.sweep(dets, c, e0, k=100)
    for tile in (1, 2, 3):
        outs = []
        for chunk in (1, 4):
            pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), work_chunk=chunk, tile=tile)
            outs.append(pt2.eval(_dev(dets), _dev(c), e0, 100, per_generator=True))
            pt2.close()
        check_totals(outs[0], ref)
        check_per_generator(outs[0], ref)
        check_selection(outs[0]["sel_dets"], outs[0]["sel_e"], ref["sel_dets"], ref["sel_e"])
        _same(outs[0], outs[1])


def test_watchdog_timeout(qp):
    """A watchdog limit far below the sweep's time: the call returns
    QP_ETIMEOUT with partial totals, and the GPU and library stay usable (a
    context without the limit then gives the whole sweep)."""
    meta, h, eri, dets, c, e0 = _cfg2_head(2500)
    full = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    ref = full.eval(_dev(dets), _dev(c), e0, 100)
    short = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri), timeout_s=1e-6)
    for _ in range(2):
        got = short.eval(_dev(dets), _dev(c), e0, 100, check=False)
        assert got["rc"] == qp.QP_ETIMEOUT
        assert got["n_perturbers"] < ref["n_perturbers"]
    assert b"watchdog" in qp.load().qp_pt2_last_error()
    again = full.eval(_dev(dets), _dev(c), e0, 100)
    assert again["rc"] == qp.QP_OK and again["e_pt2"] == ref["e_pt2"]
    short.close()
    full.close()


def test_rpt2_fields(qp, oracle_mod):
    """Z = 1/(1 + sum A^2/D^2) and E0 + Z E_PT2 come with every result."""
    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 95)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 40, 96)
    c = S.random_coefs(len(dets), 97, decay=0.05)
    c /= np.linalg.norm(c)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    ref = ham.sweep(dets, c, e0, k=0)
    pt2 = qp.PT2(norb, na, nb, h, eri)
    got = pt2.eval(dets, c, e0, 0)
    z = 1.0 / (1.0 + ref["sum_e_over_d"])
    assert got["z"] == pytest.approx(z, rel=1e-12)
    assert got["e_rpt2"] == pytest.approx(e0 + z * ref["e_pt2"], abs=1e-10)
    pt2.close()
