"""Parity of the CUDA sweep (through the C ABI) with the CPU oracle."""
import json
import os

import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import as_np, check_per_generator, check_selection, check_totals, cipsi_space

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


def _case(oracle_mod, norb, na, nb, ndet, seed, rank=None, decay=0.05):
    h, eri = S.hamiltonian(norb, rank or norb + 2, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    c = S.random_coefs(len(dets), seed + 2, decay=decay)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    return h, eri, ham, dets, c, e0


def _compare(qp, h, eri, ham, dets, c, e0, k, norb, na, nb, device=True):
    ref = ham.sweep(dets, c, e0, k=k)
    if device:
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
        got = pt2.eval(_dev(dets), _dev(c), e0, k, per_generator=True)
    else:
        pt2 = qp.PT2(norb, na, nb, h, eri)
        got = pt2.eval(np.ascontiguousarray(dets), np.ascontiguousarray(c), e0, k, per_generator=True)
    check_totals(got, ref)
    check_per_generator(got, ref)
    assert np.array_equal(as_np(got["rank_of"]).astype(np.int64), ref["rank_of"])
    check_selection(got["sel_dets"], got["sel_e"], ref["sel_dets"], ref["sel_e"])
    pt2.close()
    return got, ref


CASES = [
    # norb, na, nb, ndet, k, seed
    (8, 2, 2, 20, 10, 1),
    (10, 3, 2, 60, 50, 2),
    (12, 3, 3, 100, 100000, 3),  # k larger than the perturber count
    (16, 4, 4, 150, 300, 4),
    (20, 5, 5, 200, 100, 5),
    (24, 6, 5, 120, 64, 6),
    (9, 4, 0, 30, 20, 7),        # no spin-down electrons
    (30, 2, 2, 50, 20, 8),
    (40, 3, 3, 80, 40, 9),
    (64, 3, 3, 40, 25, 10),      # the last orbital fills bit 63
]


@pytest.mark.parametrize("norb,na,nb,ndet,k,seed", CASES)
def test_random_spaces_one_word(qp, oracle_mod, norb, na, nb, ndet, k, seed):
    h, eri, ham, dets, c, e0 = _case(oracle_mod, norb, na, nb, ndet, seed)
    _compare(qp, h, eri, ham, dets, c, e0, k, norb, na, nb)


@pytest.mark.parametrize("norb,na,nb,ndet,k,seed,rank", [
    (66, 2, 2, 40, 30, 11, 6),
    (70, 3, 3, 60, 50, 12, 6),
    (80, 4, 3, 50, 40, 13, 5),
    (128, 2, 2, 30, 20, 14, 3),
    (112, 3, 3, 40, 30, 15, 4),  # opposite-spin batches split in two row tiles
])
def test_random_spaces_two_words(qp, oracle_mod, norb, na, nb, ndet, k, seed, rank):
    h, eri, ham, dets, c, e0 = _case(oracle_mod, norb, na, nb, ndet, seed, rank=rank)
    # put electrons across the word boundary as well
    extra = []
    for up, dn in [((62, 63, 64)[:na], (1, 64, 65)[:nb]), ((63, 65, 66)[:na], (0, 63, 127 % norb)[:nb])]:
        if len(set(up)) == na and len(set(dn)) == nb:
            extra.append(S.occ_to_det(sorted(up), sorted(dn), norb))
    keys = {d.tobytes() for d in dets}
    extra = [d for d in extra if d.tobytes() not in keys]
    if extra:
        dets = np.concatenate([dets, np.stack(extra)])
        c = S.random_coefs(len(dets), seed + 5, decay=0.05)
    _compare(qp, h, eri, ham, dets, c, e0, k, norb, na, nb)


def test_hf_only_and_k_zero(qp, oracle_mod):
    norb, na, nb = 14, 3, 3
    h, eri = S.hamiltonian(norb, 10, 21)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    hf = S.hf_det(norb, na, nb)[None]
    e0 = ham.diag(hf[0])
    _compare(qp, h, eri, ham, hf, np.array([1.0]), e0, 0, norb, na, nb)
    _compare(qp, h, eri, ham, hf, np.array([1.0]), e0, 7, norb, na, nb)


def test_full_ci_space_has_no_perturbers(qp, oracle_mod):
    norb, na, nb = 6, 2, 2
    h, eri = S.hamiltonian(norb, 8, 22)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    fci = S.all_dets(norb, na, nb)
    c = S.random_coefs(len(fci), 1)
    got, ref = _compare(qp, h, eri, ham, fci, c, -20.0, 5, norb, na, nb)
    assert got["n_perturbers"] == 0 and got["e_pt2"] == 0.0 and got["n_selected"] == 0


def test_host_and_device_pointers_agree(qp, oracle_mod):
    h, eri, ham, dets, c, e0 = _case(oracle_mod, 18, 4, 4, 90, 31)
    a, _ = _compare(qp, h, eri, ham, dets, c, e0, 40, 18, 4, 4, device=True)
    b, _ = _compare(qp, h, eri, ham, dets, c, e0, 40, 18, 4, 4, device=False)
    assert a["digest"] == b["digest"] and a["n_connections"] == b["n_connections"]
    assert abs(a["e_pt2"] - b["e_pt2"]) < 1e-12


def test_input_order_invariance(qp, oracle_mod):
    h, eri, ham, dets, c, e0 = _case(oracle_mod, 16, 4, 3, 120, 41)
    pt2 = qp.PT2(16, 4, 3, _dev(h), _dev(eri))
    a = pt2.eval(_dev(dets), _dev(c), e0, 30)
    perm = np.random.default_rng(0).permutation(len(dets))
    b = pt2.eval(_dev(dets[perm]), _dev(c[perm]), e0, 30)
    assert a["digest"] == b["digest"] and a["n_perturbers"] == b["n_perturbers"]
    assert a["n_connections"] == b["n_connections"]
    assert abs(a["e_pt2"] - b["e_pt2"]) < 1e-12
    check_selection(a["sel_dets"], a["sel_e"], b["sel_dets"], b["sel_e"])


def test_validation_errors(qp, oracle_mod):
    h, eri, ham, dets, c, e0 = _case(oracle_mod, 12, 3, 3, 30, 51)
    pt2 = qp.PT2(12, 3, 3, h, eri)
    dup = np.concatenate([dets, dets[3:4]])
    cd = np.concatenate([c, c[:1]])
    with pytest.raises(qp.QPError) as ei:
        pt2.eval(dup, cd, e0, 5)
    assert ei.value.code == qp.QP_EDUP
    bad = dets.copy()
    bad[2, 1, 0] |= np.uint64(1) << np.uint64(40)  # bit beyond norb
    with pytest.raises(qp.QPError) as ei:
        pt2.eval(bad, c, e0, 5)
    assert ei.value.code == qp.QP_EINVAL
    hbad = h.copy()
    hbad[0, 1] += 1e-6
    with pytest.raises(qp.QPError) as ei:
        qp.PT2(12, 3, 3, hbad, eri)
    assert ei.value.code == qp.QP_ESYM


def _golden(name):
    p = os.path.join(GOLDEN, f"{name}_psi0.npz")
    e = os.path.join(GOLDEN, f"{name}_expected.npz")
    if not (os.path.exists(p) and os.path.exists(e)):
        pytest.skip(f"{name} golden files absent")
    P = np.load(p)
    E = np.load(e)
    meta = json.loads(str(P["meta"]))
    summ = json.loads(str(E["summary"]))
    return P, E, meta, summ


@pytest.mark.parametrize("name", ["cfg1", "cfg2", "cfg4"])
def test_golden_workloads(qp, name):
    P, E, meta, summ = _golden(name)
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    same_inputs = S.hamiltonian_digest(h, eri) == meta["digest"]
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    got = pt2.eval(_dev(P["dets"]), _dev(P["coefs"]), float(P["e0"]), meta["k"], per_generator=True)
    ref = dict(summ)
    ref["digest"] = [int(x) for x in summ["digest"]]
    ref.update(eps_by_rank=E["eps_by_rank"], na_by_rank=E["na_by_rank"], ncon_by_rank=E["ncon_by_rank"])
    # integrals regenerated on this machine: bit-identical by construction of
    # the generator; if not, energies are still compared at the same tolerance
    assert same_inputs or abs(got["e_pt2"] - ref["e_pt2"]) < 1e-10
    check_totals(got, ref)
    check_per_generator(got, ref)
    check_selection(got["sel_dets"], got["sel_e"], E["sel_dets"], E["sel_e"])
    pt2.close()


# ---------------------------------------------------------------------------
# Mixed precision: FP32 integral gathers and products, FP64 accumulation,
# denominators and reductions.  Integer outputs are structural and must match
# exactly; the energy must lie within the stated 1e-6 Eh of the FP64 oracle.
# ---------------------------------------------------------------------------
MIXED_TOL = 1e-6


@pytest.mark.parametrize("norb,na,nb,ndet,k,seed", [(16, 4, 4, 160, 100, 81), (24, 6, 5, 120, 64, 82),
                                                    (70, 3, 3, 64, 40, 83)])
def test_mixed_precision_random(qp, oracle_mod, norb, na, nb, ndet, k, seed):
    # Psi0 grown by the oracle's CIPSI rule, unit norm, variational E0: the
    # shape of the workloads on which the mixed form states its bound
    h, eri = S.hamiltonian(norb, norb + 2, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets, c, e0 = cipsi_space(oracle_mod, ham, norb, na, nb, ndet)
    ref = ham.sweep(dets, c, e0, k=k)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), precision=qp.QP_MIXED)
    got = pt2.eval(_dev(dets), _dev(c), e0, k, per_generator=True)
    assert got["n_perturbers"] == ref["n_perturbers"]
    assert got["n_connections"] == ref["n_connections"]
    assert tuple(got["digest"]) == tuple(ref["digest"])
    # the stated bound: 1e-6 Eh absolute (FP32 products, each with a relative
    # error of about 2^-24, summed exactly)
    assert abs(got["e_pt2"] - ref["e_pt2"]) <= MIXED_TOL
    assert np.array_equal(as_np(got["na_by_rank"]), ref["na_by_rank"])
    ge, re_ = as_np(got["sel_e"]), ref["sel_e"]
    assert len(ge) == len(re_)
    assert np.all(np.abs(ge - re_) <= 1e-7 + 1e-5 * np.abs(re_))
    pt2.close()


def test_mixed_precision_golden_cfg2(qp):
    P, E, meta, summ = _golden("cfg2")
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri), precision=qp.QP_MIXED)
    got = pt2.eval(_dev(P["dets"]), _dev(P["coefs"]), float(P["e0"]), meta["k"])
    assert got["n_perturbers"] == summ["n_perturbers"]
    assert got["n_connections"] == summ["n_connections"]
    assert tuple(got["digest"]) == tuple(int(x) for x in summ["digest"])
    err = abs(got["e_pt2"] - summ["e_pt2"])
    print(f"mixed precision |E - E_oracle| = {err:.3e} Eh")
    assert err <= MIXED_TOL
    pt2.close()
