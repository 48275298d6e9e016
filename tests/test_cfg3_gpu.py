"""The 128-orbital workload (two 64-bit words per spin, 14 + 14 electrons,
Cholesky rank 192) in FP64 and in mixed precision, against the oracle.

* A reduced Psi0 (the first 10 determinants of the workload's list, with the
  same Hamiltonian) is compared with the oracle's full sweep element by
  element: perturber set, per-generator arrays and selection.
* The full 10^5-determinant Psi0 is compared through properties that hold at
  any size (FP64 and mixed give the same perturber set, connection count and
  digest, and energies within the stated 1e-6 Eh) and on sampled outputs:
  selected perturbers recomputed one by one by the oracle (A_alpha and
  H_alpha,alpha from the Slater-Condon rules, e_alpha = A^2 / (E0 - H_aa)).
"""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import as_np, check_per_generator, check_selection, check_totals, e_close

pytestmark = pytest.mark.gpu

MIXED_TOL = 1e-6
SPEC = S.CFG3


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


@pytest.fixture(scope="module")
def full():
    return S.cfg3_instance()


@pytest.fixture(scope="module")
def reduced(oracle_mod, full):
    h, eri, dets, _, _ = full
    n = 10
    d = np.ascontiguousarray(dets[:n])
    c = S.random_coefs(n, SPEC["seed"] + 2, decay=4.0 / n)
    e0 = S.diagonal_lower_bound(h, eri, SPEC["nalpha"] + SPEC["nbeta"]) - 1.0
    ham = oracle_mod.Hamiltonian(SPEC["norb"], SPEC["nalpha"], SPEC["nbeta"], h, eri)
    ref = ham.sweep(d, c, e0, k=2 * n)
    return h, eri, d, c, e0, ref


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_cfg3_reduced_against_oracle(qp, reduced, precision):
    h, eri, d, c, e0, ref = reduced
    prec = qp.QP_FP64 if precision == "fp64" else qp.QP_MIXED
    pt2 = qp.PT2(SPEC["norb"], SPEC["nalpha"], SPEC["nbeta"], _dev(h), _dev(eri), precision=prec)
    got = pt2.eval(_dev(d), _dev(c), e0, 2 * len(d), per_generator=True)
    pt2.close()
    if precision == "fp64":
        check_totals(got, ref)
        check_per_generator(got, ref)
        check_selection(got["sel_dets"], got["sel_e"], ref["sel_dets"], ref["sel_e"])
    else:
        assert got["n_perturbers"] == ref["n_perturbers"]
        assert got["n_connections"] == ref["n_connections"]
        assert tuple(got["digest"]) == tuple(ref["digest"])
        assert np.array_equal(as_np(got["na_by_rank"]), ref["na_by_rank"])
        assert abs(got["e_pt2"] - ref["e_pt2"]) <= MIXED_TOL
        ge, re_ = as_np(got["sel_e"]), ref["sel_e"]
        assert len(ge) == len(re_)
        assert np.all(np.abs(ge - re_) <= 1e-7 + 1e-5 * np.abs(re_))


def _sweep(qp, full, prec):
    h, eri, dets, c, e0 = full
    pt2 = qp.PT2(SPEC["norb"], SPEC["nalpha"], SPEC["nbeta"], _dev(h), _dev(eri), precision=prec)
    got = pt2.eval(_dev(dets), _dev(c), e0, len(dets))
    pt2.close()
    return got


@pytest.fixture(scope="module")
def full_fp64(qp, full):
    return _sweep(qp, full, qp.QP_FP64)


@pytest.fixture(scope="module")
def full_mixed(qp, full):
    return _sweep(qp, full, qp.QP_MIXED)


def _spot_check(oracle_mod, full, got, n_samples, rel):
    """Selected perturbers recomputed by the oracle, one by one."""
    h, eri, dets, c, e0 = full
    ham = oracle_mod.Hamiltonian(SPEC["norb"], SPEC["nalpha"], SPEC["nbeta"], h, eri)
    sd = as_np(got["sel_dets"]).view(np.uint64)
    se = as_np(got["sel_e"])
    assert len(se) == len(dets)
    picks = np.unique(np.linspace(0, len(se) - 1, n_samples).astype(np.int64))
    for i in picks:
        a = ham.alpha(dets, c, sd[i])
        assert not a["internal"] and a["gen_rank"] >= 0 and a["n_connections"] > 0
        e = a["A"] ** 2 / (e0 - a["haa"])
        assert abs(se[i] - e) <= 1e-14 + rel * abs(e), (i, se[i], e)
    a = np.abs(se)
    assert np.all(a[:-1] >= a[1:] * (1 - 1e-12))


def test_cfg3_full_fp64_selection_spot_check(oracle_mod, full, full_fp64):
    _spot_check(oracle_mod, full, full_fp64, 48, 1e-10)


def test_cfg3_full_mixed_matches_fp64(oracle_mod, full, full_fp64, full_mixed):
    f, m = full_fp64, full_mixed
    assert m["n_perturbers"] == f["n_perturbers"]
    assert m["n_connections"] == f["n_connections"]
    assert tuple(m["digest"]) == tuple(f["digest"])
    err = abs(m["e_pt2"] - f["e_pt2"])
    print(f"128 orbitals, 10^5 determinants: |E_mixed - E_FP64| = {err:.3e} Eh")
    assert err <= MIXED_TOL
    assert e_close(m["sum_e_over_d"], f["sum_e_over_d"], 1e-12, 1e-6)
    _spot_check(oracle_mod, full, m, 24, 1e-5)
