"""Sweeps of generator subsets (qp_pt2_eval_gens) and the hybrid
deterministic/stochastic E_PT2 on the GPU."""
import json
import os

import numpy as np
import pytest

from paper_1902_08154_gb300 import stochastic as ST
from paper_1902_08154_gb300 import synthetic as S

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


@pytest.fixture(scope="module")
def case(oracle_mod):
    norb, na, nb = 16, 4, 4
    h, eri = S.hamiltonian(norb, 18, 51)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 150, 52)
    c = S.random_coefs(len(dets), 53, decay=0.03)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    return norb, na, nb, h, eri, ham, dets, c, e0


def test_subset_matches_full_sweep_and_oracle(qp, case):
    norb, na, nb, h, eri, ham, dets, c, e0 = case
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    full = pt2.eval(_dev(dets), _dev(c), e0, 0, per_generator=True)
    ranks = np.random.default_rng(5).permutation(len(dets))[:37].astype(np.int32)
    sub = pt2.eval_generators(_dev(dets), _dev(c), e0, ranks, k=25)
    feps = full["eps_by_rank"].cpu().numpy()
    assert np.array_equal(sub["na"], full["na_by_rank"].cpu().numpy()[ranks])
    assert np.array_equal(sub["ncon"], full["ncon_by_rank"].cpu().numpy()[ranks])
    assert np.abs(sub["eps"] - feps[ranks]).max() <= 1e-13
    assert sub["n_perturbers"] == int(sub["na"].sum())
    assert sub["e_pt2"] == pytest.approx(float(feps[ranks].sum()), abs=1e-12)
    for i in (0, 11, 36):  # the oracle's per-generator definition
        g = ham.generator(dets, c, e0, int(ranks[i]))
        assert sub["na"][i] == g["n_perturbers"] and sub["ncon"][i] == g["n_connections"]
        assert abs(sub["eps"][i] - g["eps"]) <= 1e-10
    # the selection of a subset holds only perturbers of its generators: every
    # selected e is one of the oracle's e of those generators
    se = sub["sel_e"].cpu().numpy()
    assert len(se) == 25 and np.all(np.abs(se[:-1]) >= np.abs(se[1:]))
    pt2.close()


def test_subset_rejects_bad_lists(qp, case):
    norb, na, nb, h, eri, ham, dets, c, e0 = case
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    for bad in ([0, 0], [len(dets)], [-1]):
        with pytest.raises(qp.QPError) as ei:
            pt2.eval_generators(_dev(dets), _dev(c), e0, np.array(bad, dtype=np.int32))
        assert ei.value.code == qp.QP_EINVAL
    pt2.close()


def test_hybrid_reaches_the_deterministic_value(qp, case):
    norb, na, nb, h, eri, ham, dets, c, e0 = case
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    full = pt2.eval(_dev(dets), _dev(c), e0, 40)
    res = ST.stochastic_pt2(pt2, _dev(dets), _dev(c), e0, rel_err=0.0, k=40, det_per_iter=16, draws_per_iter=40)
    assert res["exact"]
    assert res["e_pt2"] == pytest.approx(full["e_pt2"], abs=1e-10)
    # on-the-fly selection over all generators = the sweep's selection
    assert np.allclose(res["sel_e"], full["sel_e"].cpu().numpy(), rtol=1e-10, atol=1e-14)
    pt2.close()


def test_hybrid_on_the_stored_workload(qp):
    P = np.load(os.path.join(GOLDEN, "cfg2_psi0.npz"))
    E = json.loads(str(np.load(os.path.join(GOLDEN, "cfg2_expected.npz"))["summary"]))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    res = ST.stochastic_pt2(pt2, _dev(P["dets"]), _dev(P["coefs"]), float(P["e0"]), rel_err=0.002, seed=7)
    print(f"hybrid E_PT2 {res['e_pt2']:.8f} +- {res['error']:.2e} with {res['computed']} of {len(P['coefs'])} "
          f"generators (oracle {E['e_pt2']:.8f})")
    assert res["converged"] and not res["exact"]
    assert abs(res["e_pt2"] - E["e_pt2"]) <= 5 * res["error"]
    pt2.close()
