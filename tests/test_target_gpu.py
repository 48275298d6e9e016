"""Target spaces on the GPU (qp_pt2_set_target) against the oracle's
restricted sweep and gradient."""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import as_np, check_per_generator, check_selection, check_totals, cipsi_space

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


def _targets(norb, na, nb):
    hf = S.hf_det(norb, na, nb)
    core = S.occ_to_det([0], [0], norb)
    deleted = S.occ_to_det([norb - 1, norb - 2], [norb - 1], norb)
    return [dict(ref=hf, max_exc=2), dict(ref=hf, max_exc=3, core=core), dict(core=core, deleted=deleted)]


@pytest.mark.parametrize("norb,na,nb,ndet,k,seed,rank", [(16, 4, 4, 120, 60, 71, 18), (24, 5, 4, 90, 40, 72, 8),
                                                         (70, 3, 3, 50, 30, 73, 6)])
def test_target_space_sweep_matches_oracle(qp, oracle_mod, norb, na, nb, ndet, k, seed, rank):
    h, eri = S.hamiltonian(norb, rank, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    # Psi0 grown by the oracle's CIPSI rule, unit norm, variational E0: the
    # shape on which the mixed form states its 1e-6 Eh bound
    dets, c, e0 = cipsi_space(oracle_mod, ham, norb, na, nb, ndet)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    mix = qp.PT2(norb, na, nb, _dev(h), _dev(eri), precision=qp.QP_MIXED)
    for t in _targets(norb, na, nb):
        ham.set_target(**t)
        ref = ham.sweep(dets, c, e0, k=k)
        pt2.set_target(**t)
        got = pt2.eval(_dev(dets), _dev(c), e0, k, per_generator=True)
        check_totals(got, ref)
        check_per_generator(got, ref)
        check_selection(got["sel_dets"], got["sel_e"], ref["sel_dets"], ref["sel_e"])
        mix.set_target(**t)
        gm = mix.eval(_dev(dets), _dev(c), e0, k)
        assert gm["n_perturbers"] == ref["n_perturbers"] and tuple(gm["digest"]) == tuple(ref["digest"])
        assert abs(gm["e_pt2"] - ref["e_pt2"]) <= 1e-6
    pt2.set_target()
    ham.set_target()
    assert pt2.eval(_dev(dets), _dev(c), e0, 0)["n_perturbers"] == ham.sweep(dets, c, e0, k=0)["n_perturbers"]
    pt2.close()
    mix.close()


def test_target_space_gradient_matches_oracle(qp, oracle_mod):
    norb, na, nb = 14, 4, 3
    h, eri = S.hamiltonian(norb, 12, 74)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 60, 75)
    c = S.random_coefs(len(dets), 76, decay=0.05)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    t = dict(ref=S.hf_det(norb, na, nb), max_exc=2, core=S.occ_to_det([0], [0], norb))
    ham.set_target(**t)
    ref = ham.gradient(dets, c, e0)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    pt2.set_target(**t)
    dh = np.zeros((norb, norb))
    deri = np.zeros(len(eri))
    de0, res = qp.qp_pt2_grad(pt2.ctx, len(dets), dets, c, e0, dh, deri)
    pt2.close()
    assert abs(res.e_pt2 - ref["e_pt2"]) < 1e-10
    scale = max(1.0, np.abs(ref["deri"]).max(), np.abs(ref["dh"]).max())
    assert np.abs(dh - ref["dh"]).max() <= 1e-11 * scale
    assert np.abs(deri - ref["deri"]).max() <= 1e-11 * scale
    assert de0 == pytest.approx(ref["de0"], rel=1e-12, abs=1e-13)


def test_target_space_rejects_overlapping_masks(qp):
    norb = 10
    h, eri = S.hamiltonian(norb, 12, 77)
    pt2 = qp.PT2(norb, 3, 3, h, eri)
    m = S.occ_to_det([0], [0], norb)
    with pytest.raises(qp.QPError) as ei:
        pt2.set_target(core=m, deleted=m)
    assert ei.value.code == qp.QP_EINVAL
    pt2.close()
