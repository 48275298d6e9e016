"""Adjoint of the sweep on the GPU: dE_PT2/dh, dE_PT2/d(packed eri) and
dE_PT2/dE0 against the oracle's gradient, central finite differences of the
GPU energy, Euler's identity and torch.autograd."""
import json
import os

import numpy as np
import pytest

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


def _gpu_grad(qp, norb, na, nb, h, eri, dets, c, e0):
    import torch

    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    dh = torch.zeros((norb, norb), dtype=torch.float64, device="cuda")
    deri = torch.zeros(len(eri), dtype=torch.float64, device="cuda")
    de0, res = qp.qp_pt2_grad(pt2.ctx, len(dets), _dev(dets), _dev(c), e0, dh, deri)
    pt2.close()
    return dh.cpu().numpy(), deri.cpu().numpy(), de0, res.as_dict()


def _gpu_energy(qp, pt2, dd, cd, e0):
    return pt2.eval(dd, cd, e0, 0)["e_pt2"]


@pytest.mark.parametrize("norb,na,nb,ndet,seed", [(10, 3, 3, 40, 101), (16, 4, 4, 120, 102), (24, 5, 4, 80, 103),
                                                  (68, 2, 2, 30, 104),
                                                  (112, 3, 3, 16, 105)])  # tiled opposite-spin batches
def test_gradient_matches_oracle(qp, oracle_mod, norb, na, nb, ndet, seed):
    h, eri = S.hamiltonian(norb, min(norb + 2, 12), seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    c = S.random_coefs(len(dets), seed + 2, decay=0.05)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    ref = ham.gradient(dets, c, e0)
    dh, deri, de0, res = _gpu_grad(qp, norb, na, nb, h, eri, dets, c, e0)
    assert abs(res["e_pt2"] - ref["e_pt2"]) < 1e-10
    assert de0 == pytest.approx(ref["de0"], rel=1e-12, abs=1e-13)
    scale = max(1.0, np.abs(ref["deri"]).max(), np.abs(ref["dh"]).max())
    assert np.abs(dh - ref["dh"]).max() <= 1e-11 * scale
    assert np.abs(deri - ref["deri"]).max() <= 1e-11 * scale
    # Euler: E_PT2 is homogeneous of degree 1 in (h, eri, E0)
    assert np.sum(h * dh) + np.dot(eri, deri) + e0 * de0 == pytest.approx(res["e_pt2"], abs=1e-10)


def test_gradient_central_differences_200_entries(qp):
    """Central differences (step 1e-5) of the GPU energy on 200 random packed
    integrals and a few h entries: relative agreement 1e-6."""
    norb, na, nb = 16, 4, 4
    h, eri = S.hamiltonian(norb, 24, 105)
    dets = S.random_excited_dets(norb, na, nb, 100, 106)
    c = S.random_coefs(len(dets), 107, decay=0.05)
    e0 = float(np.min(np.diag(h))) * (na + nb) - 20.0
    dh, deri, de0, res = _gpu_grad(qp, norb, na, nb, h, eri, dets, c, e0)
    dd, cd = _dev(dets), _dev(c)
    step = 1e-5
    rng = np.random.default_rng(108)
    idx = rng.choice(np.nonzero(np.abs(deri) > 1e-6)[0], 200, replace=False)
    bad = []
    for i in idx:
        out = []
        for sgn in (+1, -1):
            e2 = eri.copy()
            e2[i] += sgn * step
            pt2 = qp.PT2(norb, na, nb, h, e2)
            out.append(_gpu_energy(qp, pt2, dd, cd, e0))
            pt2.close()
        fd = (out[0] - out[1]) / (2 * step)
        if abs(fd - deri[i]) > 1e-6 * abs(fd) + 1e-9:
            bad.append((int(i), fd, deri[i]))
    assert not bad, bad[:5]
    for p, q in [(0, 0), (3, 3), (1, 5), (6, 12)]:
        out = []
        for sgn in (+1, -1):
            h2 = h.copy()
            h2[p, q] += sgn * step
            if p != q:
                h2[q, p] += sgn * step
            pt2 = qp.PT2(norb, na, nb, h2, eri)
            out.append(_gpu_energy(qp, pt2, dd, cd, e0))
            pt2.close()
        fd = (out[0] - out[1]) / (2 * step)
        an = dh[p, p] if p == q else dh[p, q] + dh[q, p]
        assert abs(fd - an) <= 1e-6 * abs(fd) + 1e-9, (p, q, fd, an)


def test_autograd_function(qp):
    import torch

    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 109)
    dets = S.random_excited_dets(norb, na, nb, 50, 110)
    c = S.random_coefs(len(dets), 111, decay=0.05)
    e0 = float(np.min(np.diag(h))) * (na + nb) - 20.0
    ht = _dev(h).requires_grad_(True)
    et = _dev(eri).requires_grad_(True)
    e0t = torch.tensor(e0, dtype=torch.float64, device="cuda", requires_grad=True)
    E = qp.pt2_energy(ht, et, _dev(dets), _dev(c), e0t, na, nb)
    E.backward()
    dh, deri, de0, res = _gpu_grad(qp, norb, na, nb, h, eri, dets, c, e0)
    assert float(E.detach()) == pytest.approx(res["e_pt2"], abs=1e-12)
    assert np.allclose(ht.grad.cpu().numpy(), dh, rtol=1e-12, atol=1e-14)
    assert np.allclose(et.grad.cpu().numpy(), deri, rtol=1e-12, atol=1e-14)
    assert float(e0t.grad) == pytest.approx(de0, rel=1e-12)


def test_gradient_golden_cfg4(qp):
    """The adjoint workload (48 orbitals, 8+8 electrons, 2*10^4 determinants):
    the GPU gradient against the oracle's full gradient."""
    p = os.path.join(GOLDEN, "cfg4_psi0.npz")
    gfile = os.path.join(GOLDEN, "cfg4_gradient.npz")
    if not (os.path.exists(p) and os.path.exists(gfile)):
        pytest.skip("cfg4 golden files absent")
    P = np.load(p)
    G = np.load(gfile)
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    dh, deri, de0, res = _gpu_grad(qp, meta["norb"], meta["nalpha"], meta["nbeta"], h, eri, P["dets"],
                                   P["coefs"], float(P["e0"]))
    assert abs(res["e_pt2"] - float(G["e_pt2"])) < 1e-10
    scale = max(1.0, np.abs(G["deri"]).max())
    assert np.abs(deri - G["deri"]).max() <= 1e-10 * scale
    assert np.abs(dh - G["dh"]).max() <= 1e-10 * scale
    assert de0 == pytest.approx(float(G["de0"]), rel=1e-11)
