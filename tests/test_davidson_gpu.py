"""The variational step on the GPU (Sec. "Davidson diagonalization"): H over
Psi0 (qp_pt2_sigma) against the oracle's matrix, and the lowest eigenpair
(qp_pt2_davidson) against dense diagonalisation and the stored workloads'
E0, which the oracle's Davidson produced."""
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


@pytest.mark.parametrize("norb,na,nb,ndet,seed,rank", [(12, 3, 3, 120, 61, 14), (20, 5, 4, 200, 62, 22),
                                                       (70, 3, 3, 90, 63, 6)])
def test_sigma_matches_oracle_matrix(qp, oracle_mod, norb, na, nb, ndet, seed, rank):
    from oracle import psi0

    h, eri = S.hamiltonian(norb, rank, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    Hd = psi0.hamiltonian_matrix(ham, dets).toarray()
    U = np.random.default_rng(seed).standard_normal((3, len(dets)))
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    got = pt2.sigma(_dev(dets), _dev(U)).cpu().numpy()
    ref = U @ Hd  # H is symmetric
    assert np.abs(got - ref).max() <= 1e-11 * max(1.0, np.abs(ref).max())
    # host arrays in and out give the same product
    assert np.array_equal(pt2.sigma(dets, U), got)
    pt2.close()


def test_davidson_matches_dense_diagonalisation(qp, oracle_mod):
    from oracle import psi0

    norb, na, nb = 14, 4, 3
    h, eri = S.hamiltonian(norb, 16, 64)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 300, 65)
    w, v = np.linalg.eigh(psi0.hamiltonian_matrix(ham, dets).toarray())
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    e0, c, info = pt2.davidson(_dev(dets), tol=1e-10)
    c = c.cpu().numpy()
    assert info["converged"] and info["residual"] <= 1e-10
    assert e0 == pytest.approx(w[0], abs=1e-10)
    assert abs(abs(np.dot(c, v[:, 0])) - 1.0) <= 1e-12
    assert c[0] >= 0
    pt2.close()


@pytest.mark.parametrize("name", ["cfg1", "cfg2"])
def test_davidson_reproduces_stored_e0(qp, name):
    P = np.load(os.path.join(GOLDEN, f"{name}_psi0.npz"))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    e0, c, info = pt2.davidson(_dev(P["dets"]), tol=1e-10)
    c = c.cpu().numpy()
    print(f"{name}: E0 {e0:.12f} (stored {float(P['e0']):.12f}), {info['iterations']} iterations, "
          f"nnz {info['nnz']}, build {info['build_ms']:.1f} ms, solve {info['solve_ms']:.1f} ms")
    assert e0 == pytest.approx(float(P["e0"]), abs=1e-9)
    assert abs(abs(np.dot(c, P["coefs"])) - 1.0) <= 1e-10
    pt2.close()


def test_davidson_rejects_duplicates(qp):
    norb, na, nb = 10, 3, 3
    h, eri = S.hamiltonian(norb, 12, 66)
    dets = S.random_excited_dets(norb, na, nb, 30, 67)
    dup = np.concatenate([dets, dets[4:5]])
    pt2 = qp.PT2(norb, na, nb, h, eri)
    with pytest.raises(qp.QPError) as ei:
        pt2.davidson(dup)
    assert ei.value.code == qp.QP_EDUP
    pt2.close()


def test_cipsi_growth_matches_oracle(qp, oracle_mod):
    """Two CIPSI doublings on the GPU (sweep + selection + Davidson) against
    the oracle's growth rule from the same seed space."""
    from oracle import psi0

    from paper_1902_08154_gb300 import cipsi

    norb, na, nb = 16, 4, 4
    h, eri = S.hamiltonian(norb, 32, 0)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    hf = S.hf_det(norb, na, nb)
    ref_dets, ref_c, ref_e0, ref_info = psi0.cipsi_grow(ham, hf, 200, doublings=2)
    seed = psi0.seed_space(ham, hf, 50)
    e0, c, _ = psi0.ground_state(ham, seed)
    pt2 = qp.PT2(norb, na, nb, h, eri)
    dets, coefs, e_fin, info = cipsi.grow(pt2, seed, c, e0, 2)
    pt2.close()
    for a, b in zip(info, ref_info):
        assert a["ndet"] == b["ndet"]
        assert a["e0"] == pytest.approx(b["e0"], abs=1e-9)
        if "e_pt2" in b:
            assert a["e_pt2"] == pytest.approx(b["e_pt2"], abs=1e-10)
    assert {d.tobytes() for d in dets} == {d.tobytes() for d in ref_dets}
    assert e_fin == pytest.approx(ref_e0, abs=1e-9)


def test_davidson_two_words_per_spin(qp, oracle_mod):
    """Determinants across the 64-bit word boundary (70 orbitals)."""
    from oracle import psi0

    norb, na, nb = 70, 3, 3
    h, eri = S.hamiltonian(norb, 6, 68)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 250, 69)
    w, v = np.linalg.eigh(psi0.hamiltonian_matrix(ham, dets).toarray())
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    e0, c, info = pt2.davidson(_dev(dets), tol=1e-10)
    pt2.close()
    assert e0 == pytest.approx(w[0], abs=1e-10)
    assert abs(abs(np.dot(c.cpu().numpy(), v[:, 0])) - 1.0) <= 1e-12


def _csr_dense(n, rowptr, cols, vals, diag):
    H = np.zeros((n, n))
    for i in range(n):
        H[i, cols[rowptr[i]:rowptr[i + 1]]] = vals[rowptr[i]:rowptr[i + 1]]
    H[np.arange(n), np.arange(n)] = diag
    return H


@pytest.mark.parametrize("norb,na,nb,ndet,seed,rank", [(12, 3, 3, 150, 71, 14), (16, 4, 4, 300, 72, 18),
                                                       (70, 3, 3, 120, 73, 6), (128, 2, 2, 80, 74, 3)])
def test_string_search_matches_all_pairs_and_oracle(qp, oracle_mod, norb, na, nb, ndet, seed, rank):
    """The pair search through the spin strings (Appendix "Davidson
    diagonalization") gives the same CSR matrix, element for element, as the
    test of every pair, and the same matrix as the oracle's."""
    from oracle import psi0

    h, eri = S.hamiltonian(norb, rank, seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri))
    a = pt2.hamiltonian(_dev(dets), search=0)
    b = pt2.hamiltonian(dets, search=1)
    pt2.close()
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    ref = psi0.hamiltonian_matrix(ham, dets).toarray()
    got = _csr_dense(len(dets), *a[:4])
    assert np.abs(got - ref).max() <= 1e-12 * max(1.0, np.abs(ref).max())


def test_string_search_full_ci_and_duplicates(qp, oracle_mod):
    """Every determinant of a full CI space: each one meets all of its
    singles and doubles; a repeated determinant is refused (QP_EDUP)."""
    norb, na, nb = 7, 3, 2
    h, eri = S.hamiltonian(norb, 9, 75)
    fci = S.all_dets(norb, na, nb)
    pt2 = qp.PT2(norb, na, nb, h, eri)
    rowptr, cols, vals, diag, _ = pt2.hamiltonian(fci, search=0)
    deg = lambda a, b: int(sum(bin(int(x) ^ int(y)).count("1") for x, y in zip(a.ravel(), b.ravel()))) // 2
    for i in range(0, len(fci), 7):
        expect = sorted(j for j in range(len(fci)) if j != i and deg(fci[i], fci[j]) <= 2)
        assert list(cols[rowptr[i]:rowptr[i + 1]]) == expect
    dup = np.concatenate([fci[:20], fci[5:6]])
    with pytest.raises(qp.QPError) as ei:
        pt2.hamiltonian(dup, search=0)
    assert ei.value.code == qp.QP_EDUP
    pt2.close()


def test_string_search_on_the_cfg2_psi0(qp):
    """The 10^4-determinant workload: the string search and the all-pairs
    test build the same matrix, bit for bit."""
    P = np.load(os.path.join(GOLDEN, "cfg2_psi0.npz"))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], _dev(h), _dev(eri))
    d = _dev(P["dets"])
    a = pt2.hamiltonian(d, search=0)
    b = pt2.hamiltonian(d, search=1)
    pt2.close()
    for x, y in zip(a[:4], b[:4]):
        assert np.array_equal(x, y)
    print(f"cfg2 H build: strings {a[4]:.2f} ms, all pairs {b[4]:.2f} ms, nnz {len(a[1])}")
