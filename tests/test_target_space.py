"""Target spaces (Sec. "Selected CI": the method applies to CAS, CIS, CISD
... spaces by zeroing the contributions of external determinants outside
the target space).  The oracle's restricted sweep is pinned against a
dense-H sum over the external determinants that pass an independent numpy
membership test."""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.sq_hamiltonian import dense_h


def _space(oracle_mod, norb, na, nb, nint_, seed):
    h, eri = S.hamiltonian(norb, norb + 3, 300 + seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    fci = S.all_dets(norb, na, nb)
    Hm = dense_h(fci, h, eri, norb)
    rng = np.random.default_rng(seed)
    low = list(np.argsort(np.diag(Hm), kind="stable")[: nint_ - 4])
    rest = [i for i in range(len(fci)) if i not in set(low)]
    idx = np.sort(np.array(low + list(rng.choice(rest, 4, replace=False))))
    w, v = np.linalg.eigh(Hm[np.ix_(idx, idx)])
    return ham, fci, Hm, idx, v[:, 0], w[0]


def _bits(d):
    return [int(x) for x in np.asarray(d, dtype=np.uint64).reshape(-1)]


def _member(d, ref, max_exc, core, deleted):
    words = _bits(d)
    if core is not None and any((w & c) != c for w, c in zip(words, _bits(core))):
        return False
    if deleted is not None and any(w & x for w, x in zip(words, _bits(deleted))):
        return False
    if ref is not None and max_exc >= 0:
        moved = sum(bin(w ^ r).count("1") for w, r in zip(words, _bits(ref))) // 2
        return moved <= max_exc
    return True


def _dense_restricted(fci, Hm, idx, c, e0, member):
    ext = np.array([i for i in range(len(fci)) if i not in set(idx.tolist())])
    A = Hm[np.ix_(ext, idx)] @ c
    D = e0 - np.diag(Hm)[ext]
    conn = np.any(Hm[np.ix_(ext, idx)] != 0.0, axis=1)
    keep = np.array([member(fci[i]) for i in ext]) & conn
    return float(np.sum((A * A / D)[keep])), int(keep.sum())


def _targets(norb, na, nb):
    hf = S.hf_det(norb, na, nb)
    core = S.occ_to_det([0], [0], norb)
    deleted = S.occ_to_det([norb - 1], [norb - 1], norb)
    return [
        dict(ref=hf, max_exc=2),                       # CISD around the reference
        dict(ref=hf, max_exc=1),                       # CIS
        dict(core=core, deleted=deleted),              # a CAS: orbital 0 doubly occupied, the last one empty
        dict(ref=hf, max_exc=3, core=core),            # both kinds at once
    ]


@pytest.mark.parametrize("norb,na,nb,nint_,seed", [(8, 3, 2, 40, 1), (9, 3, 3, 60, 2)])
def test_restricted_sweep_matches_dense_sum(oracle_mod, norb, na, nb, nint_, seed):
    ham, fci, Hm, idx, c, e0 = _space(oracle_mod, norb, na, nb, nint_, seed)
    dets = fci[idx]
    for t in _targets(norb, na, nb):
        member = lambda d: _member(d, t.get("ref"), t.get("max_exc", -1), t.get("core"), t.get("deleted"))
        e_ref, n_ref = _dense_restricted(fci, Hm, idx, c, e0, member)
        ham.set_target(**t)
        out = ham.sweep(dets, c, e0, k=len(fci))
        assert out["n_perturbers"] == n_ref
        assert abs(out["e_pt2"] - e_ref) < 1e-12
        assert all(member(d) for d in out["sel_dets"])
        gens = [ham.generator(dets, c, e0, g) for g in range(len(dets))]
        assert abs(sum(r["eps"] for r in gens) - e_ref) < 1e-12
    ham.set_target()  # cleared: the full external space again
    e_all, n_all = _dense_restricted(fci, Hm, idx, c, e0, lambda d: True)
    out = ham.sweep(dets, c, e0, k=0)
    assert out["n_perturbers"] == n_all and abs(out["e_pt2"] - e_all) < 1e-12


def test_target_that_holds_everything_changes_nothing(oracle_mod):
    ham, fci, Hm, idx, c, e0 = _space(oracle_mod, 8, 2, 2, 30, 3)
    dets = fci[idx]
    full = ham.sweep(dets, c, e0, k=20)
    ham.set_target(ref=S.hf_det(8, 2, 2), max_exc=4)
    same = ham.sweep(dets, c, e0, k=20)
    assert same["e_pt2"] == full["e_pt2"] and same["n_perturbers"] == full["n_perturbers"]
    assert tuple(same["digest"]) == tuple(full["digest"])
