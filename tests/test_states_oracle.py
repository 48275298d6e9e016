"""Pins of the oracle's multi-state sweep (Sec. "Selected CI": one PT2 per
state and the selection criterion of Angeli et al.).

Each test compares ``Hamiltonian.states`` with something else: a dense-H
construction over the whole external space (explicit second quantisation,
numpy matrix products, degrees by bit counting), the single-state sweep (a
separate code path that groups pairs by alpha), or a symmetry of the
definition.
"""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.sq_hamiltonian import dense_h

pytestmark = pytest.mark.filterwarnings("ignore::RuntimeWarning")


def _degrees(a, b):
    """Excitation degree between every row of a and every row of b (bit counts)."""
    x = np.bitwise_xor(a.reshape(len(a), 1, -1), b.reshape(1, len(b), -1))
    bits = np.unpackbits(x.view(np.uint8), axis=-1).sum(axis=-1)
    return bits // 2


@pytest.mark.parametrize("norb,na,nb,nint_,seed", [(6, 2, 2, 30, 1), (7, 3, 2, 45, 2)])
def test_states_match_dense_sums(oracle_mod, norb, na, nb, nint_, seed):
    h, eri = S.hamiltonian(norb, norb + 3, 200 + seed)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    fci = S.all_dets(norb, na, nb)
    Hm = dense_h(fci, h, eri, norb)
    rng = np.random.default_rng(seed)
    low = list(np.argsort(np.diag(Hm), kind="stable")[: nint_ - 5])
    rest = [i for i in range(len(fci)) if i not in set(low)]
    idx = np.sort(np.array(low + list(rng.choice(rest, 5, replace=False))))
    # three states of the internal space: its three lowest eigenvectors
    w, v = np.linalg.eigh(Hm[np.ix_(idx, idx)])
    nst = 3
    C, E0 = v[:, :nst].T.copy(), w[:nst].copy()
    ext = np.setdiff1d(np.arange(len(fci)), idx)
    deg = _degrees(fci[ext], fci[idx])
    reach = deg <= 2
    connected = reach.any(axis=1)
    ext, deg, reach = ext[connected], deg[connected], reach[connected]
    A = Hm[np.ix_(ext, idx)] @ C.T                     # [n_ext, nst]
    D = E0[None, :] - np.diag(Hm)[ext][:, None]
    e = A * A / D
    crit = (e / np.max(C * C, axis=1)[None, :]).sum(axis=1)

    out = ham.states(fci[idx], C, E0, k=len(ext))
    assert out["n_perturbers"] == len(ext)
    assert out["n_connections"] == int(reach.sum())
    np.testing.assert_allclose(out["e_pt2_states"], e.sum(axis=0), rtol=0, atol=1e-12)
    np.testing.assert_allclose(out["sum_e_over_d_states"], ((A / D) ** 2).sum(axis=0), rtol=1e-12)
    assert out["min_abs_den"] == pytest.approx(np.min(np.abs(D)), rel=1e-14)
    got = {d.tobytes(): (c, a) for d, c, a in zip(out["sel_dets"], out["sel_crit"], out["sel_num"])}
    for j, i in enumerate(ext):
        c, a = got[fci[i].tobytes()]
        assert abs(c - crit[j]) < 1e-12
        assert abs(a - A[j, 0]) < 1e-13
    # top 10 by |criterion|, ties by key
    order = sorted(range(len(ext)),
                   key=lambda j: (-abs(crit[j]), tuple(int(x) for x in fci[ext[j]].reshape(-1))))
    top = ham.states(fci[idx], C, E0, k=10)
    assert [d.tobytes() for d in top["sel_dets"]] == [fci[ext[j]].tobytes() for j in order[:10]]


def _space(oracle_mod):
    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 41)
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 50, seed=42)
    e0 = min(ham.diag(d) for d in dets) - 0.3
    return ham, dets, e0


def test_one_state_is_the_single_state_sweep(oracle_mod):
    ham, dets, e0 = _space(oracle_mod)
    c = S.random_coefs(len(dets), 43, decay=0.05)
    a = ham.sweep(dets, c, e0, k=40)
    b = ham.states(dets, c[None, :], [e0], k=40)
    assert b["e_pt2_states"][0] == pytest.approx(a["e_pt2"], abs=1e-12)
    assert b["sum_e_over_d_states"][0] == pytest.approx(a["sum_e_over_d"], rel=1e-12)
    for key in ("n_perturbers", "n_connections", "n_tiny", "digest"):
        assert a[key] == b[key]
    # one state: e~ = e / max c^2, so the ranking is that of |e|
    assert np.array_equal(a["sel_dets"], b["sel_dets"])
    np.testing.assert_allclose(b["sel_crit"] * np.max(c * c), a["sel_e"], rtol=1e-13, atol=0)
    np.testing.assert_allclose(b["sel_num"], a["sel_num"], rtol=1e-12, atol=1e-15)


def test_equal_states_and_state_order(oracle_mod):
    ham, dets, e0 = _space(oracle_mod)
    c0 = S.random_coefs(len(dets), 44, decay=0.05)
    c1 = S.random_coefs(len(dets), 45, decay=0.02)
    one = ham.states(dets, c0[None, :], [e0], k=30)
    two = ham.states(dets, np.stack([c0, c0]), [e0, e0], k=30)
    assert two["e_pt2_states"][0] == two["e_pt2_states"][1] == one["e_pt2_states"][0]
    assert np.array_equal(two["sel_dets"], one["sel_dets"])
    np.testing.assert_allclose(two["sel_crit"], 2.0 * one["sel_crit"], rtol=1e-14, atol=0)
    # exchanging the states exchanges the energies and keeps the criterion
    a = ham.states(dets, np.stack([c0, c1]), [e0, e0 - 0.1], k=30)
    b = ham.states(dets, np.stack([c1, c0]), [e0 - 0.1, e0], k=30)
    assert a["e_pt2_states"][0] == pytest.approx(b["e_pt2_states"][1], abs=1e-14)
    assert a["e_pt2_states"][1] == pytest.approx(b["e_pt2_states"][0], abs=1e-14)
    assert np.array_equal(a["sel_dets"], b["sel_dets"])
    np.testing.assert_allclose(a["sel_crit"], b["sel_crit"], rtol=1e-14, atol=0)
    # a state's weight 1/max c^2 makes the criterion invariant to its scale
    d = ham.states(dets, np.stack([c0, 3.0 * c1]), [e0, e0 - 0.1], k=30)
    np.testing.assert_allclose(d["sel_crit"], a["sel_crit"], rtol=1e-12, atol=0)
    assert d["e_pt2_states"][1] == pytest.approx(9.0 * a["e_pt2_states"][1], rel=1e-12)


def test_states_rejects_a_zero_state(oracle_mod):
    ham, dets, e0 = _space(oracle_mod)
    c0 = S.random_coefs(len(dets), 46)
    with pytest.raises(ValueError):
        ham.states(dets, np.stack([c0, np.zeros_like(c0)]), [e0, e0], k=5)


def test_states_shards_follow_the_generator_rule(oracle_mod):
    """Shard (i, n) keeps the perturbers of the generators of rank i mod n
    (Eqs. calpha, edetstoch): with one state its energy is the sum of the
    one-state sweep's eps over those ranks; the shards add up to the whole."""
    ham, dets, e0 = _space(oracle_mod)
    c0 = S.random_coefs(len(dets), 47, decay=0.05)
    c1 = S.random_coefs(len(dets), 48, decay=0.02)
    ref = ham.sweep(dets, c0, e0, k=0)
    n = 3
    for i in range(n):
        part = ham.states(dets, c0[None, :], [e0], k=0, shard=(i, n))
        assert part["e_pt2_states"][0] == pytest.approx(ref["eps_by_rank"][i::n].sum(), abs=1e-12)
        assert part["n_perturbers"] == int(ref["na_by_rank"][i::n].sum())
        assert part["n_connections"] == int(ref["ncon_by_rank"][i::n].sum())
    C, E0 = np.stack([c0, c1]), [e0, e0 - 0.2]
    full = ham.states(dets, C, E0, k=10**6)
    parts = [ham.states(dets, C, E0, k=10**6, shard=(i, n)) for i in range(n)]
    assert sum(p["n_perturbers"] for p in parts) == full["n_perturbers"]
    assert sum(p["n_connections"] for p in parts) == full["n_connections"]
    np.testing.assert_allclose(sum(p["e_pt2_states"] for p in parts), full["e_pt2_states"], rtol=0, atol=1e-12)
    assert (sum(p["digest"][0] for p in parts) % (1 << 64)) == full["digest"][0]
    keys = sorted(d.tobytes() for p in parts for d in p["sel_dets"])
    assert keys == sorted(d.tobytes() for d in full["sel_dets"])
