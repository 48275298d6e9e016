"""The seeded synthetic inputs: well-formed spaces and E0 below every
diagonal energy (so that no denominator E0 - H_aa can vanish)."""
import numpy as np

from paper_1902_08154_gb300 import synthetic as S


def _check_space(oracle_mod, h, eri, dets, coefs, e0, norb, na, nb, n_diag=64):
    ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
    assert ham.validate(dets) == 0  # occupations, bits beyond norb, duplicates
    assert abs(np.linalg.norm(coefs) - 1.0) < 1e-12
    assert np.all(np.diag(h) == -2.0 + 0.15 * np.arange(norb))
    rng = np.random.default_rng(0)
    for i in rng.choice(len(dets), min(n_diag, len(dets)), replace=False):
        assert e0 < ham.diag(dets[i]) - 0.5
    # the bound also holds for substitutions of the space (the perturbers)
    for a in ham.substitutions(dets[0])[:: max(1, len(ham.substitutions(dets[0])) // 64)]:
        assert e0 < ham.diag(a) - 0.5


def test_cfg3_instance(oracle_mod):
    h, eri, dets, coefs, e0 = S.cfg3_instance()
    spec = S.CFG3
    assert dets.shape == (spec["ndet"], 2, 2) and dets.dtype == np.uint64
    assert eri.shape == (S.packed_len(spec["norb"]),)
    _check_space(oracle_mod, h, eri, dets, coefs, e0, spec["norb"], spec["nalpha"], spec["nbeta"])
    # the reduced form keeps the head of the same list
    h2, eri2, d2, c2, e02 = S.cfg3_instance(10)
    assert np.array_equal(d2, dets[:10]) and e02 == e0 and len(c2) == 10


def test_batch_instance_small(oracle_mod):
    spec = dict(norb=24, nalpha=6, nbeta=6, ndet=200, rank=36, seed=5)
    h, eri, dets, coefs, e0 = S.batch_instance(spec)
    assert dets.shape == (200, 2, 1)
    _check_space(oracle_mod, h, eri, dets, coefs, e0, 24, 6, 6)
