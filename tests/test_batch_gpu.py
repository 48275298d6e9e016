"""Batched sweeps captured into one CUDA graph: every instance must give what
its own sweep gives (and what the oracle gives), on two runs of the graph."""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import check_selection, check_totals, cipsi_space

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


SPECS = [  # norb, na, nb, ndet, k, seed, precision (0 FP64, 1 mixed)
    (12, 3, 3, 60, 30, 201, 0),
    (16, 4, 4, 150, 100, 202, 0),
    (24, 6, 6, 90, 40, 203, 1),
    (20, 5, 4, 120, 50, 204, 0),
    (70, 3, 3, 50, 20, 205, 0),
    (32, 6, 6, 40, 25, 206, 1),
]


@pytest.fixture(scope="module")
def qp():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1902_08154_gb300 import build

    build.build()
    import paper_1902_08154_gb300 as qp

    qp.load()
    return qp


def test_batch_matches_single_sweeps_and_oracle(qp, oracle_mod):
    insts, refs = [], []
    for norb, na, nb, ndet, k, seed, prec in SPECS:
        h, eri = S.hamiltonian(norb, norb + 2, seed)
        ham = oracle_mod.Hamiltonian(norb, na, nb, h, eri)
        # Psi0 grown by the oracle's CIPSI rule, unit norm, variational E0:
        # the shape on which the mixed form states its 1e-6 Eh bound
        dets, c, e0 = cipsi_space(oracle_mod, ham, norb, na, nb, ndet)
        refs.append(ham.sweep(dets, c, e0, k=k))
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), precision=prec)
        insts.append({"pt2": pt2, "dets": _dev(dets), "coefs": _dev(c), "e0": e0, "k": k, "precision": prec})
    single = [i["pt2"].eval(i["dets"], i["coefs"], i["e0"], i["k"]) for i in insts]
    # every context in the batch gets fresh workspaces sized by the batch plan
    batch = qp.Batch(insts, max_streams=4)
    for run in range(2):
        res, ms = batch.run()
        assert ms > 0
        for i, (r, s, ref, inst) in enumerate(zip(res, single, refs, insts)):
            if inst["precision"] == 0:
                check_totals(r, ref)
                check_selection(r["sel_dets"], r["sel_e"], ref["sel_dets"], ref["sel_e"])
                assert abs(r["e_pt2"] - s["e_pt2"]) < 1e-11
            else:
                assert r["n_perturbers"] == ref["n_perturbers"] and tuple(r["digest"]) == tuple(ref["digest"])
                assert abs(r["e_pt2"] - ref["e_pt2"]) <= 1e-6
                assert abs(r["e_pt2"] - s["e_pt2"]) < 1e-9
    batch.close()


def test_autotuner_picks_a_measured_shape(qp, tmp_path):
    from paper_1902_08154_gb300 import autotune

    import torch

    insts = []
    for norb, na, nb, ndet, k, seed, prec in SPECS[:3]:
        h, eri = S.hamiltonian(norb, norb + 2, seed)
        dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
        c = S.random_coefs(len(dets), seed + 2, decay=0.05)
        e0 = float(np.min(np.diag(h))) * (na + nb) - 20.0
        pt2 = qp.PT2(norb, na, nb, _dev(h), _dev(eri), precision=prec)
        insts.append({"pt2": pt2, "dets": _dev(dets), "coefs": _dev(c), "e0": e0, "k": k, "precision": prec})
    nsm = torch.cuda.get_device_properties(0).multi_processor_count
    cache = str(tmp_path / "tune.json")
    grid, streams, rec = autotune.tune(insts, nsm, repeats=1, cache=cache)
    assert len(grid) == len(insts) and streams in (8, 16)
    assert rec["ms"] == min(t["ms"] for t in rec["tried"])
    grid2, streams2, rec2 = autotune.tune(insts, nsm, repeats=1, cache=cache)  # cached
    assert grid2 == grid and streams2 == streams
