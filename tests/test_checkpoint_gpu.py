"""A sweep stopped after a few blocks of generator ranks and resumed from
its checkpoint gives the same bits as one uninterrupted sweep (Eq.
edetstoch: E_PT2 = sum_I eps_I, each eps_I independent of the others)."""
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


def test_resumed_sweep_equals_one_sweep(qp, tmp_path):
    import torch

    from paper_1902_08154_gb300.checkpoint import resumable_sweep

    P = np.load(os.path.join(GOLDEN, "cfg2_psi0.npz"))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    n = 2500
    dets = torch.from_numpy(P["dets"][:n].view(np.int64)).cuda()
    c = torch.from_numpy(P["coefs"][:n].copy()).cuda()
    e0 = float(P["e0"])
    k = 400
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], torch.from_numpy(h).cuda(), torch.from_numpy(eri).cuda())
    ref = pt2.eval(dets, c, e0, k, per_generator=True)
    path = str(tmp_path / "sweep.ck.npz")
    assert resumable_sweep(pt2, dets, c, e0, k, path, block=300, stop_after=3) is None
    assert os.path.exists(path)
    got = resumable_sweep(pt2, dets, c, e0, k, path, block=300)
    bits = lambda x: np.float64(x).view(np.uint64)  # noqa: E731
    assert bits(got["e_pt2"]) == bits(ref["e_pt2"])
    assert bits(got["sum_e_over_d"]) == bits(ref["sum_e_over_d"])
    assert bits(got["e_rpt2"]) == bits(ref["e_rpt2"])
    assert got["n_perturbers"] == ref["n_perturbers"] and got["n_connections"] == ref["n_connections"]
    assert tuple(got["digest"]) == tuple(ref["digest"])
    assert np.array_equal(got["eps_by_rank"].view(np.uint64), ref["eps_by_rank"].cpu().numpy().view(np.uint64))
    assert np.array_equal(got["sel_dets"].reshape(k, -1), ref["sel_dets"].cpu().numpy().view(np.uint64).reshape(k, -1))
    assert np.array_equal(got["sel_e"], ref["sel_e"].cpu().numpy())
    # a checkpoint of another sweep is refused
    with pytest.raises(ValueError):
        resumable_sweep(pt2, dets, c, e0, k + 1, path, block=300)
    pt2.close()
