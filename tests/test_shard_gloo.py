"""Generator sharding across processes (world size 2, gloo, CPU).

Each rank takes the generators of rank r with r % 2 == its index, forms its
partial totals, digest and selection from the oracle's per-generator
definition (no GPU here), and the exchange step of the sharded sweep
(``shard.distributed_merge``) must reproduce the oracle's full sweep exactly:
same perturber set and counts, E_PT2 to 1e-12, same selection.
"""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _case():
    import oracle
    from paper_1902_08154_gb300 import synthetic as S

    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 61)
    ham = oracle.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 50, seed=62)
    c = S.random_coefs(50, 63, decay=0.05)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    return ham, dets, c, e0


def _worker(rank, world, port, k, out_path):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1902_08154_gb300.shard import distributed_merge, merge_selections

    ham, dets, c, e0 = _case()
    res = {"e_pt2": 0.0, "sum_e_over_d": 0.0, "n_perturbers": 0, "n_connections": 0, "n_tiny": 0,
           "digest": (0, 0), "min_abs_den": float("inf")}
    es, ds = [], []
    d0, d1 = 0, 0
    for g in range(rank, len(dets), world):
        r = ham.generator(dets, c, e0, g, cap=10**6, nthreads=1)
        res["e_pt2"] += r["eps"]
        res["sum_e_over_d"] += r["sum_e_over_d"]
        res["n_perturbers"] += r["n_perturbers"]
        res["n_connections"] += r["n_connections"]
        d0 = (d0 + r["digest"][0]) & ((1 << 64) - 1)
        d1 ^= r["digest"][1]
        es.append(r["e"])
        ds.append(r["dets"].reshape(len(r["e"]), -1))
    res["digest"] = (d0, d1)
    le, ld = merge_selections(es, ds, k)  # this shard's own k best
    tot, e, d = distributed_merge(dist, res, torch.from_numpy(le),
                                  torch.from_numpy(ld.view(np.int64).reshape(len(le), 2, -1)), k, "cpu", e0)
    if rank == 0:
        np.savez(out_path, e=e, d=d, e_pt2=tot["e_pt2"], n=tot["n_perturbers"], nc=tot["n_connections"],
                 d0=np.uint64(tot["digest"][0]), d1=np.uint64(tot["digest"][1]), z=tot["z"],
                 e_rpt2=tot["e_rpt2"], s2=tot["sum_e_over_d"])
    dist.barrier()
    dist.destroy_process_group()


@pytest.fixture(scope="module")
def library():
    """The exchange step's arithmetic is the library's (qp_pt2_merge_results,
    no GPU needed): build it before the ranks start."""
    from paper_1902_08154_gb300 import build

    build.build()


def test_two_rank_merge_matches_full_sweep(tmp_path, oracle_mod, library):
    import torch.multiprocessing as mp

    k = 25
    out = str(tmp_path / "merged.npz")
    mp.start_processes(_worker, args=(2, _free_port(), k, out), nprocs=2, start_method="spawn", join=True)
    ham, dets, c, e0 = _case()
    ref = ham.sweep(dets, c, e0, k=k)
    m = np.load(out)
    assert int(m["n"]) == ref["n_perturbers"]
    assert int(m["nc"]) == ref["n_connections"]
    assert (int(m["d0"]), int(m["d1"])) == tuple(ref["digest"])
    assert abs(float(m["e_pt2"]) - ref["e_pt2"]) < 1e-12
    # Z and E_rPT2 of the merged sums (Sec. "Renormalized PT2")
    assert float(m["z"]) == pytest.approx(1.0 / (1.0 + ref["sum_e_over_d"]), rel=1e-12)
    assert float(m["e_rpt2"]) == pytest.approx(e0 + float(m["z"]) * ref["e_pt2"], abs=1e-12)
    assert np.array_equal(m["d"], ref["sel_dets"].reshape(k, -1))
    assert np.allclose(m["e"], ref["sel_e"], rtol=1e-12, atol=1e-15)


def test_merge_selection_order():
    from paper_1902_08154_gb300.shard import merge_selections

    e1 = np.array([-0.5, -0.1, 0.3])
    d1 = np.array([[5, 1], [2, 2], [9, 9]], dtype=np.uint64)
    e2 = np.array([0.5, -0.3])
    d2 = np.array([[4, 1], [1, 1]], dtype=np.uint64)
    e, d = merge_selections([e1, e2], [d1, d2], 4)
    # |e| ties (0.5, 0.5) are broken by the key: [4,1] < [5,1]
    assert d.tolist() == [[4, 1], [5, 1], [1, 1], [9, 9]]
    assert e.tolist() == [0.5, -0.5, -0.3, 0.3]


def _states_case():
    import oracle
    from paper_1902_08154_gb300 import synthetic as S

    ham, dets, c, e0 = _case()
    c1 = S.random_coefs(len(dets), 64, decay=0.02)
    return ham, dets, np.stack([c, c1]), [e0, e0 - 0.15]


def _states_worker(rank, world, port, k, out_path):
    import torch
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1902_08154_gb300.shard import distributed_merge

    ham, dets, C, E0 = _states_case()
    # this rank's generators (rank r % world), several states at once
    r = ham.states(dets, C, E0, k=k, nthreads=1, shard=(rank, world))
    tot, e, d = distributed_merge(dist, r, torch.from_numpy(r["sel_crit"]),
                                  torch.from_numpy(r["sel_dets"].view(np.int64)), k, "cpu")
    if rank == 0:
        np.savez(out_path, e=e, d=d, e_states=tot["e_pt2_states"], s_states=tot["sum_e_over_d_states"],
                 n=tot["n_perturbers"], nc=tot["n_connections"], d0=np.uint64(tot["digest"][0]),
                 d1=np.uint64(tot["digest"][1]))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_merge_of_a_multi_state_sweep(tmp_path, oracle_mod, library):
    import torch.multiprocessing as mp

    k = 30
    out = str(tmp_path / "merged_states.npz")
    mp.start_processes(_states_worker, args=(2, _free_port(), k, out), nprocs=2, start_method="spawn", join=True)
    ham, dets, C, E0 = _states_case()
    ref = ham.states(dets, C, E0, k=k)
    m = np.load(out)
    assert int(m["n"]) == ref["n_perturbers"]
    assert int(m["nc"]) == ref["n_connections"]
    assert (int(m["d0"]), int(m["d1"])) == tuple(ref["digest"])
    np.testing.assert_allclose(m["e_states"], ref["e_pt2_states"], rtol=0, atol=1e-12)
    np.testing.assert_allclose(m["s_states"], ref["sum_e_over_d_states"], rtol=1e-12, atol=0)
    assert np.array_equal(m["d"], ref["sel_dets"].reshape(k, -1))
    np.testing.assert_allclose(m["e"], ref["sel_crit"], rtol=1e-12, atol=0)
