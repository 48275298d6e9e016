"""Checkpoint/resume by generator rank and the handling of helpers that fail
(Secs. "Parallelism" and "Stochastic selection": generators are independent,
helpers may join or leave, stored eps_I are reused), on the CPU.

Failures are made on the host: a helper process that takes a block and
exits without answering, a helper that answers twice, a lease that runs out
under a fake clock.  The per-generator values come from the oracle's
per-generator definition, so no GPU is needed; the result of the whole run
must equal the oracle's full sweep rank by rank.
"""
import multiprocessing as mp
import os
import queue
import time

import numpy as np
import pytest

from paper_1902_08154_gb300.checkpoint import Coordinator, RankLedger, rank_blocks


def _case():
    import oracle
    from paper_1902_08154_gb300 import synthetic as S

    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 14, 161)
    ham = oracle.Hamiltonian(norb, na, nb, h, eri)
    dets = S.random_excited_dets(norb, na, nb, 40, seed=162)
    c = S.random_coefs(40, 163, decay=0.05)
    c /= np.linalg.norm(c)
    e0 = min(ham.diag(d) for d in dets) - 1.0
    return ham, dets, c, e0


def _block_result(ham, dets, c, e0, ranks, k):
    """What a helper returns for a block, from the oracle's per-generator
    definition (the fields of PT2.eval_generators)."""
    from paper_1902_08154_gb300.shard import merge_selections

    rs = [ham.generator(dets, c, e0, int(g), cap=10**6, nthreads=1) for g in ranks]
    d0, d1 = 0, 0
    for r in rs:
        d0 = (d0 + r["digest"][0]) & ((1 << 64) - 1)
        d1 ^= r["digest"][1]
    e, d = merge_selections([r["e"] for r in rs], [r["dets"].reshape(len(r["e"]), -1) for r in rs], k)
    return {"eps": np.array([r["eps"] for r in rs]), "s2": np.array([r["sum_e_over_d"] for r in rs]),
            "na": np.array([r["n_perturbers"] for r in rs]), "ncon": np.array([r["n_connections"] for r in rs]),
            "digest": (d0, d1), "sel_e": e, "sel_dets": d}


def test_coordinator_reissues_expired_and_ignores_duplicates():
    t = [0.0]
    co = Coordinator(rank_blocks(np.arange(10), 4), lease_s=5.0, clock=lambda: t[0])
    assert len(co.blocks) == 3
    b0, r0 = co.next_task("a")
    b1, r1 = co.next_task("b")
    assert list(r0) == [0, 1, 2, 3] and list(r1) == [4, 5, 6, 7]
    t[0] = 6.0  # helper a never answers: its lease runs out
    b2, _ = co.next_task("c")
    assert b2 == 2 and co.reissued == 2  # blocks 0 and 1 were handed out again
    b0b, _ = co.next_task("c")
    assert b0b == b0
    rec = []
    assert co.result(b0, lambda: rec.append(b0) or True)
    assert not co.result(b0, lambda: rec.append(b0) or True)  # a late answer for block 0
    assert co.duplicates == 1 and rec == [b0]
    co.forget_helper("b")  # b left: block 1 goes back to the queue at once
    assert co.next_task("d")[0] == b1
    assert co.result(b1, lambda: True) and co.result(b2, lambda: True)
    assert co.finished() and co.next_task("e") is None


def test_ledger_duplicates_and_round_trip(tmp_path):
    ham, dets, c, e0 = _case()
    led = RankLedger(len(dets), 10, 2)
    blocks = rank_blocks(np.arange(len(dets)), 16)
    for b in blocks[:2]:
        assert led.accept(b, _block_result(ham, dets, c, e0, b, 10))
    assert not led.accept(blocks[0], _block_result(ham, dets, c, e0, blocks[0], 10))
    with pytest.raises(ValueError):
        led.accept(np.array([0, 39]), _block_result(ham, dets, c, e0, [0, 39], 10))
    p = str(tmp_path / "ck.npz")
    led.save(p)
    back = RankLedger.load(p)
    for f in ("done", "eps", "s2", "na", "ncon", "sel_e", "sel_d"):
        assert np.array_equal(getattr(back, f), getattr(led, f)), f
    assert (back.d0, back.d1) == (led.d0, led.d1)
    assert list(back.missing()) == list(range(32, 40))


def _helper(hid, behaviour, tasks, results, k):
    ham, dets, c, e0 = _case()
    while True:
        task = tasks.get()
        if task is None:
            return
        b, ranks = task
        if behaviour == "crash":
            os._exit(3)  # takes a block and leaves without an answer
        out = _block_result(ham, dets, c, e0, ranks, k)
        results.put((hid, b, ranks, out))
        if behaviour == "twice":
            results.put((hid, b, ranks, out))


def test_helpers_that_fail_leave_the_result_unchanged(tmp_path):
    """Three helper processes: one exits after taking a block, one answers
    every block twice.  The lost block is handed out again, the second
    answers are ignored, and the per-rank results equal the oracle's sweep."""
    ham, dets, c, e0 = _case()
    k = 12
    ref = ham.sweep(dets, c, e0, k=k)
    ctx = mp.get_context("spawn")
    results = ctx.Queue()
    behaviours = ["crash", "twice", "ok"]
    tasks = [ctx.Queue() for _ in behaviours]
    procs = [ctx.Process(target=_helper, args=(i, bh, tasks[i], results, k)) for i, bh in enumerate(behaviours)]
    for p in procs:
        p.start()
    co = Coordinator(rank_blocks(np.arange(len(dets)), 5), lease_s=60.0)
    led = RankLedger(len(dets), k, 2)
    busy = {}
    gone = set()
    deadline = time.time() + 240
    try:
        while not co.finished():
            assert time.time() < deadline, "the run did not finish"
            for i, p in enumerate(procs):  # helpers that left are noticed on the host
                if i not in gone and not p.is_alive():
                    gone.add(i)
                    co.forget_helper(i)
                    busy.pop(i, None)
            for i in range(len(procs)):
                if i in gone or i in busy:
                    continue
                t = co.next_task(i)
                if t is None:
                    break
                busy[i] = t[0]
                tasks[i].put((t[0], t[1]))
            try:
                hid, b, ranks, out = results.get(timeout=0.5)
            except queue.Empty:
                continue
            co.result(b, lambda: led.accept(ranks, out))
            if busy.get(hid) == b:
                del busy[hid]
        # answers still on the way (the helper that answers twice) are
        # duplicates of complete blocks
        while True:
            try:
                hid, b, ranks, out = results.get(timeout=2.0)
            except queue.Empty:
                break
            assert not co.result(b, lambda: led.accept(ranks, out))
    finally:
        for i, p in enumerate(procs):
            if p.is_alive():
                tasks[i].put(None)
        for p in procs:
            p.join(timeout=30)
    assert gone == {0} and co.reissued >= 1 and co.duplicates >= 1
    assert led.done.all()
    assert np.array_equal(led.na, ref["na_by_rank"]) and np.array_equal(led.ncon, ref["ncon_by_rank"])
    assert np.max(np.abs(led.eps - ref["eps_by_rank"])) <= 1e-14
    assert (led.d0, led.d1) == tuple(int(x) for x in ref["digest"])
    assert abs(led.eps.sum() - ref["e_pt2"]) <= 1e-12
    assert np.array_equal(led.sel_d.reshape(ref["sel_dets"].shape), ref["sel_dets"])
    assert np.allclose(led.sel_e, ref["sel_e"], rtol=1e-13, atol=0)
