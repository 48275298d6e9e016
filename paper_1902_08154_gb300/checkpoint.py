"""Checkpoint and resume of a sweep by generator rank, and the bookkeeping of
work handed to helpers that may fail.

The generators are independent under the canonical rule (Eqs. calpha and
edetstoch: E_PT2 = sum_I eps_I, each eps_I set by the whole Psi0 but not by
which other eps are computed), which is what the paper's distributed PT2
relies on when helper jobs join or leave during a run (Sec. "Parallelism",
and Sec. "Stochastic selection" for reusing stored eps_I).  Here:

* ``RankLedger`` keeps, by generator rank, eps_I, sum A^2/D^2, |A_I| and the
  connection count of every generator swept so far, the per-block digests and
  minimum denominators, and the best k perturbers seen; it is written to disk
  atomically (temporary file, then rename) after every block, so a run that
  stops can resume with the ranks still missing.
* ``Coordinator`` hands out blocks of ranks with a lease; a block whose
  helper stops answering (lease expired) is handed out again, and a result
  for a block that is already complete is ignored.
* ``resumable_sweep`` sweeps the missing blocks through the library
  (``qp_pt2_eval_gens``), checkpointing after each, and assembles the whole
  sweep: per-rank values reduced by the library exactly as one
  ``qp_pt2_eval`` reduces them (``qp_pt2_reduce_ranks``), so the resumed
  E_PT2 has the same bits as an uninterrupted sweep.
"""
from __future__ import annotations

import os
import time

import numpy as np

MASK64 = (1 << 64) - 1


class RankLedger:
    def __init__(self, ndet, k, nw):
        self.ndet, self.k, self.nw = int(ndet), int(k), int(nw)
        self.done = np.zeros(self.ndet, dtype=bool)
        self.eps = np.zeros(self.ndet)
        self.s2 = np.zeros(self.ndet)
        self.na = np.zeros(self.ndet, dtype=np.int64)
        self.ncon = np.zeros(self.ndet, dtype=np.int64)
        self.d0, self.d1 = 0, 0
        self.n_tiny = 0
        self.min_den = float("inf")
        self.sel_e = np.zeros(0)
        self.sel_d = np.zeros((0, self.nw), dtype=np.uint64)

    def missing(self):
        return np.nonzero(~self.done)[0].astype(np.int32)

    def accept(self, ranks, out):
        """Record one block's results (a dict as from ``PT2.eval_generators``
        with per-rank eps, s2, na, ncon, the block's digest, n_tiny,
        min_abs_den and selection).  A block whose ranks are already recorded
        is a duplicate (a helper's late answer, a re-issued block): it is
        ignored and False returned."""
        ranks = np.asarray(ranks, dtype=np.int64)
        if self.done[ranks].any():
            if not self.done[ranks].all():
                raise ValueError("a block overlaps recorded ranks only in part")
            return False
        self.eps[ranks] = out["eps"]
        self.s2[ranks] = out["s2"]
        self.na[ranks] = out["na"]
        self.ncon[ranks] = out["ncon"]
        self.d0 = (self.d0 + int(out["digest"][0])) & MASK64
        self.d1 ^= int(out["digest"][1])
        self.n_tiny += int(out.get("n_tiny", 0))
        self.min_den = min(self.min_den, float(out.get("min_abs_den", float("inf"))))
        if self.k > 0 and len(out["sel_e"]):
            from .shard import merge_selections

            e = np.asarray(out["sel_e"].cpu() if hasattr(out["sel_e"], "cpu") else out["sel_e"], dtype=np.float64)
            d = out["sel_dets"]
            d = np.asarray(d.cpu() if hasattr(d, "cpu") else d).view(np.uint64).reshape(len(e), self.nw)
            self.sel_e, self.sel_d = merge_selections([self.sel_e, e], [self.sel_d, d], self.k)
        self.done[ranks] = True
        return True

    def save(self, path):
        tmp = f"{path}.tmp{os.getpid()}"
        with open(tmp, "wb") as f:
            np.savez(f, ndet=self.ndet, k=self.k, nw=self.nw, done=self.done, eps=self.eps, s2=self.s2, na=self.na,
                     ncon=self.ncon, d=np.array([self.d0, self.d1], dtype=np.uint64), n_tiny=self.n_tiny,
                     min_den=self.min_den, sel_e=self.sel_e, sel_d=self.sel_d)
        os.replace(tmp, path)

    @classmethod
    def load(cls, path):
        z = np.load(path)
        led = cls(int(z["ndet"]), int(z["k"]), int(z["nw"]))
        led.done, led.eps, led.s2 = z["done"].copy(), z["eps"].copy(), z["s2"].copy()
        led.na, led.ncon = z["na"].copy(), z["ncon"].copy()
        led.d0, led.d1 = int(z["d"][0]), int(z["d"][1])
        led.n_tiny, led.min_den = int(z["n_tiny"]), float(z["min_den"])
        led.sel_e, led.sel_d = z["sel_e"].copy(), z["sel_d"].copy()
        return led


class Coordinator:
    """Blocks of generator ranks handed to helpers with a lease of
    ``lease_s`` seconds.  ``clock`` is injectable for tests."""

    def __init__(self, blocks, lease_s=60.0, clock=time.monotonic):
        self.blocks = [np.asarray(b, dtype=np.int32) for b in blocks]
        self.lease_s, self.clock = lease_s, clock
        self.pending = list(range(len(self.blocks)))
        self.leased = {}  # block -> (helper, deadline)
        self.complete = set()
        self.reissued = 0
        self.duplicates = 0

    def next_task(self, helper):
        """(block id, ranks) for helper, or None when nothing is pending."""
        self.expire()
        if not self.pending:
            return None
        b = self.pending.pop(0)
        self.leased[b] = (helper, self.clock() + self.lease_s)
        return b, self.blocks[b]

    def expire(self):
        """Hand out again every block whose lease has passed."""
        now = self.clock()
        for b, (_, deadline) in list(self.leased.items()):
            if now > deadline:
                del self.leased[b]
                self.pending.append(b)
                self.reissued += 1

    def forget_helper(self, helper):
        """A helper known to have left: its blocks are handed out again now."""
        for b, (h, _) in list(self.leased.items()):
            if h == helper:
                del self.leased[b]
                self.pending.append(b)
                self.reissued += 1

    def result(self, b, accept):
        """A helper's result for block b: accept() records it unless the block
        is already complete (then the result is ignored).  Returns whether it
        was recorded."""
        if b in self.complete:
            self.duplicates += 1
            return False
        if not accept():
            self.duplicates += 1
            return False
        self.complete.add(b)
        self.leased.pop(b, None)
        if b in self.pending:
            self.pending.remove(b)
        return True

    def finished(self):
        return len(self.complete) == len(self.blocks)


def rank_blocks(ranks, block):
    ranks = np.asarray(ranks, dtype=np.int32)
    return [ranks[i:i + block] for i in range(0, len(ranks), block)]


def resumable_sweep(pt2, dets, coefs, e0, k, path, block=1000, stop_after=None):
    """The whole sweep of Psi0 by blocks of generator ranks, checkpointed to
    ``path`` after every block and resumed from it if it exists.  Returns the
    sweep's result dict (as ``PT2.eval``: totals, Z, E_rPT2, digest,
    selection, per-rank arrays).  ``stop_after`` (blocks) ends the call early,
    leaving the checkpoint, as a run that is stopped does."""
    nw = 2 * pt2.nint
    led = RankLedger.load(path) if os.path.exists(path) else RankLedger(len(dets), k, nw)
    if led.ndet != len(dets) or led.k != k or led.nw != nw:
        raise ValueError("the checkpoint belongs to another sweep")
    swept = 0
    for ranks in rank_blocks(led.missing(), block):
        if stop_after is not None and swept >= stop_after:
            return None
        out = pt2.eval_generators(dets, coefs, e0, ranks, k=k)
        led.accept(ranks, out)
        led.save(path)
        swept += 1
    tot = pt2.reduce_ranks(led.eps, led.s2, led.na, led.ncon, e0)
    tot.update(digest=(led.d0, led.d1), n_tiny=led.n_tiny, min_abs_den=led.min_den,
               n_selected=len(led.sel_e), sel_e=led.sel_e, sel_dets=led.sel_d.reshape(len(led.sel_e), 2, -1),
               eps_by_rank=led.eps, na_by_rank=led.na, ncon_by_rank=led.ncon)
    return tot
