"""Autotuner for batched sweeps.

For a batch of instances it times a small set of launch shapes of the one
CUDA graph -- the persistent CTAs given to each instance's sweep and the
number of concurrent streams the instances are spread over -- and keeps the
fastest.  Results are cached in a JSON file keyed by the batch's shape
(orbitals, electrons, determinants, k, precision of every instance), so a
batch of the same shape is tuned once per machine.
"""
from __future__ import annotations

import hashlib
import json
import os

CACHE = os.environ.get("QP_PT2_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "qp_pt2", "autotune.json"))


def signature(instances) -> str:
    rows = [(i["pt2"].norb, i["pt2"].n_alpha, i["pt2"].n_beta, len(i["dets"]), i["k"], i.get("precision", 0))
            for i in instances]
    return hashlib.sha256(json.dumps(rows).encode()).hexdigest()[:20]


def candidates(instances, nsm):
    """Launch shapes tried: (name, per-instance CTA counts, streams)."""
    work = []
    for i in instances:
        p = i["pt2"]
        nel = p.n_alpha + p.n_beta
        work.append(len(i["dets"]) * (nel + nel * (nel - 1) // 2))
    tot = float(sum(work)) or 1.0
    full = [3 * nsm] * len(instances)
    prop = [max(nsm // 4, min(3 * nsm, int(round(3 * nsm * len(instances) * w / tot / 4)))) for w in work]
    shapes = []
    for streams in (8, 16):
        shapes.append(("full", full, streams))
        shapes.append(("one_per_sm", [nsm] * len(instances), streams))
        shapes.append(("proportional", prop, streams))
    return shapes


def tune(instances, nsm, repeats=2, cache=CACHE, log=None):
    """Return (grid list, streams, record); times every candidate shape
    unless the cache holds this batch's shape."""
    from . import Batch

    sig = signature(instances)
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if sig in table:
        rec = table[sig]
        return rec["grid"], rec["streams"], rec
    best = None
    tried = []
    for name, grid, streams in candidates(instances, nsm):
        b = Batch(instances, grid=grid, max_streams=streams)
        b.run()
        t = min(b.run()[1] for _ in range(repeats))
        b.close()
        tried.append({"name": name, "streams": streams, "ms": t})
        if log:
            log(f"autotune {name:13s} streams={streams:2d}: {t:.2f} ms")
        if best is None or t < best[0]:
            best = (t, name, grid, streams)
    rec = {"grid": best[2], "streams": best[3], "policy": best[1], "ms": best[0], "tried": tried}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        table[sig] = rec
        tmp = cache + f".tmp{os.getpid()}"
        json.dump(table, open(tmp, "w"))
        os.replace(tmp, cache)
    return rec["grid"], rec["streams"], rec
