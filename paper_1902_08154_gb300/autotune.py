"""Autotuner for batched sweeps.

For a batch of instances it times launch shapes of the fused batch (one
persistent launch per wave whose queue spans all instances' work items) and
keeps the fastest: the work items a CTA takes per draw from the shared queue
(``work_chunk``), the row tiles of the opposite-spin batches (``tile``; 0
keeps each context's own choice) and the persistent CTAs per SM.  Results are
cached in a JSON file keyed by the batch's shape (orbitals, electrons,
determinants, k, precision of every instance), so a batch of the same shape
is tuned once per machine.
"""
from __future__ import annotations

import hashlib
import json
import os

CACHE = os.environ.get("QP_PT2_TUNE_CACHE",
                       os.path.join(os.path.expanduser("~"), ".cache", "qp_pt2", "autotune.json"))

CHUNKS = (1, 2, 4, 8)
TILES = (0, 2)


def signature(instances) -> str:
    rows = [(i["pt2"].norb, i["pt2"].n_alpha, i["pt2"].n_beta, len(i["dets"]), i["k"], i.get("precision", 0))
            for i in instances]
    return hashlib.sha256(json.dumps(["fused"] + rows).encode()).hexdigest()[:20]


def candidates(instances, nsm=None):
    """Launch shapes tried first: dicts of Batch keyword arguments, every
    (work_chunk, tile) pair with as many CTAs per SM as fit.  ``tune`` then
    tries the best pair with two CTAs per SM."""
    return [{"work_chunk": c, "tile": t, "blocks_per_sm": 0} for t in TILES for c in CHUNKS]


def _time(instances, shape, repeats, max_streams):
    from . import Batch

    b = Batch(instances, fused=True, max_streams=max_streams, **shape)
    b.run()
    t = min(b.run()[1] for _ in range(repeats))
    b.close()
    return t


def tune(instances, nsm, repeats=2, cache=CACHE, log=None, max_streams=16):
    """Return (shape, record): the fastest shape (Batch keyword arguments)
    and the timings of every shape tried.  Times the candidates unless the
    cache holds this batch's shape."""
    sig = signature(instances)
    table = {}
    if cache and os.path.exists(cache):
        try:
            table = json.load(open(cache))
        except (OSError, ValueError):
            table = {}
    if sig in table:
        rec = table[sig]
        return rec["shape"], rec
    tried = []
    best = None
    for shape in candidates(instances, nsm):
        t = _time(instances, shape, repeats, max_streams)
        tried.append(dict(shape, ms=t))
        if log:
            log(f"autotune work_chunk={shape['work_chunk']} tile={shape['tile']}: {t:.2f} ms")
        if best is None or t < best[0]:
            best = (t, shape)
    # the best pair with two CTAs per SM (fewer CTAs share each SM's L1)
    shape = dict(best[1], blocks_per_sm=2)
    t = _time(instances, shape, repeats, max_streams)
    tried.append(dict(shape, ms=t))
    if log:
        log(f"autotune work_chunk={shape['work_chunk']} tile={shape['tile']} blocks_per_sm=2: {t:.2f} ms")
    if t < best[0]:
        best = (t, shape)
    rec = {"shape": best[1], "ms": best[0], "tried": tried}
    if cache:
        os.makedirs(os.path.dirname(cache), exist_ok=True)
        table[sig] = rec
        tmp = cache + f".tmp{os.getpid()}"
        json.dump(table, open(tmp, "w"))
        os.replace(tmp, cache)
    return rec["shape"], rec
