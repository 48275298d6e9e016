"""Merge of generator-sharded sweeps (one process per GPU).

Each process sweeps the generators of rank r with r % N == its index (the
generators are independent under the canonical rule of Eqs. calpha and
edetstoch, which is what the paper's distributed PT2 exploits, Sec.
"Parallelism").  The partial results combine exactly:

* E_PT2, sum A^2/D^2, |A| and the connection count add, the digest words
  add modulo 2^64 and xor, and Z and E_rPT2 follow from the merged sums: the
  library's ``qp_pt2_merge_results`` does this arithmetic;
* the selection is the k best of the union of the shards' selections, in the
  library's order (|e| descending, determinant key ascending);
* a multi-state sweep's per-state E_PT2 and sum A^2/D^2 add state by state,
  and its selection (by the multi-state criterion) merges as above.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1


def merge_totals(parts, e0=0.0):
    """parts: list of result dicts (as returned by ``PT2.eval``), in shard
    order; e0: the E0 of the sweep (for Z and E_rPT2)."""
    from . import merge_results

    out = merge_results(parts, e0)
    if parts and all("e_pt2_states" in p for p in parts):
        out["e_pt2_states"] = np.sum([np.asarray(p["e_pt2_states"], dtype=np.float64) for p in parts], axis=0)
        out["sum_e_over_d_states"] = np.sum([np.asarray(p["sum_e_over_d_states"], dtype=np.float64)
                                             for p in parts], axis=0)
    return out


def merge_selections(e_lists, det_lists, k):
    """k best of the union of per-shard selections.

    e_lists: sequence of float64 arrays; det_lists: matching uint64 arrays of
    shape (n, 2*nint) (or (n, 2, nint)).  Returns (e, dets)."""
    es = [np.asarray(e, dtype=np.float64) for e in e_lists if len(e)]
    ds = [np.asarray(d).view(np.uint64).reshape(len(d), -1) for d, e in zip(det_lists, e_lists) if len(e)]
    if not es:
        return np.zeros(0), np.zeros((0, 0), dtype=np.uint64)
    e = np.concatenate(es)
    d = np.concatenate(ds)
    nw = d.shape[1]
    # np.lexsort: the last key is the primary one
    order = np.lexsort(tuple(d[:, w] for w in range(nw - 1, -1, -1)) + (-np.abs(e),))
    order = order[:k]
    return e[order], d[order]


def distributed_merge(dist, res, sel_e, sel_dets, k, device, e0=0.0):
    """Exchange step of a sharded sweep: all-gather every rank's partial
    totals and selection, then merge them identically on every rank.

    res: this rank's result dict (with ``e_pt2_states`` and
    ``sum_e_over_d_states`` for a multi-state sweep, the same number of
    states on every rank); sel_e: tensor [n]; sel_dets: tensor [n, 2, nint]
    (int64 view of the uint64 words).  Returns (totals, e, dets)."""
    import torch

    ws = dist.get_world_size()
    d0 = int(res["digest"][0])
    d1 = int(res["digest"][1])
    as_i64 = lambda u: u - (1 << 64) if u >= (1 << 63) else u  # noqa: E731
    ints = torch.tensor([int(res["n_perturbers"]), int(res["n_connections"]), int(res.get("n_tiny", 0)),
                         as_i64(d0), as_i64(d1), int(sel_e.numel())], dtype=torch.int64, device=device)
    st_e = [float(x) for x in res.get("e_pt2_states", [])]
    st_s = [float(x) for x in res.get("sum_e_over_d_states", [])]
    nst = len(st_e)
    flts = torch.tensor([res["e_pt2"], res["sum_e_over_d"], res.get("min_abs_den", float("inf"))] + st_e + st_s,
                        dtype=torch.float64, device=device)
    gi = [torch.zeros_like(ints) for _ in range(ws)]
    gf = [torch.zeros_like(flts) for _ in range(ws)]
    dist.all_gather(gi, ints)
    dist.all_gather(gf, flts)
    parts = []
    for a, b in zip(gi, gf):
        a, b = a.cpu().tolist(), b.cpu().tolist()
        part = {"n_perturbers": a[0], "n_connections": a[1], "n_tiny": a[2],
                "digest": (a[3] & MASK64, a[4] & MASK64), "e_pt2": b[0], "sum_e_over_d": b[1],
                "min_abs_den": b[2], "n_sel": a[5]}
        if nst:
            part["e_pt2_states"] = b[3:3 + nst]
            part["sum_e_over_d_states"] = b[3 + nst:3 + 2 * nst]
        parts.append(part)
    m = max(p["n_sel"] for p in parts)
    nw = sel_dets.shape[1] * sel_dets.shape[2] if sel_dets.dim() == 3 else sel_dets.shape[1]
    pe = torch.zeros(max(m, 1), dtype=torch.float64, device=device)
    pd = torch.zeros((max(m, 1), nw), dtype=torch.int64, device=device)
    n = sel_e.numel()
    if n:
        pe[:n] = sel_e
        pd[:n] = sel_dets.reshape(n, nw)
    ge = [torch.zeros_like(pe) for _ in range(ws)]
    gd = [torch.zeros_like(pd) for _ in range(ws)]
    dist.all_gather(ge, pe)
    dist.all_gather(gd, pd)
    e_all = [g[: p["n_sel"]].cpu().numpy() for g, p in zip(ge, parts)]
    d_all = [d[: p["n_sel"]].cpu().numpy().view(np.uint64) for d, p in zip(gd, parts)]
    totals = merge_totals(parts, e0)
    e, d = merge_selections(e_all, d_all, k)
    return totals, e, d
