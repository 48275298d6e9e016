"""The CIPSI loop on the GPU (Sec. "The basic algorithm"): from a Psi0 with
its coefficients and E0, each step sweeps Psi0 (E_PT2 and the selection of
the k = N_det external determinants of largest |e_alpha|), appends them,
and takes the lowest eigenpair of H over the doubled space by Davidson,
starting from the previous coefficients.  Both the sweep and Davidson run
in the CUDA library; this module only passes arrays between them.
"""
from __future__ import annotations

import numpy as np


def grow(pt2, dets, coefs, e0, doublings, tol=1e-10, log=None):
    """Doubles Psi0 `doublings` times.  dets, coefs: host arrays.  Returns
    (dets, coefs, e0, info) with one record per space: N_det, E0, the
    Davidson residual and, for every space but the last, E_PT2."""
    dets = np.ascontiguousarray(dets, dtype=np.uint64)
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    info = [{"ndet": len(dets), "e0": float(e0)}]
    for it in range(doublings):
        out = pt2.eval(dets, coefs, e0, len(dets))
        if out["n_selected"] != len(dets):
            raise RuntimeError("not enough external determinants to double the space")
        info[-1].update(e_pt2=out["e_pt2"], n_perturbers=out["n_perturbers"])
        dets = np.ascontiguousarray(np.concatenate([dets, out["sel_dets"]]), dtype=np.uint64)
        guess = np.concatenate([coefs, np.zeros(len(out["sel_dets"]))])
        e0, coefs, dinfo = pt2.davidson(dets, guess=guess, tol=tol)
        info.append({"ndet": len(dets), "e0": e0, "residual": dinfo["residual"],
                     "davidson_ms": dinfo["build_ms"] + dinfo["solve_ms"]})
        if log:
            log(f"  doubling {it + 1}: ndet={len(dets)} e0={e0:.12f}")
    return dets, coefs, e0, info


def grow_from_seed(pt2, seed_dets, doublings, tol=1e-10, log=None):
    """The growth from a seed space: the lowest eigenpair of H over the seed
    (Davidson), then ``doublings`` doublings as in ``grow``.  seed_dets: host
    array.  Returns (dets, coefs, e0, info); info starts with the seed's
    record."""
    seed_dets = np.ascontiguousarray(seed_dets, dtype=np.uint64)
    e0, coefs, dinfo = pt2.davidson(seed_dets, tol=tol)
    dets, coefs, e0, info = grow(pt2, seed_dets, coefs, e0, doublings, tol=tol, log=log)
    info[0].update(residual=dinfo["residual"], davidson_ms=dinfo["build_ms"] + dinfo["solve_ms"])
    return dets, coefs, e0, info
