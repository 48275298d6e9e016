"""Zeroth-order wave functions for the test and benchmark workloads.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Psi0 is produced the way the paper's CIPSI loop grows it (Sec. "The basic
algorithm"): diagonalise H over the internal space (Davidson, Algorithm
davidson, Sec. "Davidson diagonalization"), compute e_alpha for every external
determinant, add the determinants with the largest |e_alpha| so that the space
doubles, and repeat.  Every matrix element and every e_alpha here comes from
the oracle library; nothing comes from the CUDA path.

Readings (the paper leaves these open):
  * the synthetic "HF" determinant fills the lowest orbitals of each spin;
  * the seed space of size n is HF plus the n-1 single and double
    substitutions of HF with the lowest diagonal energy <alpha|H|alpha>
    (ties broken by determinant key), and three doublings give the final
    size (n_final / 8 -> n_final);
  * the sign of the eigenvector is fixed by c_HF > 0 and E0 is the Rayleigh
    quotient of the converged vector.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp

from . import Hamiltonian


def hamiltonian_matrix(ham: Hamiltonian, dets, nthreads=0):
    r, c, v = ham.hamiltonian_coo(dets, nthreads)
    n = len(dets)
    off = r != c
    rows = np.concatenate([r, c[off]])
    cols = np.concatenate([c, r[off]])
    vals = np.concatenate([v, v[off]])
    return sp.csr_matrix((vals, (rows, cols)), shape=(n, n))


def davidson(Hm, guess=None, tol=1e-10, max_iter=500, max_subspace=48):
    """Lowest eigenpair of the symmetric sparse matrix Hm by Davidson's
    method with the diagonal preconditioner (Algorithm davidson, one state).
    Stops when the residual norm ||H u - E u|| drops below ``tol``."""
    n = Hm.shape[0]
    diag = Hm.diagonal()
    if n <= 64:
        w, v = np.linalg.eigh(Hm.toarray())
        return float(w[0]), v[:, 0], 0.0
    u = np.zeros(n) if guess is None else np.array(guess, dtype=np.float64)
    if guess is None or not np.any(u):
        u[np.argmin(diag)] = 1.0
    U = [u / np.linalg.norm(u)]
    W = [Hm @ U[0]]
    res = np.inf
    E = 0.0
    x = U[0]
    for _ in range(max_iter):
        Um = np.array(U).T
        Wm = np.array(W).T
        hsub = Um.T @ Wm
        hsub = 0.5 * (hsub + hsub.T)
        w, y = np.linalg.eigh(hsub)
        E = float(w[0])
        x = Um @ y[:, 0]
        hx = Wm @ y[:, 0]
        r = hx - E * x
        res = float(np.linalg.norm(r))
        if res < tol:
            break
        den = E - diag
        den = np.where(np.abs(den) < 1e-8, np.copysign(1e-8, den), den)
        t = r / den
        if len(U) >= max_subspace:
            U, W = [x / np.linalg.norm(x)], [hx / np.linalg.norm(x)]
        for _gs in range(2):
            for b in U:
                t = t - (b @ t) * b
        nt = np.linalg.norm(t)
        if nt < 1e-14:
            break
        t = t / nt
        U.append(t)
        W.append(Hm @ t)
    x = x / np.linalg.norm(x)
    return E, x, res


def ground_state(ham: Hamiltonian, dets, guess=None, tol=1e-10, nthreads=0):
    """(E0, c, residual) with c_0 > 0 and E0 the Rayleigh quotient."""
    Hm = hamiltonian_matrix(ham, dets, nthreads)
    if guess is not None and len(guess) < len(dets):
        guess = np.concatenate([guess, np.zeros(len(dets) - len(guess))])
    _, c, _ = davidson(Hm, guess, tol=tol)
    if c[0] < 0:
        c = -c
    c = c / np.linalg.norm(c)
    hc = Hm @ c
    e0 = float(c @ hc)
    res = float(np.linalg.norm(hc - e0 * c))
    return e0, c, res


def seed_space(ham: Hamiltonian, hf, n):
    """HF plus the n-1 lowest-diagonal single/double substitutions of HF."""
    subs = ham.substitutions(hf)
    diag = np.array([ham.diag(a) for a in subs])
    nw = subs.shape[1] * subs.shape[2]
    keys = subs.reshape(len(subs), nw)
    # lexsort: last key is primary -> diag, then key words in order
    order = np.lexsort(tuple(keys[:, w] for w in range(nw - 1, -1, -1)) + (diag,))
    pick = subs[order[: n - 1]]
    return np.concatenate([hf[None], pick]).astype(np.uint64)


def cipsi_grow(ham: Hamiltonian, hf, n_final, doublings=3, nthreads=0, log=None):
    """Seed space of n_final / 2**doublings determinants, then CIPSI
    doublings with top-|e_alpha| selection.  Returns (dets, coefs, e0, info)."""
    n0 = n_final // (2 ** doublings)
    dets = seed_space(ham, hf, n0)
    e0, c, res = ground_state(ham, dets, nthreads=nthreads)
    info = [{"ndet": len(dets), "e0": e0, "residual": res}]
    for it in range(doublings):
        out = ham.sweep(dets, c, e0, k=len(dets), nthreads=nthreads, per_generator=False)
        if out["n_selected"] != len(dets):
            raise RuntimeError("not enough external determinants to double the space")
        info[-1].update(e_pt2=out["e_pt2"], n_perturbers=out["n_perturbers"])
        dets = np.concatenate([dets, out["sel_dets"]]).astype(np.uint64)
        e0, c, res = ground_state(ham, dets, guess=c, nthreads=nthreads)
        info.append({"ndet": len(dets), "e0": e0, "residual": res})
        if log:
            log(f"  doubling {it + 1}: ndet={len(dets)} e0={e0:.12f} residual={res:.2e}")
    return dets, c, e0, info
