"""Write the stored workloads and their expected sweep results.

Calls only the CPU oracle (``oracle/``) and the seeded input generator; no
value here comes from the CUDA path.  Usage:

    python tests/golden/make_inputs.py cfg1 [cfg2 ...]

Workloads (synthetic stand-ins for the paper's molecules, whose integrals are
not available; shapes follow the paper's CAS-sized active spaces):

  cfg1: norb 16, 4+4 electrons, Cholesky rank 32, seed 0.  Psi0 = HF + the 49
        lowest-diagonal single/double substitutions of HF; c and E0 from dense
        diagonalisation of the 50x50 block.  Expected results with k = 100.
  cfg4: norb 48, 8+8 electrons, Cholesky rank 72, seed 3.  Psi0 of 2*10^4
        determinants grown from 2500 by three CIPSI doublings; expected sweep
        results with k = 2*10^4 and the oracle's full gradient
        (dE/dh, dE/d(packed eri), dE/dE0) in ``cfg4_gradient.npz``.
  cfg2: norb 64, 10+10 electrons, Cholesky rank 96, seed 1.  Psi0 of 10^4
        determinants grown from a 1250-determinant seed space by three CIPSI
        doublings (top |e_alpha| selection), coefficients from Davidson to a
        residual below 1e-10.  Expected results with k = 2 * 10^4.
  cfg3r: the first 10 determinants of the 128-orbital workload
        (``synthetic.cfg3_instance``; 14+14 electrons, Cholesky rank 192),
        expected sweep with k = 20 (totals and per-generator arrays).
  cfg3seed: the seed space of the CIPSI growth of the 128-orbital workload
        (norb 128, 14+14 electrons, Cholesky rank 192, seed 2): HF plus the
        12,499 single and double substitutions of HF with the lowest diagonal
        energy, ties by key.  Only the determinants are stored; the three
        doublings to 10^5 determinants (Davidson, then the top-|e_alpha|
        selection, Sec. "The basic algorithm") are run from them by the
        consumer.

  cfg5seed: the seed spaces of the 64 batched instances
        (``synthetic.batch_specs``: norb in {24, 32, 48, 64, 96}, 6..12
        electrons per spin, N_det log-uniform in [1e3, 5e4], Cholesky rank
        1.5 norb, seeds 1000 + i): per instance HF plus the N_det / 8 - 1
        single and double substitutions of HF with the lowest diagonal
        energy, ties by key.  As for cfg3seed, only the determinants are
        stored and the consumer runs the three doublings.

Files: ``<cfg>_psi0.npz`` (dets, coefs, e0 and metadata) and
``<cfg>_expected.npz`` (totals, per-generator arrays by rank, selection).
"""
from __future__ import annotations

import json
import os
import sys
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
from oracle import psi0  # noqa: E402
from paper_1902_08154_gb300 import synthetic as S  # noqa: E402

CONFIGS = {
    "cfg1": dict(norb=16, nalpha=4, nbeta=4, rank=32, seed=0, ndet=50, k=100, grow=False),
    "cfg2": dict(norb=64, nalpha=10, nbeta=10, rank=96, seed=1, ndet=10000, k=20000, grow=True),
    "cfg4": dict(norb=48, nalpha=8, nbeta=8, rank=72, seed=3, ndet=20000, k=40000, grow=True, gradient=True),
    # the head (10 determinants) of the 128-orbital workload's Psi0
    "cfg3r": dict(norb=128, nalpha=14, nbeta=14, rank=192, seed=2, ndet=10, k=20, grow=False, instance="cfg3"),
    # the seed space (N_det / 8) of the 128-orbital workload's CIPSI growth
    "cfg3seed": dict(norb=128, nalpha=14, nbeta=14, rank=192, seed=2, ndet=12500, final_ndet=100000,
                     doublings=3, grow=False, instance="cfg3seed"),
    # the seed spaces (N_det / 8 each) of the 64 batched instances
    "cfg5seed": dict(n=64, seed0=1000, doublings=3, grow=False, instance="cfg5seed"),
}


def make_cfg5seed(name, cfg):
    t0 = time.time()
    specs = S.batch_specs(cfg["n"], cfg["seed0"])
    out = {}
    for i, sp in enumerate(specs):
        h, eri = S.hamiltonian_fast(sp["norb"], sp["rank"], sp["seed"])
        ham = oracle.Hamiltonian(sp["norb"], sp["nalpha"], sp["nbeta"], h, eri)
        hf = S.hf_det(sp["norb"], sp["nalpha"], sp["nbeta"])
        out[f"dets_{i}"] = psi0.seed_space(ham, hf, sp["ndet"] // 2 ** cfg["doublings"])
    log(f"{name}: {len(specs)} seed spaces, {sum(len(v) for v in out.values())} dets in {time.time() - t0:.1f}s")
    np.savez_compressed(os.path.join(HERE, f"{name}.npz"), meta=json.dumps(dict(cfg, specs=specs)), **out)


def make_cfg3r(name, cfg):
    """Expected sweep of the head of the 128-orbital workload.  Its integrals
    come from a matrix product whose last bits may depend on the BLAS, so
    only the totals are stored; a consumer regenerates the inputs and
    compares energies at the stated tolerance."""
    t0 = time.time()
    h, eri, dets, c, e0 = S.cfg3_instance(cfg["ndet"])
    ham = oracle.Hamiltonian(cfg["norb"], cfg["nalpha"], cfg["nbeta"], h, eri)
    out = ham.sweep(dets, c, e0, k=cfg["k"])
    log(f"{name}: sweep E_PT2={out['e_pt2']:.12f} |A|={out['n_perturbers']} in {time.time() - t0:.1f}s")
    summary = {k: v for k, v in out.items() if not isinstance(v, np.ndarray)}
    summary["digest"] = [str(x) for x in summary["digest"]]
    np.savez_compressed(os.path.join(HERE, f"{name}_expected.npz"), sel_e=out["sel_e"],
                        eps_by_rank=out["eps_by_rank"], na_by_rank=out["na_by_rank"],
                        summary=json.dumps(summary), meta=json.dumps(cfg))


def make_cfg3seed(name, cfg):
    t0 = time.time()
    h, eri = S.hamiltonian_fast(cfg["norb"], cfg["rank"], cfg["seed"])
    ham = oracle.Hamiltonian(cfg["norb"], cfg["nalpha"], cfg["nbeta"], h, eri)
    hf = S.hf_det(cfg["norb"], cfg["nalpha"], cfg["nbeta"])
    dets = psi0.seed_space(ham, hf, cfg["ndet"])
    log(f"{name}: seed space of {len(dets)} dets in {time.time() - t0:.1f}s")
    np.savez_compressed(os.path.join(HERE, f"{name}.npz"), dets=dets, meta=json.dumps(cfg))


def log(msg):
    print(msg, flush=True)


def make(name, mem_budget=12 << 30):
    cfg = CONFIGS[name]
    if cfg.get("instance") == "cfg3":
        return make_cfg3r(name, cfg)
    if cfg.get("instance") == "cfg3seed":
        return make_cfg3seed(name, cfg)
    if cfg.get("instance") == "cfg5seed":
        return make_cfg5seed(name, cfg)
    t0 = time.time()
    h, eri = S.hamiltonian(cfg["norb"], cfg["rank"], cfg["seed"])
    ham = oracle.Hamiltonian(cfg["norb"], cfg["nalpha"], cfg["nbeta"], h, eri)
    hf = S.hf_det(cfg["norb"], cfg["nalpha"], cfg["nbeta"])
    if cfg["grow"]:
        dets, c, e0, info = psi0.cipsi_grow(ham, hf, cfg["ndet"], doublings=3, log=log)
    else:
        dets = psi0.seed_space(ham, hf, cfg["ndet"])
        e0, c, res = psi0.ground_state(ham, dets)
        info = [{"ndet": len(dets), "e0": e0, "residual": res}]
    log(f"{name}: psi0 ready ({len(dets)} dets, e0={e0:.12f}) in {time.time() - t0:.1f}s")
    meta = dict(cfg, digest=S.hamiltonian_digest(h, eri), growth=info)
    np.savez_compressed(os.path.join(HERE, f"{name}_psi0.npz"), dets=dets, coefs=c, e0=np.float64(e0),
                        meta=json.dumps(meta))
    t1 = time.time()
    out = ham.sweep(dets, c, e0, k=cfg["k"], mem_budget=mem_budget)
    log(f"{name}: sweep E_PT2={out['e_pt2']:.12f} |A|={out['n_perturbers']} "
        f"connections={out['n_connections']} in {time.time() - t1:.1f}s")
    summary = {k: v for k, v in out.items() if not isinstance(v, np.ndarray)}
    summary["digest"] = [str(x) for x in summary["digest"]]
    np.savez_compressed(os.path.join(HERE, f"{name}_expected.npz"), sel_dets=out["sel_dets"],
                        sel_e=out["sel_e"], sel_num=out["sel_num"], eps_by_rank=out["eps_by_rank"],
                        na_by_rank=out["na_by_rank"], ncon_by_rank=out["ncon_by_rank"],
                        rank_of=out["rank_of"], summary=json.dumps(summary))
    if cfg.get("gradient"):
        t2 = time.time()
        g = ham.gradient(dets, c, e0, mem_budget=mem_budget)
        log(f"{name}: gradient in {time.time() - t2:.1f}s (E_PT2 {g['e_pt2']:.12f})")
        np.savez_compressed(os.path.join(HERE, f"{name}_gradient.npz"), dh=g["dh"], deri=g["deri"],
                            de0=np.float64(g["de0"]), e_pt2=np.float64(g["e_pt2"]))


if __name__ == "__main__":
    for name in sys.argv[1:] or ["cfg1"]:
        make(name)
