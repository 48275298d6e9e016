#!/usr/bin/env python
"""Throughput of the GB300 EN-PT2 + CIPSI selection sweep.

One step = one complete sweep (validation, generator order, coarse and fine
filters, Slater-Condon accumulation, e_alpha, E_PT2 reduction, top-k
selection) over the stored Psi0 of the mid-size workload: 64 orbitals,
10 alpha + 10 beta electrons, 10^4 determinants grown by three CIPSI
doublings, k = 2 * 10^4 selected determinants, FP64.

Prints ONE JSON line.  ``value`` is perturbers/s with inputs resident in HBM
(CUDA-event time of the C-ABI call, L2 flushed between steps); ``e2e`` is the
same metric through the C-ABI call with pinned host buffers.  With N > 1
ranks (torchrun) each rank sweeps its share of the generators
(rank r mod N) and the partial results are merged with one all-reduce and one
all-gather inside the timed region.

``--impl reference`` times the CPU oracle instead (the reference arm): each
step is a bounded sample of the same workload (a few generators of the
canonical per-generator definition), on all host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

WORKLOAD = "cfg2"
METRIC = "EN-PT2 perturbers/s and generators/s on 1 GB300 vs plain FP64 GPU sweep"
UNIT = "perturbers/s"
L2_FLUSH_BYTES = 256 << 20

# The sweep is gather-and-bit work with FP64 arithmetic; on this GPU the FP64
# pipe is the scarce unit.  Algorithmic FP64 work per unit (an FMA counts as
# one operation), as the method defines it: per connection (J, alpha) the
# one FMA of A_alpha += c_J <J|H|alpha>; per perturber the incremental
# diagonal H_aa (about 20 operations: the Fock-diagonal and two-index terms
# of the particles and holes), one division and two FMAs (e = A^2/D and the
# sum of A^2/D^2).  The kernels form H_aa from per-batch row sums in 3 adds
# and 1/D by a Newton reciprocal; the smallest form the kernels execute,
# 9 operations per perturber, is reported beside it.
FP64_OPS_PER_CONNECTION = 1
FP64_OPS_PER_PERTURBER = 23
FP64_OPS_PER_PERTURBER_MIN = 9
# Integer work per unit: about 15 XOR/POPC/add operations per connection
# (excitation degree and phase) per 64-bit word of a spin string, and
# 2 x 2 x nint XOR+POPC per pair test of the coarse filter (N_det per
# generator).
INT_OPS_PER_CONNECTION_PER_WORD = 15
# DRAM bytes (read + write) of the sweep kernels (prep and batch, all four
# waves) over one sweep of the bench workload, from one ncu capture of the
# current kernels (dram__bytes_read.sum + dram__bytes_write.sum; None when
# the kernels have changed since the capture).
TRAFFIC_BYTES_PER_SWEEP = 18.099e9


def load_workload(name=WORKLOAD):
    from paper_1902_08154_gb300 import synthetic as S

    P = np.load(os.path.join(ROOT, "tests", "golden", f"{name}_psi0.npz"))
    meta = json.loads(str(P["meta"]))
    h, eri = S.hamiltonian(meta["norb"], meta["rank"], meta["seed"])
    return meta, h, eri, np.ascontiguousarray(P["dets"]), np.ascontiguousarray(P["coefs"]), float(P["e0"])


def workload_config(meta, n):
    return {
        "workload": f"{WORKLOAD}: norb={meta['norb']}, {meta['nalpha']}a+{meta['nbeta']}b electrons, "
                    f"ndet={meta['ndet']} (3 CIPSI doublings), k={meta['k']}, Cholesky rank {meta['rank']}, "
                    f"seed {meta['seed']}",
        "ndet": meta["ndet"],
        "k_select": meta["k"],
        "norb": meta["norb"],
        "precision": "fp64",
        "l2": "flushed between timed steps (256 MiB device write)",
        "parallelism": f"generator shards x{n}" if n > 1 else "single GPU",
    }


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.p.terminate()
        self.p.wait()
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r.strip()]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            r = [x.strip() for x in r]
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
            except (ValueError, IndexError):
                continue
            for nm, v in zip(names, r[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def cpu_baseline(meta, h, eri, dets, coefs, e0, budget_s=15.0, stride=97):
    """The oracle's per-generator definition on a bounded sample of
    generators (ranks 0, stride, 2*stride, ...), all host cores; then on one
    core over the same generators from rank `stride` on (rank 0, the
    HF-like generator, is far heavier than the rest)."""
    import oracle

    ham = oracle.Hamiltonian(meta["norb"], meta["nalpha"], meta["nbeta"], h, eri)
    threads = oracle.max_threads()
    t0 = time.perf_counter()
    ranks, per, npert, ncon = [], [], 0, 0
    g = 0
    while g < len(dets) and (time.perf_counter() - t0) < budget_s:
        tg = time.perf_counter()
        r = ham.generator(dets, coefs, e0, g, nthreads=threads)
        per.append((g, r["n_perturbers"], time.perf_counter() - tg))
        npert += r["n_perturbers"]
        ncon += r["n_connections"]
        ranks.append(g)
        g += stride
    dt = time.perf_counter() - t0
    t1 = time.perf_counter()
    n1, tall, g1 = 0, 0.0, 0
    for g, n, t in per[1:]:
        if time.perf_counter() - t1 > budget_s / 3:
            break
        n1 += ham.generator(dets, coefs, e0, g, nthreads=1)["n_perturbers"]
        tall += t
        g1 += 1
    dt1 = time.perf_counter() - t1
    return {"value": npert / dt, "unit": UNIT, "cores": threads, "kind": "oracle",
            "sample": f"per-generator oracle on {len(ranks)} of {len(dets)} generators (ranks 0, {stride}, "
                      f"{2 * stride}, ...): {npert} perturbers in {dt:.2f} s",
            "generators_per_s": len(ranks) / dt, "seconds": dt,
            "single_core": {"value": n1 / dt1 if g1 > 0 else None, "unit": UNIT, "cores": 1, "generators": g1,
                            "seconds": dt1, "all_cores_on_same_generators": n1 / tall if tall > 0 else None}}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    meta, h, eri, dets, coefs, e0 = load_workload()
    import oracle

    ham = oracle.Hamiltonian(meta["norb"], meta["nalpha"], meta["nbeta"], h, eri)
    threads = oracle.max_threads()
    per_step = 2  # generators per step (a bounded sample of the workload)
    stride = 97
    g = 0
    times, perts = [], []
    for it in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        n = 0
        for _ in range(per_step):
            n += ham.generator(dets, coefs, e0, g % len(dets), nthreads=threads)["n_perturbers"]
            g += stride
        dt = time.perf_counter() - t0
        if it >= args.warmup:
            times.append(dt)
            perts.append(n)
    T = sum(times)
    value = sum(perts) / T
    sample = (f"per-generator oracle, {per_step} generators per step (ranks stepping by {stride}), "
              f"{sum(perts)} perturbers over {args.steps} steps")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * T / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": workload_config(meta, 1),
            "generators_per_s": per_step * args.steps / T,
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def batched_leg(qp, torch, device, log=None):
    """64 independent instances (orbitals, electrons and N_det drawn per
    instance), each Psi0 grown in the library from the oracle's stored seed
    space (N_det / 8 determinants) by three CIPSI doublings.  The batch runs
    in mixed precision as one CUDA graph of fused launches (one persistent
    launch per wave whose queue spans all instances of a word count), with
    work_chunk, tile and CTAs per SM chosen by the autotuner; it is timed
    against 64 sequential plain FP64 sweeps of the same instances, and the
    same fused graph in FP64 is timed too.  The mixed error is stated per
    instance against its FP64 sweep.  Returns the report dict."""
    from paper_1902_08154_gb300 import autotune, cipsi
    from paper_1902_08154_gb300 import synthetic as S

    z = np.load(os.path.join(ROOT, "tests", "golden", "cfg5seed.npz"))
    specs = json.loads(str(z["meta"]))["specs"]
    t0 = time.perf_counter()
    data = []
    for i, sp in enumerate(specs):
        h, eri = S.hamiltonian_fast(sp["norb"], sp["rank"], sp["seed"])
        hd, ed = torch.from_numpy(h).to(device), torch.from_numpy(eri).to(device)
        g = qp.PT2(sp["norb"], sp["nalpha"], sp["nbeta"], hd, ed)
        dets, coefs, e0, info = cipsi.grow_from_seed(g, z[f"dets_{i}"], 3, tol=1e-10)
        g.close()
        data.append((sp, hd, ed, torch.from_numpy(dets.view(np.int64)).to(device), torch.from_numpy(coefs).to(device),
                     e0, info[-1]["residual"]))
    t_grow = time.perf_counter() - t0
    # sequential plain FP64 sweeps: one context at a time (warm call, timed call)
    seq_ms, seq_pert, e_fp64 = 0.0, 0, []
    for sp, hd, ed, dd, cd, e0, _ in data:
        pt2 = qp.PT2(sp["norb"], sp["nalpha"], sp["nbeta"], hd, ed)
        k = len(dd)
        pt2.eval(dd, cd, e0, k)
        r = pt2.eval(dd, cd, e0, k)
        seq_ms += qp.qp_pt2_last_timings(pt2.ctx)[1]
        seq_pert += r["n_perturbers"]
        e_fp64.append(r["e_pt2"])
        pt2.close()
    torch.cuda.empty_cache()

    def instances(precision):
        out = []
        for sp, hd, ed, dd, cd, e0, _ in data:
            pt2 = qp.PT2(sp["norb"], sp["nalpha"], sp["nbeta"], hd, ed, precision=precision)
            out.append({"pt2": pt2, "dets": dd, "coefs": cd, "e0": e0, "k": len(dd),
                        "precision": int(precision == qp.QP_MIXED)})
        return out

    def run(insts, shape):
        b = qp.Batch(insts, fused=True, **shape)
        b.run()
        res, ms = b.run()
        b.close()
        for i in insts:
            i["pt2"].close()
        torch.cuda.empty_cache()
        return res, ms

    nsm = torch.cuda.get_device_properties(device).multi_processor_count
    insts = instances(qp.QP_MIXED)
    # launch shapes tuned on truncated copies of the instances (first 2000
    # determinants each), cached per batch shape
    trunc = [dict(i, dets=i["dets"][:2000], coefs=i["coefs"][:2000], k=min(i["k"], 2000)) for i in insts]
    t1 = time.perf_counter()
    shape, rec = autotune.tune(trunc, nsm, repeats=1, log=log)
    t_tune = time.perf_counter() - t1
    res, ms = run(insts, shape)
    res64, ms64 = run(instances(qp.QP_FP64), shape)
    pert = sum(r["n_perturbers"] for r in res)
    errs = [abs(r["e_pt2"] - e) for r, e in zip(res, e_fp64)]
    errs64 = [abs(r["e_pt2"] - e) for r, e in zip(res64, e_fp64)]
    same_set = all(r["n_perturbers"] == q["n_perturbers"] and tuple(r["digest"]) == tuple(q["digest"])
                   for r, q in zip(res, res64))
    return {"workload": "64 instances: norb in {24,32,48,64,96}, 6..12 electrons per spin, N_det log-uniform "
                        "1e3..5e4 (total %d determinants), each Psi0 grown from the stored seed space (N_det/8) by "
                        "3 CIPSI doublings, k = N_det, seeds 1000+i" % sum(len(d[3]) for d in data),
            "value": pert / (ms * 1e-3), "unit": UNIT, "graph_ms": ms, "n_perturbers": pert,
            "form": "fused: one persistent launch per wave over all instances of a word count",
            "sequential_fp64": {"value": seq_pert / (seq_ms * 1e-3), "ms": seq_ms, "n_perturbers": seq_pert},
            "speedup_vs_sequential_fp64": seq_ms / ms,
            "fused_fp64": {"ms": ms64, "speedup_vs_sequential_fp64": seq_ms / ms64,
                           "max_abs_diff_vs_sequential_fp64": max(errs64)},
            "precision": "mixed",
            "mixed_abs_err_vs_fp64": {"max": max(errs), "median": float(np.median(errs)), "stated_tolerance": 1e-6,
                                      "instances_within": sum(e <= 1e-6 for e in errs)},
            "same_perturber_sets": same_set,
            "max_davidson_residual": max(d[6] for d in data),
            "autotune": {"shape": shape, "tuned_on": "first 2000 dets of each", "seconds": t_tune,
                         "tried": rec.get("tried")},
            "growth_seconds": t_grow}


def wide_leg(qp, torch, device, flush):
    """The 128-orbital workload (two words per spin; 14+14 electrons, Cholesky
    rank 192, 10^5 determinants, k = N_det).  Psi0 is grown as the workload
    defines it: from the oracle's stored seed space of 12,500 determinants by
    three CIPSI doublings (Davidson to a 1e-10 residual, then the external
    determinants of largest |e_alpha|), in the library.  Then the plain FP64
    sweep and the mixed-precision sweep on the same inputs, one timed sweep
    each after a warm-up on the first 3000 determinants; the mixed error is
    stated against the FP64 GPU sweep (the sampled-generator parity with the
    oracle is in the tests)."""
    from paper_1902_08154_gb300 import cipsi
    from paper_1902_08154_gb300 import synthetic as S

    spec = S.CFG3
    t0 = time.perf_counter()
    h, eri = S.hamiltonian_fast(spec["norb"], spec["rank"], spec["seed"])
    seed = np.load(os.path.join(ROOT, "tests", "golden", "cfg3seed.npz"))
    t_in = time.perf_counter() - t0
    hd, ed = torch.from_numpy(h).to(device), torch.from_numpy(eri).to(device)
    grow_ctx = qp.PT2(spec["norb"], spec["nalpha"], spec["nbeta"], hd, ed)
    t0 = time.perf_counter()
    dets, coefs, e0, info = cipsi.grow_from_seed(grow_ctx, seed["dets"], 3, tol=1e-10)
    t_grow = time.perf_counter() - t0
    grow_ctx.close()
    dd, cd = torch.from_numpy(dets.view(np.int64)).to(device), torch.from_numpy(coefs).to(device)
    n = len(dets)
    hctx = qp.PT2(spec["norb"], spec["nalpha"], spec["nbeta"], hd, ed)
    h_strings = hctx.hamiltonian(dd, search=0)[4]
    h_all = hctx.hamiltonian(dd, search=1)[4]
    hctx.close()
    out = {"h_build_ms_strings": h_strings, "h_build_ms_all_pairs": h_all,
           "workload": f"norb {spec['norb']}, {spec['nalpha']}+{spec['nbeta']} electrons, Cholesky rank "
                       f"{spec['rank']}, seed {spec['seed']}, N_det {n} grown from 12,500 by 3 CIPSI doublings, "
                       "k = N_det",
           "inputs_seconds": t_in, "growth_seconds": t_grow,
           "growth": [{k: v for k, v in r.items() if k in ("ndet", "e0", "residual", "e_pt2", "davidson_ms")}
                      for r in info],
           "e0": e0}
    for name, prec in (("fp64", qp.QP_FP64), ("mixed", qp.QP_MIXED)):
        pt2 = qp.PT2(spec["norb"], spec["nalpha"], spec["nbeta"], hd, ed, precision=prec)
        pt2.eval(dd[:3000], cd[:3000], e0, 3000)
        flush.zero_()
        torch.cuda.synchronize()
        r = pt2.eval(dd, cd, e0, n)
        ms = qp.qp_pt2_last_timings(pt2.ctx)[1]
        if prec == qp.QP_FP64:
            # hybrid deterministic/stochastic E_PT2 to a 0.2 % statistical error
            from paper_1902_08154_gb300 import stochastic as ST

            torch.cuda.synchronize()
            t0 = time.perf_counter()
            st = ST.stochastic_pt2(pt2, dd, cd, e0, rel_err=0.002, seed=11)
            t_st = time.perf_counter() - t0
            out["hybrid_stochastic"] = {
                "seconds": t_st, "e_pt2": st["e_pt2"], "error": st["error"], "prefix": st["prefix"],
                "generators_computed": st["computed"], "draws": st["draws"], "iterations": st["iterations"],
                "deviation_from_deterministic": st["e_pt2"] - r["e_pt2"],
                "speedup_vs_deterministic": (ms * 1e-3) / t_st, "rel_err_target": 0.002}
        pt2.close()
        out[name] = {"ms": ms, "value": r["n_perturbers"] / (ms * 1e-3), "unit": UNIT,
                     "generators_per_s": n / (ms * 1e-3), "e_pt2": r["e_pt2"], "n_perturbers": r["n_perturbers"],
                     "n_connections": r["n_connections"], "digest": [str(x) for x in r["digest"]],
                     "min_abs_denominator": r["min_abs_den"], "e_rpt2": r["e_rpt2"]}
    f, m = out["fp64"], out["mixed"]
    out["mixed_abs_err_vs_fp64_gpu"] = abs(m["e_pt2"] - f["e_pt2"])
    out["same_perturber_set"] = f["digest"] == m["digest"] and f["n_perturbers"] == m["n_perturbers"]
    out["mixed_speedup_vs_fp64"] = f["ms"] / m["ms"]
    out["stated_tolerance"] = 1e-6
    del hd, ed, dd, cd
    torch.cuda.empty_cache()
    return out


def states_leg(qp, torch, pt2, d_dets, k, flush, stream, steps=3):
    """Two states of the same Psi0 (the two lowest eigenpairs of H over it,
    by ARPACK on the library's H U product): one multi-state sweep (per-state
    E_PT2, selection by the multi-state criterion) against the two one-state
    sweeps it replaces."""
    from scipy.sparse.linalg import LinearOperator, eigsh

    n = len(d_dets)

    def hv(v):
        u = torch.from_numpy(np.ascontiguousarray(np.asarray(v, dtype=np.float64).reshape(1, n))).to(d_dets.device)
        return pt2.sigma(d_dets, u).cpu().numpy().reshape(n)

    w, v = eigsh(LinearOperator((n, n), matvec=hv, dtype=np.float64), k=2, which="SA", tol=1e-12)
    order = np.argsort(w)
    E = np.ascontiguousarray(w[order])
    C = torch.from_numpy(np.ascontiguousarray(v[:, order].T)).to(d_dets.device)
    sel = torch.zeros((k, 2, pt2.nint), dtype=torch.int64, device=d_dets.device)
    crit = torch.zeros(k, dtype=torch.float64, device=d_dets.device)
    num = torch.zeros(k, dtype=torch.float64, device=d_dets.device)
    sel1 = torch.zeros_like(sel)
    se1 = torch.zeros_like(crit)
    ms_t, one_t = [], []
    with torch.cuda.stream(stream):
        for it in range(1 + steps):
            flush.zero_()
            rc, res = qp.qp_pt2_eval_states(pt2.ctx, n, d_dets, C, E, k, sel, crit, num, check=False)
            if it:
                ms_t.append(qp.qp_pt2_last_timings(pt2.ctx)[1])
            one = []
            for s in range(2):
                flush.zero_()
                _, r1 = qp.qp_pt2_eval_ex(pt2.ctx, n, d_dets, C[s].contiguous(), float(E[s]), k, sel1, se1,
                                          check=False)
                one.append(r1.as_dict())
                if it:
                    one_t.append(qp.qp_pt2_last_timings(pt2.ctx)[1])
    ms = statistics.mean(ms_t)
    two = 2 * statistics.mean(one_t)
    return {"workload": "the same Psi0 with its two lowest eigenpairs (ARPACK on H U), k as above",
            "rc": rc, "e0": E.tolist(), "e_pt2": [r.e_pt2 for r in res],
            "ms": ms, "value": res[0].n_perturbers / (ms * 1e-3), "unit": UNIT,
            "two_one_state_sweeps_ms": two, "speedup_vs_two_one_state_sweeps": two / ms,
            "abs_err_vs_one_state_sweeps": max(abs(res[s].e_pt2 - one[s]["e_pt2"]) for s in range(2)),
            "min_abs_denominator": res[0].min_abs_denominator, "n_selected": res[0].n_selected}


def run_gb300(args):
    import torch

    import paper_1902_08154_gb300 as qp
    from paper_1902_08154_gb300.shard import distributed_merge

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist

        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    device = torch.device("cuda", torch.cuda.current_device())
    qp.load()
    meta, h, eri, dets, coefs, e0 = load_workload()
    if args.ndet:
        dets, coefs = dets[: args.ndet].copy(), coefs[: args.ndet].copy()
        meta = dict(meta, ndet=len(dets), k=min(meta["k"], 2 * len(dets)))
    k = meta["k"]
    stream = torch.cuda.Stream(device=device)
    pt2 = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], h, eri, stream=stream.cuda_stream,
                 shard_index=rank if world > 1 else 0, shard_count=world if world > 1 else 0)
    nint = pt2.nint
    d_dets = torch.from_numpy(dets.view(np.int64)).to(device)
    d_coefs = torch.from_numpy(coefs).to(device)
    sel = torch.zeros((k, 2, nint), dtype=torch.int64, device=device)
    sel_e = torch.zeros(k, dtype=torch.float64, device=device)
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=device)
    ndet = len(dets)

    def step():
        res = qp.qp_pt2_eval(pt2.ctx, ndet, d_dets, d_coefs, e0, k, sel, sel_e).as_dict()
        return res

    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            flush.zero_()
            res = step()
            if dist:
                distributed_merge(dist, res, sel_e[: res["n_selected"]], sel[: res["n_selected"]], k, device, e0)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = Clocks(local)
    clocks.start()
    evs = []
    sweep_ms, call_ms, launches, units = [], [], 0, 0
    with torch.cuda.stream(stream):
        for _ in range(args.steps):
            flush.zero_()
            e0v, e1v = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0v.record(stream)
            res = step()
            if dist:
                tot, _, _ = distributed_merge(dist, res, sel_e[: res["n_selected"]], sel[: res["n_selected"]],
                                              k, device, e0)
                units = int(tot["n_perturbers"])
            else:
                units = res["n_perturbers"]
            e1v.record(stream)
            evs.append((e0v, e1v))
            tms = qp.qp_pt2_last_timings(pt2.ctx)
            sweep_ms.append(tms[0])
            call_ms.append(tms[1])
            launches += qp.qp_pt2_last_launches(pt2.ctx)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    ck = clocks.stop()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    T = sum(step_ms)
    if dist:
        tt = torch.tensor([T], dtype=torch.float64, device=device)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        T = float(tt.item())
    ms_step = T / args.steps
    value = units / (ms_step * 1e-3)
    gens_per_s = ndet / (ms_step * 1e-3)

    e2e = None
    if not args.no_e2e:
        # end to end through the C ABI with pinned host buffers
        h_dets = torch.from_numpy(dets.view(np.int64)).pin_memory()
        h_coefs = torch.from_numpy(coefs).pin_memory()
        h_sel = torch.zeros((k, 2, nint), dtype=torch.int64).pin_memory()
        h_sel_e = torch.zeros(k, dtype=torch.float64).pin_memory()
        e2e_times = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + args.steps):
                flush.zero_()
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                res2 = qp.qp_pt2_eval(pt2.ctx, ndet, h_dets, h_coefs, e0, k, h_sel, h_sel_e).as_dict()
                if dist:
                    distributed_merge(dist, res2, h_sel_e[: res2["n_selected"]].to(device),
                                      h_sel[: res2["n_selected"]].to(device), k, device)
                t1 = time.perf_counter()
                if it >= args.warmup:
                    e2e_times.append(t1 - t0)
        e2e_T = sum(e2e_times)
        if dist:
            tt = torch.tensor([e2e_T], dtype=torch.float64, device=device)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            e2e_T = float(tt.item())
        e2e_val = units / (e2e_T / args.steps)
        h2d = dets.nbytes + coefs.nbytes
        d2h = res2["n_selected"] * (2 * nint * 8 + 8) + 88

        e2e = {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h}

    # mixed precision on the same inputs: FP32 numerator, FP64 accumulation,
    # denominators and reductions; error stated against the FP64 sweep and
    # against the oracle's stored value
    mixed = None
    if not args.no_mixed:
        pt2m = qp.PT2(meta["norb"], meta["nalpha"], meta["nbeta"], h, eri, stream=stream.cuda_stream,
                      shard_index=rank if world > 1 else 0, shard_count=world if world > 1 else 0,
                      precision=qp.QP_MIXED)
        mt = []
        with torch.cuda.stream(stream):
            for it in range(args.warmup + args.steps):
                flush.zero_()
                resm = qp.qp_pt2_eval(pt2m.ctx, ndet, d_dets, d_coefs, e0, k, sel, sel_e).as_dict()
                if it >= args.warmup:
                    mt.append(qp.qp_pt2_last_timings(pt2m.ctx)[1])
        pt2m.close()
        ms_m = statistics.mean(mt)
        ref_e = None
        if not args.ndet:
            E = np.load(os.path.join(ROOT, "tests", "golden", f"{WORKLOAD}_expected.npz"))
            ref_e = json.loads(str(E["summary"]))["e_pt2"]
        mixed = {"value": resm["n_perturbers"] / (ms_m * 1e-3), "unit": UNIT, "ms_per_step": ms_m,
                 "speedup_vs_fp64": ms_step / ms_m, "e_pt2": resm["e_pt2"],
                 "abs_err_vs_fp64_gpu": abs(resm["e_pt2"] - res["e_pt2"]),
                 "abs_err_vs_oracle": None if ref_e is None else abs(resm["e_pt2"] - ref_e),
                 "stated_tolerance": 1e-6}

    batched = None
    if not args.no_batched and world == 1:
        batched = batched_leg(qp, torch, device)

    wide = None
    if not args.no_wide and world == 1:
        wide = wide_leg(qp, torch, device, flush)

    # the adjoint (pattern 3) on the stored 48-orbital workload: dE_PT2/dh,
    # dE_PT2/d(packed eri) and dE/dE0, against the oracle's stored gradient
    adj = None
    if world == 1 and not args.ndet and not args.no_davidson:
        G = np.load(os.path.join(ROOT, "tests", "golden", "cfg4_gradient.npz"))
        P4 = np.load(os.path.join(ROOT, "tests", "golden", "cfg4_psi0.npz"))
        m4 = json.loads(str(P4["meta"]))
        from paper_1902_08154_gb300 import synthetic as S4

        h4, eri4 = S4.hamiltonian(m4["norb"], m4["rank"], m4["seed"])
        ctx4 = qp.PT2(m4["norb"], m4["nalpha"], m4["nbeta"], torch.from_numpy(h4).to(device),
                      torch.from_numpy(eri4).to(device))
        d4 = torch.from_numpy(P4["dets"].view(np.int64)).to(device)
        c4 = torch.from_numpy(P4["coefs"]).to(device)
        dh4 = torch.zeros((m4["norb"], m4["norb"]), dtype=torch.float64, device=device)
        de4 = torch.zeros(len(eri4), dtype=torch.float64, device=device)
        qp.qp_pt2_grad(ctx4.ctx, len(d4), d4, c4, float(P4["e0"]), dh4, de4)
        ta, tb = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        ta.record()
        g0, r4 = qp.qp_pt2_grad(ctx4.ctx, len(d4), d4, c4, float(P4["e0"]), dh4, de4)
        tb.record()
        torch.cuda.synchronize()
        ctx4.close()
        scale = max(1.0, float(np.abs(G["deri"]).max()))
        adj = {"workload": f"norb {m4['norb']}, {m4['nalpha']}+{m4['nbeta']} electrons, N_det {len(d4)}",
               "ms": ta.elapsed_time(tb), "e_pt2": r4.e_pt2,
               "max_rel_err_vs_oracle": max(float(np.abs(de4.cpu().numpy() - G["deri"]).max()),
                                            float(np.abs(dh4.cpu().numpy() - G["dh"]).max())) / scale,
               "de0_abs_err_vs_oracle": abs(g0 - float(G["de0"]))}

    # the variational step on the same Psi0: H over Psi0 and its lowest
    # eigenpair by Davidson (residual 1e-10), against the stored E0 of the
    # oracle's Davidson
    dav = None
    if world == 1 and not args.ndet and not args.no_davidson:
        e0d, _, di = pt2.davidson(d_dets, tol=1e-10)
        # the pair search of the H build: through the spin strings (used by
        # Davidson) against the test of every pair
        hs = pt2.hamiltonian(d_dets, search=0)
        ha = pt2.hamiltonian(d_dets, search=1)
        dav = {"ms": di["build_ms"] + di["solve_ms"], "build_ms": di["build_ms"], "solve_ms": di["solve_ms"],
               "iterations": di["iterations"], "nnz": di["nnz"], "e0": e0d,
               "abs_err_vs_oracle_e0": abs(e0d - e0),
               "h_build_ms_strings": hs[4], "h_build_ms_all_pairs": ha[4],
               "same_matrix": bool(np.array_equal(hs[1], ha[1]) and np.array_equal(hs[2], ha[2]))}

    # several states of the same Psi0: one multi-state sweep against two
    # one-state sweeps
    states = None
    if world == 1 and not args.ndet and not args.no_states:
        states = states_leg(qp, torch, pt2, d_dets, k, flush, stream)

    # roofline of the dominant kernel (the persistent sweep), against the
    # FP64 and integer rates measured on this GPU in this run
    from paper_1902_08154_gb300 import peaks

    pk64 = peaks.measure("fp64")
    pkint = peaks.measure("int")
    ms_sweep = statistics.mean(sweep_ms)
    ops = FP64_OPS_PER_CONNECTION * res["n_connections"] + FP64_OPS_PER_PERTURBER * res["n_perturbers"]
    ops_min = FP64_OPS_PER_CONNECTION * res["n_connections"] + FP64_OPS_PER_PERTURBER_MIN * res["n_perturbers"]
    achieved = ops / (ms_sweep * 1e-3) / 1e9
    int_ops = (INT_OPS_PER_CONNECTION_PER_WORD * nint * res["n_connections"]
               + 4 * nint * float(ndet) * float(ndet) / max(world, 1))
    int_ach = int_ops / (ms_sweep * 1e-3) / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": pk64["gops"], "unit": "G FP64 op/s",
            "frac": achieved / pk64["gops"], "traffic": None if args.ndet else TRAFFIC_BYTES_PER_SWEEP,
            "kernel": "qp::prep_kernel + qp::batch_kernel (all waves of one sweep)",
            "kernel_ms": ms_sweep, "call_ms": statistics.mean(call_ms),
            "peak_source": "measured in this run: FP64 FMA throughput kernel (paper_1902_08154_gb300/csrc/peaks.cu), "
                           f"{pk64['ops_per_sm_clock']:.3f} FMA per SM clock at {pk64['implied_sm_mhz']:.0f} MHz",
            "ops_model": f"{FP64_OPS_PER_CONNECTION} FP64 op/connection + {FP64_OPS_PER_PERTURBER} FP64 op/perturber",
            "frac_min_ops": ops_min / (ms_sweep * 1e-3) / 1e9 / pk64["gops"],
            "min_ops_model": f"{FP64_OPS_PER_CONNECTION} FP64 op/connection + {FP64_OPS_PER_PERTURBER_MIN} "
                             "FP64 op/perturber (the operations the kernels execute at least)",
            "int_issue": {"achieved": int_ach, "peak": pkint["gops"], "unit": "G int op/s",
                          "frac": int_ach / pkint["gops"],
                          "ops_model": f"{INT_OPS_PER_CONNECTION_PER_WORD} x nint per connection + "
                                       "4 x nint per coarse-filter pair test"}}
    if rank != 0:
        return 0
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_step, "higher_is_better": True, "scaling": "strong",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "config": workload_config(meta, world),
            "generators_per_s": gens_per_s, "n_perturbers": units, "e_pt2": res["e_pt2"],
            "rpt2": qp.rpt2(res, e0),
            "e2e": e2e,
            "gpu_launches": launches, "roofline": roof, "clocks": ck, "mixed_precision": mixed,
            "batched": batched, "workload_128_orbitals": wide, "davidson": dav, "adjoint": adj,
            "multi_state": states}
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(meta, h, eri, dets, coefs, e0)
    print(json.dumps(line), flush=True)
    pt2.close()
    if dist:
        dist.destroy_process_group()
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="gb300", choices=["gb300", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer leg (profiling runs)")
    ap.add_argument("--no-mixed", action="store_true", help="skip the mixed-precision leg (profiling runs)")
    ap.add_argument("--no-batched", action="store_true", help="skip the 64-instance batched leg")
    ap.add_argument("--no-wide", action="store_true", help="skip the 128-orbital, 10^5-determinant leg")
    ap.add_argument("--no-davidson", action="store_true", help="skip the Davidson leg")
    ap.add_argument("--no-states", action="store_true", help="skip the two-state leg")
    ap.add_argument("--ndet", type=int, default=0,
                    help="profiling runs only: sweep the first NDET determinants of the stored Psi0")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_gb300(args)


if __name__ == "__main__":
    sys.exit(main())
