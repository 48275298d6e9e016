"""Build the CUDA library ``_build/libqp_pt2.so`` for sm_103a with nvcc.

Translation units are compiled in parallel and linked into one shared
library; nothing is installed outside this directory.
"""
from __future__ import annotations

import os
import subprocess
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
SO = os.path.join(OUT, "libqp_pt2.so")
# measured pipe throughput (FP64 FMA, integer XOR/POPC/add) for the roofline
PEAKS_SO = os.path.join(OUT, "libqp_peaks.so")
UNITS = ["qp_pt2.cu", "sweep.cu", "sweep_mixed.cu", "sweep_grad.cu", "sweep_states.cu", "sweep_packed.cu",
         "noalloc.cu", "davidson.cu"]
HEADERS = ["common.cuh", "sweep_impl.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(SRC, h) for h in HEADERS] + [os.path.join(HERE, "..", "include", "qp_pt2.h")]
    objs, jobs = [], []
    for u in UNITS:
        src = os.path.join(SRC, u)
        obj = os.path.join(OUT, u.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdrs):
            jobs.append([nvcc, *ARCH, *FLAGS, "-c", src, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
        if verbose:
            print(r.stdout + r.stderr)

    peaks_src = os.path.join(SRC, "peaks.cu")
    if force or _stale(PEAKS_SO, [peaks_src]):
        jobs.append([nvcc, *ARCH, *FLAGS, "-shared", peaks_src, "-o", PEAKS_SO + f".tmp{os.getpid()}"])
    with ThreadPoolExecutor(max_workers=len(UNITS) + 1) as ex:
        list(ex.map(run, jobs))
    if os.path.exists(PEAKS_SO + f".tmp{os.getpid()}"):
        os.replace(PEAKS_SO + f".tmp{os.getpid()}", PEAKS_SO)
    if force or jobs or _stale(SO, objs):
        tmp = SO + f".tmp{os.getpid()}"
        run([nvcc, *ARCH, "-shared", *objs, "-o", tmp])
        os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force=True, verbose=True))
