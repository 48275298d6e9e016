"""GB300 (sm_103a) EN-PT2 + CIPSI selection sweep: Python binding.

Thin ctypes binding over the C ABI of ``include/qp_pt2.h`` with the same
entry-point names.  It only marshals arguments (numpy arrays for host memory,
torch CUDA tensors for device memory); every step of the sweep runs in the
CUDA library ``_build/libqp_pt2.so``.  If that library is missing or cannot
be loaded, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SO = os.path.join(HERE, "_build", "libqp_pt2.so")

QP_OK, QP_EINVAL, QP_EDUP, QP_ESYM, QP_ESINGULAR, QP_ENOMEM, QP_ECUDA, QP_ENOTSUP = 0, -1, -2, -3, -4, -5, -6, -8
QP_ETIMEOUT, QP_ENOTCONV = -7, -9
QP_FP64 = 0
QP_MIXED = 1

EXPORTS = (
    "qp_pt2_create",
    "qp_pt2_eval",
    "qp_pt2_eval_ex",
    "qp_pt2_eval_gens",
    "qp_pt2_eval_states",
    "qp_pt2_sigma",
    "qp_pt2_set_target",
    "qp_pt2_davidson",
    "qp_pt2_hamiltonian",
    "qp_pt2_last_launches",
    "qp_pt2_last_timings",
    "qp_pt2_destroy",
    "qp_pt2_strerror",
    "qp_pt2_last_error",
    "qp_pt2_eval_noalloc",
    "qp_pt2_merge_results",
    "qp_pt2_reduce_ranks",
    "qp_pt2_grad",
    "qp_pt2_batch_create",
    "qp_pt2_batch_create_ex",
    "qp_pt2_batch_run",
    "qp_pt2_batch_destroy",
)


class Config(C.Structure):
    _fields_ = [("precision", C.c_int), ("stream", C.c_void_p), ("blocks_per_sm", C.c_int), ("threads", C.c_int),
                ("shard_index", C.c_int), ("shard_count", C.c_int), ("work_chunk", C.c_int), ("tile", C.c_int),
                ("timeout_s", C.c_double)]


class Result(C.Structure):
    _fields_ = [
        ("e_pt2", C.c_double),
        ("sum_e_over_d", C.c_double),
        ("min_abs_denominator", C.c_double),
        ("n_perturbers", C.c_int64),
        ("n_connections", C.c_int64),
        ("n_selected", C.c_int64),
        ("n_tiny", C.c_int64),
        ("perturber_digest", C.c_uint64 * 2),
        ("z", C.c_double),
        ("e_rpt2", C.c_double),
    ]

    def as_dict(self):
        return {
            "e_pt2": self.e_pt2,
            "sum_e_over_d": self.sum_e_over_d,
            "min_abs_den": self.min_abs_denominator,
            "n_perturbers": self.n_perturbers,
            "n_connections": self.n_connections,
            "n_selected": self.n_selected,
            "n_tiny": self.n_tiny,
            "digest": (int(self.perturber_digest[0]), int(self.perturber_digest[1])),
            "z": self.z,
            "e_rpt2": self.e_rpt2,
        }


def rpt2(res, e0=None):
    """Renormalised PT2 (Sec. "Renormalized PT2") of a result dict: Z and
    E0 + Z E_PT2, as the library computed them."""
    return {"z": res["z"], "e_rpt2": res["e_rpt2"]}


def merge_results(parts, e0):
    """Merge of the partial results of generator shards (dicts as returned
    by the sweeps) through qp_pt2_merge_results: sums and counts add, the
    digest words add modulo 2^64 and xor, Z and E_rPT2 are recomputed."""
    n = len(parts)
    arr = (Result * n)()
    for i, p in enumerate(parts):
        r = arr[i]
        r.e_pt2 = float(p["e_pt2"])
        r.sum_e_over_d = float(p["sum_e_over_d"])
        r.min_abs_denominator = float(p.get("min_abs_den", float("inf")))
        r.n_perturbers = int(p["n_perturbers"])
        r.n_connections = int(p["n_connections"])
        r.n_tiny = int(p.get("n_tiny", 0))
        r.perturber_digest[0] = int(p["digest"][0]) & ((1 << 64) - 1)
        r.perturber_digest[1] = int(p["digest"][1]) & ((1 << 64) - 1)
    out = Result()
    _check(load().qp_pt2_merge_results(n, arr, float(e0), C.byref(out)))
    return out.as_dict()


class DavidsonInfo(C.Structure):
    _fields_ = [("iterations", C.c_int), ("converged", C.c_int), ("residual", C.c_double), ("nnz", C.c_int64),
                ("build_ms", C.c_double), ("solve_ms", C.c_double)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class QPError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{msg} (code {code})")
        self.code = code


_lib = None


def load(path: str = SO):
    """Load the CUDA library (raises if it is absent: no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise ImportError(f"CUDA library not built: {path} (run __graft_entry__.build())")
    L = C.CDLL(path)
    vp, i64, dbl = C.c_void_p, C.c_int64, C.c_double
    L.qp_pt2_create.restype = C.c_int
    L.qp_pt2_create.argtypes = [C.POINTER(vp), C.c_int, C.c_int, C.c_int, vp, vp, C.POINTER(Config)]
    L.qp_pt2_eval.restype = C.c_int
    L.qp_pt2_eval.argtypes = [vp, i64, vp, vp, dbl, i64, vp, vp, C.POINTER(Result)]
    L.qp_pt2_eval_ex.restype = C.c_int
    L.qp_pt2_eval_ex.argtypes = [vp, i64, vp, vp, dbl, i64, vp, vp, vp, vp, vp, vp, vp, C.POINTER(Result)]
    L.qp_pt2_set_target.restype = C.c_int
    L.qp_pt2_set_target.argtypes = [vp, vp, C.c_int, vp, vp]
    L.qp_pt2_sigma.restype = C.c_int
    L.qp_pt2_sigma.argtypes = [vp, i64, vp, C.c_int, vp, vp]
    L.qp_pt2_davidson.restype = C.c_int
    L.qp_pt2_davidson.argtypes = [vp, i64, vp, vp, dbl, C.c_int, vp, vp, C.POINTER(DavidsonInfo)]
    L.qp_pt2_hamiltonian.restype = C.c_int
    L.qp_pt2_hamiltonian.argtypes = [vp, i64, vp, C.c_int, C.POINTER(C.c_int64), vp, vp, vp, vp,
                                     C.POINTER(C.c_double)]
    L.qp_pt2_eval_gens.restype = C.c_int
    L.qp_pt2_eval_gens.argtypes = [vp, i64, vp, vp, dbl, i64, vp, i64, vp, vp, vp, vp, vp, vp, C.POINTER(Result)]
    L.qp_pt2_reduce_ranks.restype = C.c_int
    L.qp_pt2_reduce_ranks.argtypes = [vp, i64, vp, vp, vp, vp, dbl, C.POINTER(Result)]
    L.qp_pt2_eval_states.restype = C.c_int
    L.qp_pt2_eval_states.argtypes = [vp, i64, vp, C.c_int, vp, vp, i64, vp, vp, vp, C.POINTER(Result)]
    L.qp_pt2_last_launches.restype = i64
    L.qp_pt2_last_launches.argtypes = [vp]
    L.qp_pt2_last_timings.restype = C.c_int
    L.qp_pt2_last_timings.argtypes = [vp, C.POINTER(C.c_double)]
    L.qp_pt2_destroy.restype = None
    L.qp_pt2_destroy.argtypes = [vp]
    L.qp_pt2_strerror.restype = C.c_char_p
    L.qp_pt2_strerror.argtypes = [C.c_int]
    L.qp_pt2_last_error.restype = C.c_char_p
    L.qp_pt2_last_error.argtypes = []
    L.qp_pt2_grad.restype = C.c_int
    L.qp_pt2_grad.argtypes = [vp, i64, vp, vp, dbl, vp, vp, vp, C.POINTER(Result)]
    L.qp_pt2_merge_results.restype = C.c_int
    L.qp_pt2_merge_results.argtypes = [C.c_int, C.c_void_p, C.c_double, C.POINTER(Result)]
    L.qp_pt2_eval_noalloc.restype = C.c_int
    L.qp_pt2_eval_noalloc.argtypes = [C.c_int, C.c_int, C.c_int, vp, vp, i64, vp, vp, dbl, i64, vp, vp,
                                      C.POINTER(Result), vp]
    _lib = L
    return L


def _ptr(a):
    """Raw pointer of a numpy array or torch tensor (None stays NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _check(rc):
    if rc != QP_OK:
        L = load()
        raise QPError(rc, f"{L.qp_pt2_strerror(rc).decode()}: {L.qp_pt2_last_error().decode()}")


def qp_pt2_create(norb, n_alpha, n_beta, h, eri, stream=None, blocks_per_sm=0, precision=QP_FP64,
                  shard_index=0, shard_count=0, work_chunk=0, tile=0, timeout_s=0.0):
    """Create a context; h and eri are float64 numpy arrays or CUDA tensors."""
    L = load()
    cfg = Config(precision, stream or None, blocks_per_sm, 0, shard_index, shard_count, work_chunk, tile,
                 float(timeout_s))
    out = C.c_void_p()
    _check(L.qp_pt2_create(C.byref(out), norb, n_alpha, n_beta, _ptr(h), _ptr(eri), C.byref(cfg)))
    return out


def qp_pt2_destroy(ctx):
    load().qp_pt2_destroy(ctx)


def qp_pt2_eval(ctx, ndet, dets, coefs, e0, k, sel_dets=None, sel_e=None):
    res = Result()
    _check(load().qp_pt2_eval(ctx, ndet, _ptr(dets), _ptr(coefs), float(e0), k, _ptr(sel_dets), _ptr(sel_e),
                              C.byref(res)))
    return res


def qp_pt2_eval_ex(ctx, ndet, dets, coefs, e0, k, sel_dets=None, sel_e=None, sel_num=None, eps_by_rank=None,
                   na_by_rank=None, ncon_by_rank=None, rank_of=None, check=True):
    res = Result()
    rc = load().qp_pt2_eval_ex(ctx, ndet, _ptr(dets), _ptr(coefs), float(e0), k, _ptr(sel_dets), _ptr(sel_e),
                               _ptr(sel_num), _ptr(eps_by_rank), _ptr(na_by_rank), _ptr(ncon_by_rank),
                               _ptr(rank_of), C.byref(res))
    if check:
        _check(rc)
    return rc, res


def qp_pt2_eval_gens(ctx, ndet, dets, coefs, e0, ranks, k=0, sel_dets=None, sel_e=None, gen_eps=None, gen_na=None,
                     gen_ncon=None, check=True, gen_s2=None):
    """Sweep of the listed generator ranks only (``ranks``: host int32 array)."""
    ranks = np.ascontiguousarray(ranks, dtype=np.int32)
    res = Result()
    rc = load().qp_pt2_eval_gens(ctx, ndet, _ptr(dets), _ptr(coefs), float(e0), len(ranks), _ptr(ranks), k,
                                 _ptr(sel_dets), _ptr(sel_e), _ptr(gen_eps), _ptr(gen_s2), _ptr(gen_na),
                                 _ptr(gen_ncon), C.byref(res))
    if check:
        _check(rc)
    return rc, res


def qp_pt2_eval_states(ctx, ndet, dets, coefs, e0, k=0, sel_dets=None, sel_crit=None, sel_num=None, check=True):
    """Several states at once (``coefs``: [nstates, ndet]; ``e0``: host
    energies); returns (return code, list of per-state Results)."""
    e0 = np.ascontiguousarray(np.atleast_1d(e0), dtype=np.float64)
    nst = len(e0)
    res = (Result * max(nst, 1))()
    rc = load().qp_pt2_eval_states(ctx, ndet, _ptr(dets), nst, _ptr(coefs), _ptr(e0), k, _ptr(sel_dets),
                                   _ptr(sel_crit), _ptr(sel_num), res)
    if check:
        _check(rc)
    return rc, [res[i] for i in range(nst)]


def qp_pt2_sigma(ctx, ndet, dets, U, S):
    """S[k] = H U[k] over Psi0 (U, S: [nvec, ndet], host or device)."""
    _check(load().qp_pt2_sigma(ctx, ndet, _ptr(dets), int(U.shape[0]), _ptr(U), _ptr(S)))
    return S


def qp_pt2_davidson(ctx, ndet, dets, coefs_out, guess=None, tol=1e-10, max_iter=1000, check=True):
    """Lowest eigenpair of H over Psi0; returns (rc, e0, info dict)."""
    e0 = C.c_double(0.0)
    info = DavidsonInfo()
    rc = load().qp_pt2_davidson(ctx, ndet, _ptr(dets), _ptr(guess), float(tol), int(max_iter), _ptr(coefs_out),
                                C.byref(e0), C.byref(info))
    if check:
        _check(rc)
    return rc, e0.value, info.as_dict()


def qp_pt2_eval_noalloc(norb, n_alpha, n_beta, h, eri, ndet, dets, coefs, e0, k, sel_dets=None, sel_e=None,
                        stream=None):
    """The sweep with no device allocation (every array a CUDA tensor); see
    include/qp_pt2.h.  Returns (return code, Result)."""
    res = Result()
    rc = load().qp_pt2_eval_noalloc(norb, n_alpha, n_beta, _ptr(h), _ptr(eri), ndet, _ptr(dets), _ptr(coefs),
                                    float(e0), k, _ptr(sel_dets), _ptr(sel_e), C.byref(res), stream or None)
    return rc, res


def qp_pt2_grad(ctx, ndet, dets, coefs, e0, dh, deri):
    """Gradient of E_PT2 (see include/qp_pt2.h); fills dh and deri, returns
    (dE/dE0, Result)."""
    res = Result()
    de0 = C.c_double()
    _check(load().qp_pt2_grad(ctx, ndet, _ptr(dets), _ptr(coefs), float(e0), _ptr(dh), _ptr(deri),
                              C.byref(de0), C.byref(res)))
    return de0.value, res


def qp_pt2_last_launches(ctx):
    return int(load().qp_pt2_last_launches(ctx))


def qp_pt2_last_timings(ctx):
    """(sweep kernel ms, whole call ms) of the last call, from CUDA events."""
    ms = (C.c_double * 2)()
    _check(load().qp_pt2_last_timings(ctx, ms))
    return float(ms[0]), float(ms[1])


class PT2:
    """Owning wrapper: one context per (Hamiltonian, electron count)."""

    def __init__(self, norb, n_alpha, n_beta, h, eri, stream=None, blocks_per_sm=0, shard_index=0,
                 shard_count=0, precision=QP_FP64, work_chunk=0, tile=0, timeout_s=0.0):
        self.norb, self.n_alpha, self.n_beta = norb, n_alpha, n_beta
        self.nint = (norb - 1) // 64 + 1
        self.ctx = qp_pt2_create(norb, n_alpha, n_beta, h, eri, stream, blocks_per_sm, precision=precision,
                                 shard_index=shard_index, shard_count=shard_count, work_chunk=work_chunk,
                                 tile=tile, timeout_s=timeout_s)

    def close(self):
        if getattr(self, "ctx", None) is not None and _lib is not None:
            qp_pt2_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        self.close()

    def eval(self, dets, coefs, e0, k, per_generator=False, check=True):
        """Sweep with host (numpy) or device (torch CUDA) inputs; outputs are
        allocated in the same kind of memory as ``dets``."""
        ndet = len(dets)
        on_device = not isinstance(dets, np.ndarray)
        if on_device:
            import torch

            dev = dets.device
            sel = torch.zeros((max(k, 1), 2, self.nint), dtype=torch.int64, device=dev)
            se = torch.zeros(max(k, 1), dtype=torch.float64, device=dev)
            sn = torch.zeros(max(k, 1), dtype=torch.float64, device=dev)
            if per_generator:
                eps = torch.zeros(max(ndet, 1), dtype=torch.float64, device=dev)
                na = torch.zeros(max(ndet, 1), dtype=torch.int64, device=dev)
                nc = torch.zeros(max(ndet, 1), dtype=torch.int64, device=dev)
                rk = torch.zeros(max(ndet, 1), dtype=torch.int32, device=dev)
        else:
            sel = np.zeros((max(k, 1), 2, self.nint), dtype=np.uint64)
            se = np.zeros(max(k, 1))
            sn = np.zeros(max(k, 1))
            if per_generator:
                eps = np.zeros(max(ndet, 1))
                na = np.zeros(max(ndet, 1), dtype=np.int64)
                nc = np.zeros(max(ndet, 1), dtype=np.int64)
                rk = np.zeros(max(ndet, 1), dtype=np.int32)
        if not per_generator:
            eps = na = nc = rk = None
        rc, res = qp_pt2_eval_ex(self.ctx, ndet, dets, coefs, e0, k, sel if k else None, se if k else None,
                                 sn if k else None, eps, na, nc, rk, check=check)
        out = res.as_dict()
        out["rc"] = rc
        m = res.n_selected
        out.update(sel_dets=sel[:m], sel_e=se[:m], sel_num=sn[:m])
        if per_generator:
            out.update(eps_by_rank=eps[:ndet], na_by_rank=na[:ndet], ncon_by_rank=nc[:ndet], rank_of=rk[:ndet])
        out["launches"] = qp_pt2_last_launches(self.ctx)
        return out

    def set_target(self, ref=None, max_exc=-1, core=None, deleted=None):
        """Restrict the external space (see qp_pt2_set_target); host arrays
        in determinant layout, all None clears it."""
        arrs = [None if a is None else np.ascontiguousarray(a, dtype=np.uint64) for a in (ref, core, deleted)]
        self._tgt = arrs
        _check(load().qp_pt2_set_target(self.ctx, _ptr(arrs[0]), int(max_exc), _ptr(arrs[1]), _ptr(arrs[2])))

    def sigma(self, dets, U):
        """H U over Psi0 for the rows of U ([nvec, ndet]), in U's memory kind."""
        if isinstance(U, np.ndarray):
            U = np.ascontiguousarray(U, dtype=np.float64)
            S = np.zeros_like(U)
        else:
            U = U.contiguous()
            S = U.new_zeros(U.shape)
        return qp_pt2_sigma(self.ctx, len(dets), dets, U, S)

    def davidson(self, dets, guess=None, tol=1e-10, max_iter=1000):
        """(E0, coefficients, info) of the lowest eigenpair of H over Psi0."""
        if isinstance(dets, np.ndarray):
            c = np.zeros(len(dets))
        else:
            import torch

            c = torch.zeros(len(dets), dtype=torch.float64, device=dets.device)
        _, e0, info = qp_pt2_davidson(self.ctx, len(dets), dets, c, guess, tol, max_iter)
        return e0, c, info

    def hamiltonian(self, dets, search=0):
        """H over Psi0: (rowptr, cols, vals, diag, build ms) as host arrays;
        search 0 = through the spin strings, 1 = every pair."""
        L = load()
        nnz = C.c_int64()
        ms = C.c_double()
        _check(L.qp_pt2_hamiltonian(self.ctx, len(dets), _ptr(dets), int(search), C.byref(nnz), None, None, None,
                                    None, None))
        n = len(dets)
        rowptr = np.zeros(n + 1, dtype=np.int64)
        cols = np.zeros(max(nnz.value, 1), dtype=np.int32)
        vals = np.zeros(max(nnz.value, 1))
        diag = np.zeros(n)
        _check(L.qp_pt2_hamiltonian(self.ctx, n, _ptr(dets), int(search), C.byref(nnz), _ptr(rowptr), _ptr(cols),
                                    _ptr(vals), _ptr(diag), C.byref(ms)))
        return rowptr, cols[: nnz.value], vals[: nnz.value], diag, ms.value

    def eval_states(self, dets, coefs, e0, k, check=True):
        """Several states of one internal space (``coefs`` [nstates, ndet],
        ``e0`` [nstates]): per-state E_PT2 and sum A^2/D^2, the shared
        counts, and the k determinants of largest multi-state criterion
        (``sel_crit``) with state 0's numerator (``sel_num``), in the memory
        kind of ``dets``."""
        if isinstance(dets, np.ndarray):
            coefs = np.ascontiguousarray(np.atleast_2d(coefs), dtype=np.float64)
            sel = np.zeros((max(k, 1), 2, self.nint), dtype=np.uint64)
            sc = np.zeros(max(k, 1))
            sn = np.zeros(max(k, 1))
        else:
            import torch

            coefs = coefs.reshape(-1, len(dets)).contiguous()
            sel = torch.zeros((max(k, 1), 2, self.nint), dtype=torch.int64, device=dets.device)
            sc = torch.zeros(max(k, 1), dtype=torch.float64, device=dets.device)
            sn = torch.zeros(max(k, 1), dtype=torch.float64, device=dets.device)
        rc, res = qp_pt2_eval_states(self.ctx, len(dets), dets, coefs, e0, k, sel if k else None,
                                     sc if k else None, sn if k else None, check=check)
        out = res[0].as_dict()
        out["rc"] = rc
        out["e_pt2_states"] = np.array([r.e_pt2 for r in res])
        out["sum_e_over_d_states"] = np.array([r.sum_e_over_d for r in res])
        m = res[0].n_selected
        out.update(sel_dets=sel[:m], sel_crit=sc[:m], sel_num=sn[:m])
        out["launches"] = qp_pt2_last_launches(self.ctx)
        return out

    def eval_generators(self, dets, coefs, e0, ranks, k=0):
        """Sweep of the generators of the listed ranks (0 = largest c_I^2):
        their eps_I, |A_I| and connections (host arrays, list order), the
        totals over them and, with k > 0, the best k of their perturbers
        (in the memory kind of ``dets``)."""
        ranks = np.ascontiguousarray(ranks, dtype=np.int32)
        n = len(ranks)
        eps = np.zeros(max(n, 1))
        s2 = np.zeros(max(n, 1))
        na = np.zeros(max(n, 1), dtype=np.int64)
        nc = np.zeros(max(n, 1), dtype=np.int64)
        if isinstance(dets, np.ndarray):
            sel = np.zeros((max(k, 1), 2, self.nint), dtype=np.uint64)
            se = np.zeros(max(k, 1))
        else:
            import torch

            sel = torch.zeros((max(k, 1), 2, self.nint), dtype=torch.int64, device=dets.device)
            se = torch.zeros(max(k, 1), dtype=torch.float64, device=dets.device)
        _, res = qp_pt2_eval_gens(self.ctx, len(dets), dets, coefs, e0, ranks, k, sel if k else None,
                                  se if k else None, eps, na, nc, gen_s2=s2)
        out = res.as_dict()
        m = res.n_selected
        out.update(eps=eps[:n], s2=s2[:n], na=na[:n], ncon=nc[:n], sel_dets=sel[:m], sel_e=se[:m])
        return out

    def reduce_ranks(self, eps, s2, na, ncon, e0):
        """E_PT2, sum A^2/D^2, counts, Z and E_rPT2 from per-rank arrays,
        reduced exactly as a whole sweep reduces them (qp_pt2_reduce_ranks)."""
        arrs = [np.ascontiguousarray(a, dtype=t) for a, t in
                ((eps, np.float64), (s2, np.float64), (na, np.int64), (ncon, np.int64))]
        res = Result()
        _check(load().qp_pt2_reduce_ranks(self.ctx, len(arrs[0]), *[_ptr(a) for a in arrs], float(e0),
                                          C.byref(res)))
        return res.as_dict()


def pt2_energy(h, eri, dets, coefs, e0, n_alpha, n_beta, stream=None):
    """E_PT2 as a differentiable function of the integrals (and of E0).

    h: CUDA tensor [norb, norb] (symmetric), eri: CUDA tensor of packed
    integrals, dets / coefs: CUDA tensors, e0: 0-d tensor or float.  The
    backward pass calls qp_pt2_grad, which recomputes every matrix element
    (Psi0's coefficients are held fixed).  The gradient returned for h is the
    symmetric one described in include/qp_pt2.h."""
    import torch

    class _PT2Energy(torch.autograd.Function):
        @staticmethod
        def forward(ctx, h_, eri_, e0_):
            norb = h_.shape[0]
            pt2 = PT2(norb, n_alpha, n_beta, h_.detach().contiguous(), eri_.detach().contiguous(), stream=stream)
            ctx.pt2 = pt2
            ctx.e0 = float(e0_)
            res = pt2.eval(dets, coefs, ctx.e0, 0)
            return torch.tensor(res["e_pt2"], dtype=torch.float64, device=h_.device)

        @staticmethod
        def backward(ctx, gout):
            pt2 = ctx.pt2
            dh = torch.zeros((pt2.norb, pt2.norb), dtype=torch.float64, device=gout.device)
            deri = torch.zeros_like(eri)
            de0, _ = qp_pt2_grad(pt2.ctx, len(dets), dets, coefs, ctx.e0, dh, deri)
            pt2.close()
            return gout * dh, gout * deri, gout * de0

    if not torch.is_tensor(e0):
        e0 = torch.tensor(float(e0), dtype=torch.float64, device=h.device)
    return _PT2Energy.apply(h, eri, e0)


class BatchOptions(C.Structure):
    _fields_ = [("fused", C.c_int), ("max_streams", C.c_int), ("work_chunk", C.c_int), ("tile", C.c_int),
                ("blocks_per_sm", C.c_int), ("wave_gb", C.c_double)]


class Batch:
    """Many independent sweeps captured into one CUDA graph (see
    qp_pt2_batch_create_ex in include/qp_pt2.h).

    instances: list of dicts with keys pt2 (a PT2 context), dets, coefs (CUDA
    tensors), e0 (float), k (int).  Output tensors are allocated here.
    fused=True: one persistent launch per wave over all instances of a word
    count and precision, with work_chunk items per draw of its queue, tile
    row tiles applied to every instance (0: each context's own) and
    blocks_per_sm CTAs per SM (0: as many as fit); fused=False: each
    instance's own launches on up to max_streams streams, with grid[i]
    persistent CTAs (None: the context's default)."""

    def __init__(self, instances, grid=None, max_streams=0, stream=None, fused=True, work_chunk=0, tile=0,
                 blocks_per_sm=0, wave_gb=0.0):
        import torch

        L = load()
        n = len(instances)
        self.instances = instances
        self.sel, self.sel_e = [], []
        for inst in instances:
            k = inst["k"]
            dev = inst["dets"].device
            self.sel.append(torch.zeros((max(k, 1), 2, inst["pt2"].nint), dtype=torch.int64, device=dev))
            self.sel_e.append(torch.zeros(max(k, 1), dtype=torch.float64, device=dev))
        VP = C.c_void_p * n
        ctxs = VP(*[inst["pt2"].ctx.value for inst in instances])
        ndet = (C.c_int64 * n)(*[len(inst["dets"]) for inst in instances])
        dets = VP(*[inst["dets"].data_ptr() for inst in instances])
        coefs = VP(*[inst["coefs"].data_ptr() for inst in instances])
        e0 = (C.c_double * n)(*[float(inst["e0"]) for inst in instances])
        ks = (C.c_int64 * n)(*[inst["k"] for inst in instances])
        sel = VP(*[t.data_ptr() for t in self.sel])
        se = VP(*[t.data_ptr() for t in self.sel_e])
        g = (C.c_int * n)(*(grid or [0] * n))
        opt = BatchOptions(int(bool(fused)), int(max_streams), int(work_chunk), int(tile), int(blocks_per_sm),
                           float(wave_gb))
        self.options = {"fused": bool(fused), "max_streams": max_streams, "work_chunk": work_chunk, "tile": tile,
                        "blocks_per_sm": blocks_per_sm, "wave_gb": wave_gb}
        self._keep = (ctxs, ndet, dets, coefs, e0, ks, sel, se, g, opt)
        L.qp_pt2_batch_create_ex.restype = C.c_int
        L.qp_pt2_batch_create_ex.argtypes = [C.POINTER(C.c_void_p), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.POINTER(BatchOptions), C.c_void_p]
        L.qp_pt2_batch_run.restype = C.c_int
        L.qp_pt2_batch_run.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(C.c_double)]
        L.qp_pt2_batch_destroy.restype = None
        L.qp_pt2_batch_destroy.argtypes = [C.c_void_p]
        self.handle = C.c_void_p()
        _check(L.qp_pt2_batch_create_ex(C.byref(self.handle), n, ctxs, ndet, dets, coefs, e0, ks, sel, se, g,
                                        C.byref(opt), stream or None))

    def run(self):
        """Run the graph once: (list of result dicts, device ms)."""
        n = len(self.instances)
        res = (Result * n)()
        ms = C.c_double()
        _check(load().qp_pt2_batch_run(self.handle, res, C.byref(ms)))
        out = []
        for i in range(n):
            d = res[i].as_dict()
            m = d["n_selected"]
            d.update(sel_dets=self.sel[i][:m], sel_e=self.sel_e[i][:m])
            out.append(d)
        return out, ms.value

    def close(self):
        if getattr(self, "handle", None) and _lib is not None:
            _lib.qp_pt2_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        self.close()
