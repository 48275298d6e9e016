"""Plain FP64 CPU oracle for the EN-PT2 + CIPSI selection sweep.

TEST INFRASTRUCTURE ONLY: the test suite, the smoke check and the benchmark's
CPU-baseline leg are the only code that may import this package.  The product
library (``paper_1902_08154_gb300``) never imports it, and the two share no
code other than the seeded input generator.

``build()`` compiles ``pt2_oracle.c`` with gcc (OpenMP) into
``oracle/_build/libpt2_oracle.so``; every other function here is a thin
ctypes wrapper or plain numpy.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD_DIR = os.path.join(HERE, "_build")
SO = os.path.join(BUILD_DIR, "libpt2_oracle.so")
SRC = os.path.join(HERE, "pt2_oracle.c")

_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle library (a few seconds)."""
    os.makedirs(BUILD_DIR, exist_ok=True)
    if force or not os.path.exists(SO) or os.path.getmtime(SO) < os.path.getmtime(SRC):
        tmp = SO + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fopenmp", "-fPIC", "-shared", SRC, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, SO)
    return SO


class Result(C.Structure):
    _fields_ = [
        ("e_pt2", C.c_double),
        ("sum_e_over_d", C.c_double),
        ("min_abs_den", C.c_double),
        ("n_perturbers", C.c_int64),
        ("n_connections", C.c_int64),
        ("n_selected", C.c_int64),
        ("n_tiny", C.c_int64),
        ("digest", C.c_uint64 * 2),
    ]

    def as_dict(self):
        return {
            "e_pt2": self.e_pt2,
            "sum_e_over_d": self.sum_e_over_d,
            "min_abs_den": self.min_abs_den,
            "n_perturbers": self.n_perturbers,
            "n_connections": self.n_connections,
            "n_selected": self.n_selected,
            "n_tiny": self.n_tiny,
            "digest": (int(self.digest[0]), int(self.digest[1])),
        }


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(SO)
        P, D, I64, I, U64P, DP, I64P = C.c_void_p, C.c_double, C.c_int64, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p
        L.or_ham_new.restype = P
        L.or_ham_new.argtypes = [I, I, I, DP, DP]
        L.or_ham_free.argtypes = [P]
        L.or_eri.restype = D
        L.or_eri.argtypes = [P, I, I, I, I]
        L.or_hij.restype = D
        L.or_hij.argtypes = [P, U64P, U64P]
        L.or_diag.restype = D
        L.or_diag.argtypes = [P, U64P]
        L.or_degree.restype = I
        L.or_degree.argtypes = [I, U64P, U64P]
        L.or_n_substitutions.restype = I64
        L.or_n_substitutions.argtypes = [P]
        L.or_substitutions.restype = I64
        L.or_substitutions.argtypes = [P, U64P, I64, U64P]
        L.or_key_hash.restype = C.c_uint64
        L.or_key_hash.argtypes = [I, U64P]
        L.or_ranks.argtypes = [I64, DP, I64P]
        L.or_validate.restype = I
        L.or_validate.argtypes = [P, I64, U64P]
        L.or_sweep.restype = I
        L.or_sweep.argtypes = [P, I64, U64P, DP, D, I64, U64P, DP, DP, DP, I64P, I64P, I64P,
                               C.POINTER(Result), I, I64]
        L.or_generator.restype = I
        L.or_generator.argtypes = [P, I64, U64P, DP, D, I64, DP, I64P, I64P, DP, U64P, I64, U64P, DP, I]
        L.or_alpha.restype = I
        L.or_alpha.argtypes = [P, I64, U64P, DP, U64P, DP, DP, I64P, I64P]
        L.or_hamiltonian.restype = I64
        L.or_hamiltonian.argtypes = [P, I64, U64P, I64, I64P, I64P, DP, I]
        L.or_gradient.restype = I
        L.or_gradient.argtypes = [P, I64, U64P, DP, D, DP, DP, DP, DP, I, I64]
        L.or_states.restype = I
        L.or_states.argtypes = [P, I64, U64P, I, DP, DP, I64, U64P, DP, DP, DP, DP, C.c_void_p, I, I, I]
        L.or_max_threads.restype = I
        L.or_set_target.restype = None
        L.or_set_target.argtypes = [P, I, U64P, I, U64P, U64P]
        _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class Hamiltonian:
    """Owns an oracle copy of (h, eri) for a given (norb, nalpha, nbeta)."""

    def __init__(self, norb, nalpha, nbeta, h, eri):
        self.norb, self.nalpha, self.nbeta = norb, nalpha, nbeta
        self.nint = (norb - 1) // 64 + 1
        self.h = np.ascontiguousarray(h, dtype=np.float64)
        self.eri = np.ascontiguousarray(eri, dtype=np.float64)
        self._p = lib().or_ham_new(norb, nalpha, nbeta, _ptr(self.h), _ptr(self.eri))
        if not self._p:
            raise ValueError("bad Hamiltonian sizes")

    def __del__(self):
        if getattr(self, "_p", None) and _lib is not None:
            _lib.or_ham_free(self._p)
            self._p = None

    def _det(self, d):
        d = np.ascontiguousarray(d, dtype=np.uint64)
        assert d.shape == (2, self.nint), d.shape
        return d

    def set_target(self, ref=None, max_exc=-1, core=None, deleted=None):
        """Restrict the external space to a target space (CISD-like with ref
        and max_exc, CAS-like with core/deleted masks in determinant
        layout); all None clears it."""
        on = int(ref is not None or core is not None or deleted is not None)
        arrs = [None if a is None else self._det(a) for a in (ref, core, deleted)]
        self._tgt = arrs  # keep alive
        lib().or_set_target(self._p, on, _ptr(arrs[0]), int(max_exc), _ptr(arrs[1]), _ptr(arrs[2]))

    def eri_value(self, p, q, r, s):
        return lib().or_eri(self._p, p, q, r, s)

    def hij(self, a, b):
        a, b = self._det(a), self._det(b)
        return lib().or_hij(self._p, _ptr(a), _ptr(b))

    def diag(self, d):
        d = self._det(d)
        return lib().or_diag(self._p, _ptr(d))

    def degree(self, a, b):
        a, b = self._det(a), self._det(b)
        return lib().or_degree(self.nint, _ptr(a), _ptr(b))

    def substitutions(self, d):
        d = self._det(d)
        n = lib().or_n_substitutions(self._p)
        out = np.zeros((n, 2, self.nint), dtype=np.uint64)
        m = lib().or_substitutions(self._p, _ptr(d), n, _ptr(out))
        assert m == n
        return out

    def validate(self, dets):
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        return lib().or_validate(self._p, len(dets), _ptr(dets))

    def sweep(self, dets, coefs, e0, k, nthreads=0, mem_budget=0, per_generator=True):
        """Plain-definition sweep.  Returns a dict (see ``Result``) plus the
        selection and, if asked, per-generator arrays indexed by rank."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        n = len(dets)
        sel = np.zeros((max(k, 0), 2, self.nint), dtype=np.uint64)
        sel_e = np.zeros(max(k, 0))
        sel_num = np.zeros(max(k, 0))
        eps = np.zeros(n) if per_generator else None
        na = np.zeros(n, dtype=np.int64) if per_generator else None
        nc = np.zeros(n, dtype=np.int64) if per_generator else None
        rank_of = np.zeros(n, dtype=np.int64)
        res = Result()
        rc = lib().or_sweep(self._p, n, _ptr(dets), _ptr(coefs), float(e0), int(k), _ptr(sel),
                            _ptr(sel_e), _ptr(sel_num), _ptr(eps), _ptr(na), _ptr(nc), _ptr(rank_of),
                            C.byref(res), int(nthreads), int(mem_budget))
        if rc != 0:
            raise ValueError(f"oracle sweep rejected its input (code {rc})")
        out = res.as_dict()
        m = res.n_selected
        out.update(sel_dets=sel[:m], sel_e=sel_e[:m], sel_num=sel_num[:m], rank_of=rank_of,
                   eps_by_rank=eps, na_by_rank=na, ncon_by_rank=nc)
        return out

    def generator(self, dets, coefs, e0, g, cap=0, nthreads=0):
        """Per-generator definition for the generator of rank g."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        eps = np.zeros(1)
        s2 = np.zeros(1)
        na = np.zeros(1, dtype=np.int64)
        nc = np.zeros(1, dtype=np.int64)
        dg = np.zeros(2, dtype=np.uint64)
        out_d = np.zeros((max(cap, 1), 2, self.nint), dtype=np.uint64)
        out_e = np.zeros(max(cap, 1))
        rc = lib().or_generator(self._p, len(dets), _ptr(dets), _ptr(coefs), float(e0), int(g),
                                _ptr(eps), _ptr(na), _ptr(nc), _ptr(s2), _ptr(dg), int(cap),
                                _ptr(out_d), _ptr(out_e), int(nthreads))
        if rc != 0:
            raise ValueError(f"oracle generator rejected its input (code {rc})")
        m = min(int(na[0]), cap)
        return {"eps": float(eps[0]), "n_perturbers": int(na[0]), "n_connections": int(nc[0]),
                "sum_e_over_d": float(s2[0]), "digest": (int(dg[0]), int(dg[1])),
                "dets": out_d[:m], "e": out_e[:m]}

    def alpha(self, dets, coefs, alpha):
        """A_alpha, H_aa, internal flag, lowest connected rank and connection count."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        a = self._det(alpha)
        A = np.zeros(1)
        haa = np.zeros(1)
        g = np.zeros(1, dtype=np.int64)
        nc = np.zeros(1, dtype=np.int64)
        internal = lib().or_alpha(self._p, len(dets), _ptr(dets), _ptr(coefs), _ptr(a), _ptr(A),
                                  _ptr(haa), _ptr(g), _ptr(nc))
        return {"A": float(A[0]), "haa": float(haa[0]), "internal": bool(internal),
                "gen_rank": int(g[0]), "n_connections": int(nc[0])}

    def states(self, dets, coefs, e0, k, nthreads=0, shard=(0, 0)):
        """Several states: ``coefs`` [nst][ndet], ``e0`` [nst].  Per-state
        E_PT2 and sum A^2/D^2, the shared counts and digest, and the k best
        determinants by the multi-state criterion (``sel_crit``) with A of
        state 0 (``sel_num``).  ``shard`` = (index, count) keeps the
        perturbers of the generators of rank index mod count."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        coefs = np.ascontiguousarray(np.atleast_2d(coefs), dtype=np.float64)
        e0 = np.ascontiguousarray(np.atleast_1d(e0), dtype=np.float64)
        nst = coefs.shape[0]
        if coefs.shape[1] != len(dets) or len(e0) != nst:
            raise ValueError("coefs must be [nst][ndet] and e0 [nst]")
        sel = np.zeros((max(k, 1), 2, self.nint), dtype=np.uint64)
        crit = np.zeros(max(k, 1))
        num = np.zeros(max(k, 1))
        ept2 = np.zeros(nst)
        s2 = np.zeros(nst)
        res = Result()
        rc = lib().or_states(self._p, len(dets), _ptr(dets), nst, _ptr(coefs), _ptr(e0), int(k), _ptr(sel),
                             _ptr(crit), _ptr(num), _ptr(ept2), _ptr(s2), C.byref(res), int(nthreads),
                             int(shard[0]), int(shard[1]))
        if rc != 0:
            raise ValueError(f"oracle states rejected its input (code {rc})")
        out = res.as_dict()
        m = res.n_selected
        out.update(e_pt2_states=ept2, sum_e_over_d_states=s2, sel_dets=sel[:m], sel_crit=crit[:m],
                   sel_num=num[:m])
        return out

    def gradient(self, dets, coefs, e0, nthreads=0, mem_budget=0):
        """dE_PT2/dh (symmetric, halves off the diagonal), dE_PT2/d(packed
        eri), dE_PT2/dE0 and E_PT2, with Psi0 and E0 held fixed."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        coefs = np.ascontiguousarray(coefs, dtype=np.float64)
        dh = np.zeros((self.norb, self.norb))
        deri = np.zeros(len(self.eri))
        de0 = np.zeros(1)
        e = np.zeros(1)
        rc = lib().or_gradient(self._p, len(dets), _ptr(dets), _ptr(coefs), float(e0), _ptr(dh), _ptr(deri),
                               _ptr(de0), _ptr(e), int(nthreads), int(mem_budget))
        if rc != 0:
            raise ValueError(f"oracle gradient rejected its input (code {rc})")
        return {"dh": dh, "deri": deri, "de0": float(de0[0]), "e_pt2": float(e[0])}

    def hamiltonian_coo(self, dets, nthreads=0):
        """Upper triangle (diagonal included) of H over ``dets``."""
        dets = np.ascontiguousarray(dets, dtype=np.uint64)
        n = len(dets)
        nnz = lib().or_hamiltonian(self._p, n, _ptr(dets), 0, None, None, None, int(nthreads))
        r = np.zeros(nnz, dtype=np.int64)
        c = np.zeros(nnz, dtype=np.int64)
        v = np.zeros(nnz)
        lib().or_hamiltonian(self._p, n, _ptr(dets), nnz, _ptr(r), _ptr(c), _ptr(v), int(nthreads))
        return r, c, v


def ranks(coefs):
    coefs = np.ascontiguousarray(coefs, dtype=np.float64)
    out = np.zeros(len(coefs), dtype=np.int64)
    lib().or_ranks(len(coefs), _ptr(coefs), _ptr(out))
    return out


def key_hash(det):
    d = np.ascontiguousarray(det, dtype=np.uint64)
    return int(lib().or_key_hash(d.size, _ptr(d)))


def max_threads():
    return int(lib().or_max_threads())
