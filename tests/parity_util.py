"""Comparison rules between the CUDA sweep and the CPU oracle.

* integer outputs (perturber count, connection counts, per-generator counts,
  perturber-set digest) must match exactly;
* energies must agree within E_TOL = 1e-10 Eh (FP64), per-perturber e_alpha
  within 1e-12 absolute plus 1e-10 relative;
* the selection must hold the same determinants with the same e_alpha,
  except that determinants whose |e_alpha| lies within a relative 1e-9 of
  the k-th value may be exchanged (several answers are then correct), and
  the sequences of e_alpha values must agree position by position.
"""
import numpy as np

E_TOL = 1e-10


def as_np(x, dtype=None):
    if hasattr(x, "detach"):
        x = x.detach().cpu().numpy()
    x = np.asarray(x)
    return x.view(dtype) if dtype is not None else x


def e_close(a, b, abs_tol=1e-12, rel_tol=1e-10):
    return abs(a - b) <= abs_tol + rel_tol * max(abs(a), abs(b))


def check_totals(got, ref, e_tol=E_TOL):
    assert got["n_perturbers"] == ref["n_perturbers"], (got["n_perturbers"], ref["n_perturbers"])
    assert got["n_connections"] == ref["n_connections"], (got["n_connections"], ref["n_connections"])
    assert tuple(got["digest"]) == tuple(int(x) for x in ref["digest"]), "perturber sets differ"
    assert abs(got["e_pt2"] - ref["e_pt2"]) <= e_tol, (got["e_pt2"], ref["e_pt2"])
    s = max(1.0, abs(ref["sum_e_over_d"]))
    assert abs(got["sum_e_over_d"] - ref["sum_e_over_d"]) <= e_tol * s
    if ref["n_perturbers"]:
        assert got["min_abs_den"] == ref["min_abs_den"] or e_close(got["min_abs_den"], ref["min_abs_den"])
    assert got["n_selected"] == ref["n_selected"]


def check_per_generator(got, ref, e_tol=E_TOL):
    assert np.array_equal(as_np(got["na_by_rank"]), as_np(ref["na_by_rank"]))
    assert np.array_equal(as_np(got["ncon_by_rank"]), as_np(ref["ncon_by_rank"]))
    d = np.abs(as_np(got["eps_by_rank"]) - as_np(ref["eps_by_rank"]))
    assert d.max(initial=0.0) <= e_tol, d.max()


def check_selection(got_dets, got_e, ref_dets, ref_e, rel=1e-9):
    ge, re_ = as_np(got_e), as_np(ref_e)
    gd = as_np(got_dets).view(np.uint64)
    rd = as_np(ref_dets).view(np.uint64)
    gd = gd.reshape(len(ge), int(np.prod(gd.shape[1:])))
    rd = rd.reshape(len(re_), int(np.prod(rd.shape[1:])))
    assert len(ge) == len(re_)
    if len(ge) == 0:
        return
    for a, b in zip(ge, re_):
        assert e_close(a, b), (a, b)
    gmap = {r.tobytes(): e for r, e in zip(gd, ge)}
    rmap = {r.tobytes(): e for r, e in zip(rd, re_)}
    kth = abs(re_[-1])
    for key, e in gmap.items():
        if key in rmap:
            assert e_close(e, rmap[key]), (e, rmap[key])
        else:
            assert abs(abs(e) - kth) <= rel * kth + 1e-15, ("selected by the GPU only", e, kth)
    for key, e in rmap.items():
        if key not in gmap:
            assert abs(abs(e) - kth) <= rel * kth + 1e-15, ("selected by the oracle only", e, kth)
    # best-first order
    a = np.abs(ge)
    assert np.all(a[:-1] >= a[1:] * (1 - 1e-12) - 1e-300)


def variational(ham, dets):
    """Lowest eigenpair of H over the determinant set (dense, from the
    oracle's matrix elements): a unit-norm Psi0 with a variational E0, as
    the CIPSI workloads have, for the small random test spaces."""
    n = len(dets)
    H = np.array([[ham.hij(dets[i], dets[j]) for j in range(n)] for i in range(n)])
    w, v = np.linalg.eigh(H)
    c = v[:, 0] * (1.0 if v[0, 0] >= 0 else -1.0)
    return np.ascontiguousarray(c), float(w[0])


def cipsi_space(oracle_mod, ham, norb, na, nb, ndet, doublings=2):
    """A small Psi0 grown by the oracle's CIPSI rule (seed space of
    ndet / 2^doublings determinants, then doublings), with its coefficients
    and variational E0: the shape of the workloads (Sec. "The basic
    algorithm"), at sizes the oracle grows in a fraction of a second."""
    from oracle import psi0

    from paper_1902_08154_gb300 import synthetic as S

    dets, c, e0, _ = psi0.cipsi_grow(ham, S.hf_det(norb, na, nb), ndet, doublings=doublings)
    return np.ascontiguousarray(dets), np.ascontiguousarray(c), float(e0)
