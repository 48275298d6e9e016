"""qp_pt2_eval_noalloc against qp_pt2_eval (GPU).

The no-allocation entry point serves callers that cannot call cudaMalloc or
cudaFree -- for instance a host program that reserves all of the GPU's
memory up front and gives its plugins no allocator.  It keeps its scratch in
one fixed device array inside the library, which every call reuses.  Two
calls in a row must each give what the ordinary entry point gives on the
same inputs (same exact counts and perturber digest, energies within the
suite's 1e-10 Eh, same selection), which also shows that the leftovers of
the first call do not leak into the second.

This file is named so that pytest collects it after every other test file.
"""
import numpy as np
import pytest

from paper_1902_08154_gb300 import synthetic as S
from tests.parity_util import check_selection, check_totals

pytestmark = pytest.mark.gpu


def _dev(a):
    import torch

    if a.dtype == np.uint64:
        a = a.view(np.int64)
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


# The last case needs several waves of generator slots inside the fixed
# array: one slot of 64 orbitals, 10+10 electrons and 1000 determinants holds
# 1000 coarse-filter records (44 bytes each) and up to 6000 bucket entries
# (20 bytes each), about 164 KB, so the 64 MiB array holds fewer than 410
# slots for the 1000 generators.
@pytest.mark.parametrize("norb,na,nb,ndet,k,seed", [(16, 4, 4, 300, 200, 71), (70, 3, 3, 80, 50, 72),
                                                    (64, 10, 10, 1000, 1000, 76)])
def test_noalloc_matches_eval_twice(norb, na, nb, ndet, k, seed):
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    from paper_1902_08154_gb300 import build

    build.build()
    import paper_1902_08154_gb300 as qp

    h, eri = S.hamiltonian(norb, norb + 2, seed)
    dets = S.random_excited_dets(norb, na, nb, ndet, seed + 1)
    c = S.random_coefs(len(dets), seed + 2, decay=0.05)
    hd, ed, dd, cd = _dev(h), _dev(eri), _dev(dets), _dev(c)
    # E0 below every internal diagonal energy (as a variational E0 is)
    e0 = float(np.min(np.diag(h))) * (na + nb) - 50.0

    pt2 = qp.PT2(norb, na, nb, hd, ed)
    ref = pt2.eval(dd, cd, e0, k)
    pt2.close()
    assert ref["n_perturbers"] > k

    nint = (norb - 1) // 64 + 1
    for _ in range(2):
        sel = torch.zeros((k, 2, nint), dtype=torch.int64, device="cuda")
        sel_e = torch.zeros(k, dtype=torch.float64, device="cuda")
        rc, res = qp.qp_pt2_eval_noalloc(norb, na, nb, hd, ed, len(dets), dd, cd, e0, k, sel, sel_e)
        torch.cuda.synchronize()
        assert rc == qp.QP_OK, rc
        got = res.as_dict()
        check_totals(got, ref)
        m = got["n_selected"]
        check_selection(sel[:m], sel_e[:m], ref["sel_dets"], ref["sel_e"])


def test_noalloc_refuses_host_memory_and_oversize():
    import torch

    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    import paper_1902_08154_gb300 as qp

    norb, na, nb = 12, 3, 3
    h, eri = S.hamiltonian(norb, 10, 73)
    dets = S.random_excited_dets(norb, na, nb, 20, 74)
    c = S.random_coefs(20, 75)
    # host arrays are refused: the entry point copies nothing
    rc, _ = qp.qp_pt2_eval_noalloc(norb, na, nb, h, eri, 20, dets, c, -10.0, 0)
    assert rc == qp.QP_EINVAL
    assert b"device memory" in qp.load().qp_pt2_last_error()
    # so is page-locked host memory, which the GPU could reach but which is
    # not memory of the current device
    hp = torch.from_numpy(h).pin_memory()
    rc, _ = qp.qp_pt2_eval_noalloc(norb, na, nb, hp, _dev(eri), 20, _dev(dets), _dev(c), -10.0, 0)
    assert rc == qp.QP_EINVAL
    # a selection that cannot fit in the fixed scratch is refused cleanly
    hd, ed, dd, cd = _dev(h), _dev(eri), _dev(dets), _dev(c)
    k = 10**7
    sel = torch.zeros((1, 2, 1), dtype=torch.int64, device="cuda")
    sel_e = torch.zeros(1, dtype=torch.float64, device="cuda")
    rc, _ = qp.qp_pt2_eval_noalloc(norb, na, nb, hd, ed, 20, dd, cd, -10.0, k, sel, sel_e)
    assert rc == qp.QP_EINVAL
    assert b"too large" in qp.load().qp_pt2_last_error()
