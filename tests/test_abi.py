"""The C ABI library loads here (no GPU needed) and exports every entry point
that include/qp_pt2.h declares."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_1902_08154_gb300 import build

    build.build()
    import paper_1902_08154_gb300 as qp

    return qp.load()


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "qp_pt2.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(qp_pt2_\w+)\s*\(", txt)))


def test_header_declares_the_entry_points():
    names = declared_functions()
    assert "qp_pt2_create" in names and "qp_pt2_eval" in names and "qp_pt2_destroy" in names


def test_library_exports_every_declared_symbol(lib):
    import paper_1902_08154_gb300 as qp

    for name in declared_functions():
        assert hasattr(lib, name), name
        assert isinstance(getattr(lib, name), ctypes._CFuncPtr)
    assert set(qp.EXPORTS) == set(declared_functions())


def test_strerror_without_gpu(lib):
    import paper_1902_08154_gb300 as qp

    assert lib.qp_pt2_strerror(qp.QP_EDUP) == b"duplicate determinant"
    assert lib.qp_pt2_strerror(0) == b"ok"


def test_missing_library_fails_loudly(tmp_path):
    import paper_1902_08154_gb300 as qp

    saved = qp._lib
    qp._lib = None
    try:
        with pytest.raises(ImportError):
            qp.load(str(tmp_path / "absent.so"))
    finally:
        qp._lib = saved
