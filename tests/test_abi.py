"""CPU checks of the C ABI: the library builds for sm_103a, loads, exports
every function include/gs2.h declares, and its host-side validation rejects
bad matrices before touching a GPU."""
import ctypes
import os
import re

import numpy as np
import pytest

import paper_2104_01196_gb300 as gs2
from paper_2104_01196_gb300 import build as B
from paper_2104_01196_gb300 import problems as P

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    B.build()
    return gs2.load()


def declared_functions():
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not hdr.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", hdr)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*"
                            r"([a-z][a-z0-9_]*)\s*\(", src, flags=re.M)
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for f in ("gs2_setup", "gs2_apply", "gs_apply", "jr_apply", "gmres_solve",
              "gs2_batch_solve", "gs2_destroy", "gs2_last_error"):
        assert f in names


def test_library_exports_every_declared_symbol(lib):
    missing = [f for f in declared_functions() if not hasattr(lib, f)]
    assert not missing, missing


def test_library_targets_sm103a():
    assert "arch=compute_103a,code=sm_103a" in " ".join(B.NVCC_FLAGS)


def test_version_string(lib):
    assert b"sm_103a" in lib.gs2_version()


def _setup_status(lib, A):
    rp, ci, va = (np.ascontiguousarray(A[0], np.int64), np.ascontiguousarray(A[1], np.int32),
                  np.ascontiguousarray(A[2], np.float64))
    out = ctypes.c_void_p()
    st = lib.gs2_setup(len(rp) - 1, int(rp[-1]), rp.ctypes.data, ci.ctypes.data,
                       va.ctypes.data, 0, 0, None, ctypes.byref(out))
    return st, lib.gs2_last_error().decode()


def test_setup_rejects_zero_and_missing_diagonal(lib):
    M = np.array([[2.0, 1.0], [1.0, 0.0]])
    st, msg = _setup_status(lib, P.dense_to_csr(M, keep_zero_diag=True))
    assert st == 2 and "diagonal" in msg
    A = (np.array([0, 1, 2]), np.array([0, 0]), np.array([1.0, 1.0]))
    st, _ = _setup_status(lib, A)
    assert st == 2


def test_setup_rejects_bad_structure(lib):
    # duplicate entry
    st, msg = _setup_status(lib, (np.array([0, 2, 3]), np.array([0, 0, 1]),
                                  np.array([1.0, 1.0, 1.0])))
    assert st == 1 and "duplicate" in msg
    # column out of range
    st, msg = _setup_status(lib, (np.array([0, 1, 2]), np.array([0, 5]), np.array([1.0, 1.0])))
    assert st == 1 and "range" in msg
    # non-monotone rowptr / wrong nnz
    st, _ = _setup_status(lib, (np.array([0, 2, 1]), np.array([0, 1]), np.array([1.0, 1.0])))
    assert st == 1
    st, _ = _setup_status(lib, (np.array([1, 1, 2]), np.array([0, 1]), np.array([1.0, 1.0])))
    assert st == 1


def test_setup_reports_the_first_bad_row_of_a_large_matrix(lib):
    """Validation runs on several host threads over row ranges; the error
    reported is still the one of the first bad row."""
    n = 300_000
    rp = np.arange(n + 1, dtype=np.int64)
    ci = np.arange(n, dtype=np.int32)
    va = np.ones(n)
    bad = ci.copy()
    bad[250_000] = 7          # row 250000 loses its diagonal
    bad[280_000] = n + 5      # row 280000: column out of range
    st, msg = _setup_status(lib, (rp, bad, va))
    assert st == 2 and msg.endswith("row 250000")
    bad[200_001] = -1         # an earlier row, out of range
    st, msg = _setup_status(lib, (rp, bad, va))
    assert st == 1 and "range" in msg and msg.endswith("row 200001")
    # a long row with a duplicate (the sorted check) before it all
    rp2 = np.concatenate([[0, 40], 40 + np.arange(1, n)]).astype(np.int64)
    ci2 = np.concatenate([np.arange(40), np.arange(1, n)]).astype(np.int32)
    ci2[39] = 3
    st, msg = _setup_status(lib, (rp2, ci2, np.ones(len(ci2))))
    assert st == 1 and "duplicate" in msg and msg.endswith("row 0")


def test_null_arguments_are_rejected(lib):
    assert lib.gs2_apply(None, None, None, 1, 1, 1.0, 0) != 0
    assert lib.gmres_solve(None, None, None, 30, 1e-8, 10, None, None) != 0
    lib.gs2_destroy(None)  # no-op


def test_binding_fails_loudly_without_library(tmp_path):
    saved = gs2._lib
    try:
        gs2._lib = None
        with pytest.raises(RuntimeError, match="missing"):
            gs2.load(str(tmp_path / "nope.so"))
    finally:
        gs2._lib = saved
