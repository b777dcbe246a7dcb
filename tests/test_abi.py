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


def _pack_status(lib, mats):
    cnt = len(mats)
    keep = []
    N = (ctypes.c_int64 * cnt)()
    R, C, V = (ctypes.c_void_p * cnt)(), (ctypes.c_void_p * cnt)(), (ctypes.c_void_p * cnt)()
    for s, (rp, ci, va) in enumerate(mats):
        rp, ci, va = (np.ascontiguousarray(rp, np.int64), np.ascontiguousarray(ci, np.int32),
                      np.ascontiguousarray(va, np.float64))
        keep += [rp, ci, va]
        N[s] = len(rp) - 1
        R[s], C[s], V[s] = rp.ctypes.data, ci.ctypes.data, va.ctypes.data
    out = ctypes.c_void_p()
    st = lib.gs2_pack_setup(cnt, N, R, C, V, 0, None, ctypes.byref(out))
    return st, lib.gs2_last_error().decode()


def test_pack_setup_names_the_bad_system_and_row(lib):
    """A pack is validated per system before any device work: a column of
    system s must lie inside system s (so no entry couples two systems), and
    the errors of the whole-pack checks are reported as (system, its row)."""
    good = P.poisson2d(4).A
    # column 16 is inside the 32-row pack but outside system 1 (16 rows)
    rp, ci, va = (a.copy() for a in good)
    ci[rp[2]] = 16
    st, msg = _pack_status(lib, [good, (rp, ci, va), good])
    assert st == 1 and msg == "system 1: column index out of range in row 2", msg
    # zero diagonal in row 3 of system 2
    rp, ci, va = (a.copy() for a in good)
    va[(ci == 3) & (np.arange(len(ci)) >= rp[3]) & (np.arange(len(ci)) < rp[4])] = 0.0
    st, msg = _pack_status(lib, [good, good, (rp, ci, va)])
    assert st == 2 and msg == "system 2: zero or missing diagonal in row 3", msg
    # duplicate entry in row 0 of system 0
    rp, ci, va = (a.copy() for a in good)
    ci[1] = ci[0]
    st, msg = _pack_status(lib, [(rp, ci, va), good])
    assert st == 1 and msg == "system 0: duplicate entry in row 0", msg
    # rowptr not starting at 0
    st, msg = _pack_status(lib, [good, (good[0] + 1, good[1], good[2])])
    assert st == 1 and msg.startswith("system 1: rowptr[0]")
    out = ctypes.c_void_p()
    assert lib.gs2_pack_setup(0, None, None, None, None, 0, None, ctypes.byref(out)) == 1
    assert lib.gs2_pack_gmres(None, None, None, 30, 1e-8, 10, None, None) != 0
