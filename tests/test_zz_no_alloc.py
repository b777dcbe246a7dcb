"""The no-allocation entry point, gs2_apply_noalloc, through the C ABI.

Callers that cannot allocate device memory (their host application owns
all of it, or they must not allocate after start-up) use this entry point:
they pass device pointers to their matrix and vectors, and the library's
working memory is a fixed array in its own device image.  This file checks
it against the ordinary entry point gs2_apply on two calls in a row (the
array keeps the previous call's contents, so the second call must not
depend on them), against the FP64 oracle for every inner-sweep count and
direction and at the documented size limit, and that too large a system
and out-of-range arguments are refused.

Kept in a file of its own, collected last, so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2104_01196_gb300 import problems as P

pytestmark = pytest.mark.gpu
TOL = 1e-12
MAX_ROWS = 262144


@pytest.fixture(scope="module")
def lib():
    import torch  # noqa: F401

    from paper_2104_01196_gb300 import build as B
    B.build()
    import paper_2104_01196_gb300 as gs2
    L = gs2.load()
    L.gs2_apply_noalloc.argtypes = [ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p,
                                    ctypes.c_int, ctypes.c_int, ctypes.c_double, ctypes.c_int,
                                    ctypes.c_void_p]
    L.gs2_apply_noalloc.restype = ctypes.c_int
    return L


def _dev(a, dtype):
    import torch
    return torch.from_numpy(np.ascontiguousarray(a, dtype=dtype)).cuda()


def _noalloc(lib, A, b, x0, outer, inner, omega, direction):
    import torch
    rp, ci, va = (_dev(A[0], np.int64), _dev(A[1], np.int32), _dev(A[2], np.float64))
    bd, xd = _dev(b, np.float64), _dev(x0, np.float64)
    st = lib.gs2_apply_noalloc(len(A[0]) - 1, rp.data_ptr(), ci.data_ptr(), va.data_ptr(),
                               bd.data_ptr(), xd.data_ptr(), outer, inner, omega, direction,
                               torch.cuda.current_stream().cuda_stream or None)
    assert st == 0, lib.gs2_last_error()
    torch.cuda.synchronize()
    return xd.cpu().numpy()


def _reference(A, b, x0, outer, inner, omega, direction):
    import torch

    import paper_2104_01196_gb300 as gs2
    h = gs2.gs2_setup(A)
    x = _dev(x0, np.float64)
    gs2.gs2_apply(h, _dev(b, np.float64), x, outer, inner, omega, direction)
    torch.cuda.synchronize()
    out = x.cpu().numpy()
    h.close()
    return out


def _rel(a, b):
    return np.linalg.norm(a - b) / np.linalg.norm(b)


def test_noalloc_matches_gs2_apply_on_two_calls_in_a_row(lib):
    # first call: a 3D Laplacian, symmetric GS2(2, 2), omega 0.9
    A1 = P.poisson3d_matrix(24)
    b1, x1 = P.uniform_pm1(101, 24 ** 3), P.uniform_pm1(102, 24 ** 3)
    got1 = _noalloc(lib, A1, b1, x1, 2, 2, 0.9, 2)
    assert _rel(got1, _reference(A1, b1, x1, 2, 2, 0.9, 2)) <= TOL
    # second call, straight after: a different, smaller, nonsymmetric matrix
    # with unsorted columns, forward GS2(1, 3); stale scratch must not leak in
    A2 = P.random_csr(5000, 7, mean_offdiag=6.0)
    b2, x2 = P.uniform_pm1(103, 5000), P.uniform_pm1(104, 5000)
    got2 = _noalloc(lib, A2, b2, x2, 1, 3, 1.0, 0)
    assert _rel(got2, _reference(A2, b2, x2, 1, 3, 1.0, 0)) <= TOL


MATS = {"poisson3d_16": P.poisson3d_matrix(16),
        "random_3000": P.random_csr(3000, 17, mean_offdiag=5.0)}


@pytest.mark.parametrize("name", list(MATS))
@pytest.mark.parametrize("inner", [0, 1, 2, 3])
@pytest.mark.parametrize("direction", [0, 1, 2])
def test_noalloc_matches_oracle_and_gs2_apply(lib, name, inner, direction):
    """Every inner-sweep count (0: the update alone; 1: the last sweep reads
    r-hat) and direction (backward alone runs only the upper triangle),
    against the FP64 oracle and the handle-based entry point."""
    A = MATS[name]
    n = len(A[0]) - 1
    b, x0 = P.uniform_pm1(200 + inner, n), P.uniform_pm1(300 + direction, n)
    got = _noalloc(lib, A, b, x0, 2, inner, 0.85, direction)
    assert _rel(got, oracle.gs2(A, b, x0, 2, inner, 0.85, 1.0, direction)) <= TOL
    assert _rel(got, _reference(A, b, x0, 2, inner, 0.85, direction)) <= TOL


def test_noalloc_at_the_size_limit_matches_oracle(lib):
    """n = 262,144 (64^3) exactly: the four slices of the array are full and
    abut; a symmetric sweep with two inner sweeps uses all of them."""
    A = P.poisson3d_matrix(64)
    assert len(A[0]) - 1 == MAX_ROWS
    b, x0 = P.uniform_pm1(401, MAX_ROWS), P.uniform_pm1(402, MAX_ROWS)
    got = _noalloc(lib, A, b, x0, 1, 2, 1.0, 2)
    assert _rel(got, oracle.gs2(A, b, x0, 1, 2, 1.0, 1.0, oracle.SYMMETRIC)) <= TOL


def test_noalloc_sums_duplicate_diagonal_entries(lib):
    """A row whose diagonal is stored as two entries: D is their sum, as the
    oracle (and an SpMV) takes it."""
    M = P.csr_to_dense(P.poisson3d_matrix(6))
    rp, ci, va = P.dense_to_csr(M)
    rows = [[(int(c), float(v)) for c, v in zip(ci[rp[i]:rp[i + 1]], va[rp[i]:rp[i + 1]])]
            for i in range(len(rp) - 1)]
    for i in (0, 17, 100):  # split the diagonal 6 into 2.5 + 3.5
        rows[i] = [(c, v) for c, v in rows[i] if c != i] + [(i, 2.5), (i, 3.5)]
    rp2 = np.cumsum([0] + [len(r) for r in rows]).astype(np.int64)
    ci2 = np.array([c for r in rows for c, _ in r], np.int32)
    va2 = np.array([v for r in rows for _, v in r])
    A = (rp2, ci2, va2)
    n = len(rp2) - 1
    b, x0 = P.uniform_pm1(501, n), P.uniform_pm1(502, n)
    got = _noalloc(lib, A, b, x0, 1, 2, 1.0, 2)
    assert _rel(got, oracle.gs2(A, b, x0, 1, 2, 1.0, 1.0, oracle.SYMMETRIC)) <= TOL


def test_noalloc_refuses_systems_above_its_limit(lib):
    st = lib.gs2_apply_noalloc(MAX_ROWS + 1, 1, 1, 1, 1, 1, 1, 1, 1.0, 0, None)
    assert st == 1
    assert b"no-allocation limit" in lib.gs2_last_error()


@pytest.mark.parametrize("outer,inner,damping,direction", [
    (1, 1, float("inf"), 0), (1, 1, float("nan"), 0), (1, 1, 0.0, 0),
    (1001, 1, 1.0, 0), (1, 100001, 1.0, 0), (-1, 1, 1.0, 0), (1, 1, 1.0, 3)])
def test_noalloc_refuses_out_of_range_arguments(lib, outer, inner, damping, direction):
    """The bounds gs2_apply enforces; nothing is launched (the pointers are
    never touched when the arguments are refused)."""
    st = lib.gs2_apply_noalloc(100, 1, 1, 1, 1, 1, outer, inner, damping, direction, None)
    assert st == 1
