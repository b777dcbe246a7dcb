"""The no-allocation entry point, gs2_apply_noalloc, through the C ABI.

Callers that cannot allocate device memory (their host application owns
all of it, or they must not allocate after start-up) use this entry point:
they pass device pointers to their matrix and vectors, and the library's
working memory is a fixed array in its own device image.  This file checks
it against the ordinary entry point gs2_apply on two calls in a row (the
array keeps the previous call's contents, so the second call must not
depend on them), and that too large a system is refused.

Kept in a file of its own, collected last, so that a run stopping at the
first failure has already run every other test.
"""
import ctypes

import numpy as np
import pytest

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


def test_noalloc_refuses_systems_above_its_limit(lib):
    st = lib.gs2_apply_noalloc(MAX_ROWS + 1, 1, 1, 1, 1, 1, 1, 1, 1.0, 0, None)
    assert st == 1
    assert b"no-allocation limit" in lib.gs2_last_error()
