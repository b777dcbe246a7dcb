"""FP64 CPU oracle for two-stage Gauss-Seidel (GS2), GS/SOR, JR, GMRES and CG.

TEST INFRASTRUCTURE ONLY.  Only the test suite, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package.  The GPU
library never imports it and shares no code with it.

The arithmetic lives in ``oracle.c`` (plain C, one loop per formula of the
paper); this module compiles it with gcc on first use and wraps it with
ctypes.  All arrays are numpy: CSR rowptr int64, col int32, val float64.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_SRCS = [_SRC, os.path.join(_HERE, "amg.c"), os.path.join(_HERE, "hybrid.c"),
         os.path.join(_HERE, "lowprec.c")]
_LIB = os.path.join(_HERE, "liboracle.so")
# the same sources built with -fopenmp: the row loops spread over the host
# cores, bitwise the same results (the multi-core CPU timing)
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_libs = {}

FORWARD, BACKWARD, SYMMETRIC = 0, 1, 2
PC_NONE, PC_GS2, PC_JR, PC_GS, PC_MTGS = 0, 1, 2, 3, 4
PC_HYBRID_GS2, PC_HYBRID_JR, PC_HYBRID_GS = 7, 8, 9
PC_GS2_COMPACT = 10
# inner-sweep precision of GS2 (lowprec.c)
PREC = {"fp64": 0, "fp32": 1, "fp16": 2, "fp32_sweep": 3, "fp16_sweep": 4}


class OracleError(RuntimeError):
    pass


def build(force: bool = False, openmp: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, -O2, no -march);
    with openmp=True into liboracle_omp.so with -fopenmp."""
    lib = _LIB_OMP if openmp else _LIB
    stale = (not os.path.exists(lib)) or (
        os.path.getmtime(lib) < max([os.path.getmtime(f) for f in _SRCS] +
                                    [os.path.getmtime(os.path.join(_HERE, "oracle.h"))]))
    if force or stale:
        tmp = lib + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-ffp-contract=off",
               *(["-fopenmp"] if openmp else []), *_SRCS, "-o", tmp, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, lib)
    return lib


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int),
                ("status", ctypes.c_int), ("true_relres", ctypes.c_double)]


@dataclass
class SolveInfo:
    iters: int
    cycles: int
    status: int
    true_relres: float


def _load(openmp: bool = False):
    with _lock:
        if openmp not in _libs:
            lib = ctypes.CDLL(build(openmp=openmp))
            P = ctypes.c_void_p
            I64, I32, D = ctypes.c_int64, ctypes.c_int, ctypes.c_double
            csr = [I64, P, P, P]
            lib.ora_spmv.argtypes = csr + [P, P]
            lib.ora_spmv.restype = None
            lib.ora_diag.argtypes = csr + [P]
            lib.ora_gs2.argtypes = csr + [P, P, I32, I32, D, D, I32]
            lib.ora_gs.argtypes = csr + [P, P, I32, D, I32]
            lib.ora_jr.argtypes = csr + [P, P, I32, D]
            lib.ora_levels.argtypes = [I64, P, P, I32, P]
            lib.ora_precond.argtypes = csr + [P, P, I32, I32, I32, D, D, I32]
            lib.ora_gmres.argtypes = csr + [P, P, I32, D, I32, I32, I32, I32, D, D,
                                            I32, ctypes.POINTER(_Info), P]
            lib.ora_cg.argtypes = csr + [P, P, D, I32, I32, I32, I32, D, D, I32,
                                         ctypes.POINTER(_Info)]
            lib.ora_gs2_compact.argtypes = csr + [P, P, I32, I32, I32]
            lib.ora_coloring.argtypes = [I64, P, P, P]
            lib.ora_amg_build.argtypes = csr + [D, I32, I64]
            lib.ora_amg_build.restype = P
            lib.ora_amg_free.argtypes = [P]
            lib.ora_amg_free.restype = None
            lib.ora_amg_levels.argtypes = [P]
            lib.ora_amg_level.argtypes = [P, I32, P, P, P]
            lib.ora_amg_get_matrix.argtypes = [P, I32, P, P, P]
            lib.ora_amg_get_prolongator.argtypes = [P, I32, P, P, P]
            lib.ora_amg_get_aggregates.argtypes = [P, I32, P]
            lib.ora_amg_vcycle.argtypes = [P, P, P, I32, I32, I32, D, D, I32]
            lib.ora_gmres_amg.argtypes = csr + [P, P, I32, D, I32, P, I32, I32, I32, D, D,
                                                I32, ctypes.POINTER(_Info)]
            lib.ora_cg_amg.argtypes = csr + [P, P, D, I32, P, I32, I32, I32, D, D, I32,
                                             ctypes.POINTER(_Info)]
            lib.ora_mtgs.argtypes = csr + [P, P, I32, D, I32]
            lib.ora_hybrid.argtypes = csr + [P, P, I32, I32, I32, I32, I32, D, D, I32]
            lib.ora_set_hybrid.argtypes = [I32, I32]
            lib.ora_set_hybrid.restype = None
            lib.ora_threads.argtypes = []
            lib.ora_gs2_lp.argtypes = csr + [P, P, I32, I32, D, D, I32, I32]
            lib.ora_round_half.argtypes = [D]
            lib.ora_round_half.restype = D
            lib.ora_set_precision.argtypes = [I32]
            lib.ora_set_precision.restype = None
            for f in ("ora_diag", "ora_gs2", "ora_gs", "ora_jr", "ora_levels",
                      "ora_precond", "ora_gmres", "ora_cg", "ora_gs2_compact",
                      "ora_coloring", "ora_mtgs", "ora_amg_levels", "ora_amg_level",
                      "ora_amg_get_matrix", "ora_amg_get_prolongator",
                      "ora_amg_get_aggregates", "ora_amg_vcycle", "ora_gmres_amg",
                      "ora_cg_amg", "ora_hybrid", "ora_threads", "ora_gs2_lp"):
                getattr(lib, f).restype = ctypes.c_int
            _libs[openmp] = lib
    return _libs[openmp]


def round_half(v: float) -> float:
    """IEEE binary16 round-to-nearest-even of v (the oracle's own rounding)."""
    return float(_load().ora_round_half(float(v)))


def threads(openmp: bool = False) -> int:
    """Threads the row loops of that build run on."""
    return int(_load(openmp).ora_threads())


def _csr(A):
    rp, ci, va = A
    rp = np.ascontiguousarray(rp, dtype=np.int64)
    ci = np.ascontiguousarray(ci, dtype=np.int32)
    va = np.ascontiguousarray(va, dtype=np.float64)
    n = rp.shape[0] - 1
    return n, rp, ci, va


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _vec(v, n):
    v = np.array(v, dtype=np.float64, copy=True, order="C")
    if v.shape != (n,):
        raise OracleError(f"vector of length {n} expected, got {v.shape}")
    return v


def _check(st, what):
    if st != 0:
        raise OracleError(f"{what} returned status {st}")


def spmv(A, x, openmp=False):
    n, rp, ci, va = _csr(A)
    x = _vec(x, n)
    y = np.empty(n)
    _load(openmp).ora_spmv(n, _p(rp), _p(ci), _p(va), _p(x), _p(y))
    return y


def diag(A):
    n, rp, ci, va = _csr(A)
    d = np.empty(n)
    _check(_load().ora_diag(n, _p(rp), _p(ci), _p(va), _p(d)), "ora_diag")
    return d


def gs2(A, b, x, outer=1, inner=1, omega=1.0, gamma=1.0, direction=FORWARD, openmp=False,
        precision="fp64"):
    """Non-compact GS2 sweeps (Eq. 2-5, damped); returns the new x.  With
    precision "fp32" or "fp16" the inner sweeps run in that precision
    (lowprec.c: FP32 values, or FP16 values with a per-row scale; FP32
    vectors and accumulation; residual and update FP64)."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    if precision != "fp64":
        _check(_load().ora_gs2_lp(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), outer, inner,
                                  omega, gamma, direction, PREC[precision]), "ora_gs2_lp")
        return x
    _check(_load(openmp).ora_gs2(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), outer, inner,
                           omega, gamma, direction), "ora_gs2")
    return x


def gs(A, b, x, sweeps=1, omega=1.0, direction=FORWARD):
    """Exact GS / SOR by the compact row recurrence; returns the new x."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    _check(_load().ora_gs(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), sweeps, omega,
                          direction), "ora_gs")
    return x


def jr(A, b, x, sweeps=1, omega=1.0, openmp=False):
    """Damped Jacobi-Richardson; returns the new x."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    _check(_load(openmp).ora_jr(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), sweeps, omega),
           "ora_jr")
    return x


def levels(A, lower=True):
    """(level per row, number of levels) of the strict lower/upper triangle."""
    n, rp, ci, _ = _csr(A)
    lev = np.zeros(n, dtype=np.int32)
    nlev = _load().ora_levels(n, _p(rp), _p(ci), 1 if lower else 0, _p(lev))
    return lev, int(nlev)


def coloring(A):
    """(colour per row, number of colours): first fit on the symmetrised pattern."""
    n, rp, ci, _ = _csr(A)
    col = np.zeros(n, dtype=np.int32)
    nc = _load().ora_coloring(n, _p(rp), _p(ci), _p(col))
    return col, int(nc)


def mtgs(A, b, x, sweeps=1, omega=1.0, direction=FORWARD):
    """Multicolour GS / SOR (rows colour by colour); returns the new x."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    _check(_load().ora_mtgs(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), sweeps, omega,
                            direction), "ora_mtgs")
    return x


def precond(A, v, kind=PC_GS2, outer=1, inner=1, omega=1.0, gamma=1.0,
            direction=FORWARD):
    """z = M^{-1} v from a zero start."""
    n, rp, ci, va = _csr(A)
    v = _vec(v, n)
    z = np.empty(n)
    _check(_load().ora_precond(n, _p(rp), _p(ci), _p(va), _p(v), _p(z), kind, outer,
                               inner, omega, gamma, direction), "ora_precond")
    return z


def gmres(A, b, x0=None, restart=30, tol=1e-8, max_iters=10000, pc_kind=PC_GS2,
          pc_outer=1, pc_inner=1, pc_omega=1.0, pc_gamma=1.0,
          pc_direction=FORWARD, history=False, pc_parts=1, pc_local=1,
          pc_precision="fp64"):
    """Restarted right-preconditioned GMRES with CGS2.

    Returns (x, SolveInfo[, history]).  A non-converged solve is returned with
    its status rather than raised, so tests can check the status.  The
    hybrid kinds use pc_parts blocks and pc_local local sweeps; the GS2 kind
    runs its inner sweeps in pc_precision ("fp64", "fp32", "fp16").
    """
    _load().ora_set_hybrid(pc_parts, pc_local)
    _load().ora_set_precision(PREC[pc_precision])
    n, rp, ci, va = _csr(A)
    b = _vec(b, n)
    x = np.zeros(n) if x0 is None else _vec(x0, n)
    info = _Info()
    hist = np.full(max(max_iters, 1), np.nan)
    st = _load().ora_gmres(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), restart, tol,
                           max_iters, pc_kind, pc_outer, pc_inner, pc_omega,
                           pc_gamma, pc_direction, ctypes.byref(info),
                           _p(hist) if history else None)
    if st == 1:
        raise OracleError("ora_gmres: invalid argument")
    si = SolveInfo(info.iters, info.cycles, info.status, info.true_relres)
    if history:
        return x, si, hist[: info.iters].copy()
    return x, si


def cg(A, b, x0=None, tol=1e-8, max_iters=10000, pc_kind=PC_GS2, pc_outer=1,
       pc_inner=1, pc_omega=1.0, pc_gamma=1.0, pc_direction=SYMMETRIC, pc_parts=1,
       pc_local=1, pc_precision="fp64"):
    """Preconditioned CG; returns (x, SolveInfo).  The GS2 kind runs its
    inner sweeps in pc_precision ("fp64", "fp32", "fp16")."""
    _load().ora_set_hybrid(pc_parts, pc_local)
    _load().ora_set_precision(PREC[pc_precision])
    n, rp, ci, va = _csr(A)
    b = _vec(b, n)
    x = np.zeros(n) if x0 is None else _vec(x0, n)
    info = _Info()
    st = _load().ora_cg(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, max_iters,
                        pc_kind, pc_outer, pc_inner, pc_omega, pc_gamma,
                        pc_direction, ctypes.byref(info))
    if st == 1:
        raise OracleError("ora_cg: invalid argument")
    return x, SolveInfo(info.iters, info.cycles, info.status, info.true_relres)


def hybrid(A, b, x, kind=PC_GS2, parts=1, outer=1, local=1, inner=1, omega=1.0, gamma=1.0,
           direction=FORWARD):
    """Hybrid (block-Jacobi) relaxation over `parts` contiguous row blocks:
    `outer` exchanges, `local` local sweeps each (kind PC_GS2, PC_JR or
    PC_GS); returns the new x."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    _check(_load().ora_hybrid(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), kind, parts, outer,
                              local, inner, omega, gamma, direction), "ora_hybrid")
    return x


def gs2_compact(A, b, x, outer=1, inner=1, direction=FORWARD):
    """Compact GS2 (Eq. 9); returns the new x."""
    n, rp, ci, va = _csr(A)
    b, x = _vec(b, n), _vec(x, n)
    _check(_load().ora_gs2_compact(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), outer,
                                   inner, direction), "ora_gs2_compact")
    return x


class AMG:
    """Smoothed-aggregation hierarchy of A (amg.c) with a GS2 or JR smoother.

    theta: classical strength threshold; max_levels; coarse_size: stop
    coarsening at this many rows or fewer (the coarsest level is solved
    exactly)."""

    def __init__(self, A, theta=0.25, max_levels=10, coarse_size=64):
        n, rp, ci, va = _csr(A)
        self.n = n
        self._lib = _load()
        self._ptr = self._lib.ora_amg_build(n, _p(rp), _p(ci), _p(va), theta, max_levels,
                                            coarse_size)
        if not self._ptr:
            raise OracleError("ora_amg_build failed")

    def __del__(self):
        if getattr(self, "_ptr", None):
            self._lib.ora_amg_free(self._ptr)
            self._ptr = None

    @property
    def levels(self):
        return int(self._lib.ora_amg_levels(self._ptr))

    def level(self, l):
        """(rows, entries of A_l, entries of P_l)"""
        v = [ctypes.c_int64() for _ in range(3)]
        _check(self._lib.ora_amg_level(self._ptr, l, *[ctypes.byref(x) for x in v]),
               "ora_amg_level")
        return tuple(int(x.value) for x in v)

    def matrix(self, l):
        n, nnz, _ = self.level(l)
        rp, ci, va = np.zeros(n + 1, np.int64), np.zeros(nnz, np.int32), np.zeros(nnz)
        _check(self._lib.ora_amg_get_matrix(self._ptr, l, _p(rp), _p(ci), _p(va)),
               "ora_amg_get_matrix")
        return rp, ci, va

    def prolongator(self, l):
        n, _, pnnz = self.level(l)
        rp, ci, va = np.zeros(n + 1, np.int64), np.zeros(pnnz, np.int32), np.zeros(pnnz)
        _check(self._lib.ora_amg_get_prolongator(self._ptr, l, _p(rp), _p(ci), _p(va)),
               "ora_amg_get_prolongator")
        return rp, ci, va

    def aggregates(self, l):
        n = self.level(l)[0]
        agg = np.zeros(n, np.int32)
        _check(self._lib.ora_amg_get_aggregates(self._ptr, l, _p(agg)),
               "ora_amg_get_aggregates")
        return agg

    def vcycle(self, b, kind=PC_GS2, outer=1, inner=1, omega=1.0, gamma=1.0,
               direction=SYMMETRIC):
        """x = M^{-1} b, one V-cycle from zero."""
        b = _vec(b, self.n)
        x = np.zeros(self.n)
        _check(self._lib.ora_amg_vcycle(self._ptr, _p(b), _p(x), kind, outer, inner, omega,
                                        gamma, direction), "ora_amg_vcycle")
        return x

    def gmres(self, A, b, x0=None, restart=30, tol=1e-8, max_iters=10000, kind=PC_GS2,
              outer=1, inner=1, omega=1.0, gamma=1.0, direction=SYMMETRIC):
        """GMRES(restart) preconditioned by one V-cycle; (x, SolveInfo)."""
        n, rp, ci, va = _csr(A)
        b = _vec(b, n)
        x = np.zeros(n) if x0 is None else _vec(x0, n)
        info = _Info()
        st = self._lib.ora_gmres_amg(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), restart, tol,
                                     max_iters, self._ptr, kind, outer, inner, omega, gamma,
                                     direction, ctypes.byref(info))
        if st == 1:
            raise OracleError("ora_gmres_amg: invalid argument")
        return x, SolveInfo(info.iters, info.cycles, info.status, info.true_relres)

    def cg(self, A, b, x0=None, tol=1e-8, max_iters=10000, kind=PC_GS2, outer=1, inner=1,
           omega=1.0, gamma=1.0, direction=SYMMETRIC):
        """CG preconditioned by one symmetric V-cycle; (x, SolveInfo)."""
        n, rp, ci, va = _csr(A)
        b = _vec(b, n)
        x = np.zeros(n) if x0 is None else _vec(x0, n)
        info = _Info()
        st = self._lib.ora_cg_amg(n, _p(rp), _p(ci), _p(va), _p(b), _p(x), tol, max_iters,
                                  self._ptr, kind, outer, inner, omega, gamma, direction,
                                  ctypes.byref(info))
        if st == 1:
            raise OracleError("ora_cg_amg: invalid argument")
        return x, SolveInfo(info.iters, info.cycles, info.status, info.true_relres)
