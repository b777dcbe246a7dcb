"""GB300 two-stage Gauss-Seidel (GS2) library: Python binding.

Thin ctypes marshalling over the C ABI in ``include/gs2.h`` (libgs2.so, built
in-tree by ``paper_2104_01196_gb300.build``).  Every step of every solve runs
in the library's CUDA kernels; this module only turns arrays into pointers.
There is no CPU fallback: if libgs2.so is missing, loading fails loudly.

Vectors may be torch CUDA tensors (float64, contiguous; used in place) or
numpy float64 arrays (host memory, staged by the library).
"""
from __future__ import annotations

import ctypes
import os
from dataclasses import dataclass

import numpy as np

__all__ = [
    "GS2Error", "Params", "SolveInfo", "Handle", "load", "gs2_setup", "gs2_apply",
    "gs2_apply_ex", "gs_apply", "mtgs_apply", "jr_apply", "amg_vcycle", "gs2_spmv", "gmres_solve", "cg_solve",
    "gs2_batch_solve", "params", "FORWARD", "BACKWARD", "SYMMETRIC", "FP64", "FP32",
    "FP16_ROWSCALED", "PC_NONE", "PC_GS2", "PC_JR", "PC_GS", "PC_MTGS", "PC_AMG", "PC_AMG_JR", "NONCOMPACT", "COMPACT",
    "STATUS",
]

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libgs2.so")

FORWARD, BACKWARD, SYMMETRIC = 0, 1, 2
FP64, FP32, FP16_ROWSCALED, FP32_SWEEP, FP16_SWEEP = 0, 1, 2, 3, 4
PC_NONE, PC_GS2, PC_JR, PC_GS, PC_MTGS, PC_AMG, PC_AMG_JR = 0, 1, 2, 3, 4, 5, 6
AMG_MAX_LEVELS = 16
NONCOMPACT, COMPACT = 0, 1
STATUS = {0: "OK", 1: "INVALID_ARG", 2: "ZERO_DIAGONAL", 3: "OOM", 4: "CUDA",
          5: "NOT_CONVERGED", 6: "BREAKDOWN", 7: "NAN", 8: "TIMEOUT", 9: "BUSY",
          10: "NOT_FOUND"}
_DIR = {"forward": FORWARD, "backward": BACKWARD, "symmetric": SYMMETRIC}
_PREC = {"fp64": FP64, "fp32": FP32, "fp16": FP16_ROWSCALED, "fp32_sweep": FP32_SWEEP,
         "fp16_sweep": FP16_SWEEP}
_KIND = {"none": PC_NONE, "gs2": PC_GS2, "jr": PC_JR, "gs": PC_GS, "mtgs": PC_MTGS,
         "amg": PC_AMG, "amg_jr": PC_AMG_JR}


class GS2Error(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


class _AmgCfg(ctypes.Structure):
    _fields_ = [("theta", ctypes.c_double), ("max_levels", ctypes.c_int),
                ("coarse_size", ctypes.c_int64)]


class Params(ctypes.Structure):
    _fields_ = [("kind", ctypes.c_int), ("outer", ctypes.c_int), ("inner", ctypes.c_int),
                ("omega", ctypes.c_double), ("gamma", ctypes.c_double),
                ("direction", ctypes.c_int), ("precision", ctypes.c_int),
                ("form", ctypes.c_int), ("parts", ctypes.c_int), ("local_sweeps", ctypes.c_int)]


class _Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int), ("cycles", ctypes.c_int), ("status", ctypes.c_int),
                ("true_relres", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("nnz_lower", ctypes.c_int64),
                ("nnz_upper", ctypes.c_int64), ("levels_lower", ctypes.c_int),
                ("levels_upper", ctypes.c_int), ("device_bytes", ctypes.c_int64),
                ("tpr_a", ctypes.c_int), ("tpr_tri", ctypes.c_int),
                ("rpt_a", ctypes.c_int), ("rpt_tri", ctypes.c_int), ("colors", ctypes.c_int),
                ("sell_a", ctypes.c_int), ("sell_tri", ctypes.c_int),
                ("offset_frac_a", ctypes.c_double), ("offset_frac_tri", ctypes.c_double),
                ("solve_mode", ctypes.c_int), ("solve_modes_timed", ctypes.c_int)]


class _KStat(ctypes.Structure):
    _fields_ = [("name", ctypes.c_char * 32), ("launches", ctypes.c_int64),
                ("total_ms", ctypes.c_double), ("bytes", ctypes.c_double)]


class _ServerCfg(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_int64), ("max_slots", ctypes.c_int),
                ("prep_threads", ctypes.c_int), ("restart", ctypes.c_int),
                ("tol", ctypes.c_double), ("max_iters", ctypes.c_int),
                ("has_precond", ctypes.c_int), ("precond", Params),
                ("fail_ticket", ctypes.c_uint64), ("pack_rows", ctypes.c_int64),
                ("pack_max", ctypes.c_int), ("small_rows", ctypes.c_int64),
                ("small_slots", ctypes.c_int)]


class _Request(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("nnz", ctypes.c_int64), ("rowptr", ctypes.c_void_p),
                ("col", ctypes.c_void_p), ("val", ctypes.c_void_p), ("b", ctypes.c_void_p),
                ("x0", ctypes.c_void_p)]


class _ServerStats(ctypes.Structure):
    _fields_ = [(f, ctypes.c_int64) for f in
                ("submitted", "admitted", "completed", "failed", "pending", "active",
                 "max_active", "reserved_bytes", "budget_bytes")]


@dataclass
class SolveInfo:
    iters: int
    cycles: int
    status: int
    true_relres: float

    @property
    def ok(self) -> bool:
        return self.status == 0


_lib = None


def load(path: str | None = None):
    """Load libgs2.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    p = path or LIB_PATH
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build it with "
                           "`python -m paper_2104_01196_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(p)
    P, I, I64, D, U = (ctypes.c_void_p, ctypes.c_int, ctypes.c_int64, ctypes.c_double,
                       ctypes.c_uint)
    sig = {
        "gs2_setup": [I64, I64, P, P, P, I, U, P, ctypes.POINTER(P)],
        "gs2_set_stream": [P, P],
        "gs2_get_stats": [P, ctypes.POINTER(_Stats)],
        "gs2_apply": [P, P, P, I, I, D, I],
        "gs2_apply_ex": [P, P, P, ctypes.POINTER(Params)],
        "relax_apply": [P, P, P, ctypes.POINTER(Params)],
        "gs_apply": [P, P, P, I, D, I],
        "mtgs_apply": [P, P, P, I, D, I],
        "jr_apply": [P, P, P, I, D],
        "gs2_spmv": [P, P, P],
        "gmres_solve": [P, P, P, I, D, I, ctypes.POINTER(Params), ctypes.POINTER(_Info)],
        "cg_solve": [P, P, P, D, I, ctypes.POINTER(Params), ctypes.POINTER(_Info)],
        "gs2_batch_solve": [P, P, P, I, I, D, I, ctypes.POINTER(Params), ctypes.POINTER(_Info)],
        "gs2_profile_enable": [P, I],
        "gs2_profile_filter": [P, ctypes.c_char_p],
        "gs2_check": [P],
        "gs2_set_graph_mode": [P, I],
        "gs2_test_stall_barrier": [P],
        "gs2_autotune": [P],
        "gs2_autotune_gmres": [P, I, ctypes.POINTER(Params), ctypes.POINTER(I)],
        "gs2_profile_read": [P, ctypes.POINTER(_KStat), I, ctypes.POINTER(I)],
        "gs2_profile_reset": [P],
        "gs2_amg_setup": [P, ctypes.POINTER(_AmgCfg)],
        "gs2_amg_info": [P, ctypes.POINTER(I), P, P, P],
        "gs2_amg_vcycle": [P, P, P, ctypes.POINTER(Params)],
        "gs2_pack_setup": [I, P, P, P, P, U, P, ctypes.POINTER(P)],
        "gs2_pack_info": [P, ctypes.POINTER(I), P],
        "gs2_pack_gmres": [P, P, P, I, D, I, ctypes.POINTER(Params), P],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = ctypes.c_int
    lib.gs2_destroy.argtypes = [P]
    lib.gs2_destroy.restype = None
    lib.gs2_last_error.restype = ctypes.c_char_p
    lib.gs2_version.restype = ctypes.c_char_p
    lib.gs2_launch_count.restype = ctypes.c_int64
    lib.gs2_server_create.argtypes = [ctypes.POINTER(_ServerCfg), ctypes.POINTER(P)]
    lib.gs2_server_create.restype = I
    lib.gs2_server_submit.argtypes = [P, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]
    lib.gs2_server_submit.restype = I
    lib.gs2_server_poll.argtypes = [P, ctypes.c_uint64, ctypes.POINTER(_Info), P,
                                    ctypes.POINTER(D)]
    lib.gs2_server_poll.restype = I
    lib.gs2_server_wait.argtypes = [P, ctypes.c_uint64, D, ctypes.POINTER(_Info), P,
                                    ctypes.POINTER(D)]
    lib.gs2_server_wait.restype = I
    lib.gs2_server_get_stats.argtypes = [P, ctypes.POINTER(_ServerStats)]
    lib.gs2_server_get_stats.restype = I
    lib.gs2_server_footprint.argtypes = [ctypes.POINTER(_ServerCfg), I64, I64]
    lib.gs2_server_footprint.restype = I64
    lib.gs2_server_destroy.argtypes = [P]
    lib.gs2_server_destroy.restype = None
    _lib = lib
    return lib


def _err(st: int):
    msg = load().gs2_last_error().decode(errors="replace")
    raise GS2Error(st, msg)


def _check(st: int):
    if st != 0:
        _err(st)


def _torch():
    import torch
    return torch


def _ptr(a, writable=False):
    """(pointer, keepalive) of a float64 vector: torch CUDA tensor or numpy."""
    if a is None:
        return None, None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float64 or not a.flags.c_contiguous:
            raise TypeError("numpy vectors must be contiguous float64")
        if writable and not a.flags.writeable:
            raise TypeError("output vector is read-only")
        return a.ctypes.data, a
    t = a
    if t.dtype != _torch().float64 or not t.is_contiguous():
        raise TypeError("torch vectors must be contiguous float64")
    return t.data_ptr(), t


def params(kind="gs2", outer=1, inner=1, omega=1.0, gamma=1.0, direction="forward",
           precision="fp64", form="noncompact", parts=1, local=1) -> Params:
    """gs2_params in the paper's notation: GS2(n_t = outer, n_k = local,
    n_j = inner); parts > 1 is the hybrid (block-Jacobi) form over that many
    row blocks."""
    k = _KIND[kind] if isinstance(kind, str) else int(kind)
    d = _DIR[direction] if isinstance(direction, str) else int(direction)
    p = _PREC[precision] if isinstance(precision, str) else int(precision)
    f = {"noncompact": NONCOMPACT, "compact": COMPACT}[form] if isinstance(form, str) else int(form)
    return Params(k, outer, inner, omega, gamma, d, p, f, parts, local)


class Handle:
    """A matrix resident on the device with its split, triangles and
    temporaries (library-owned)."""

    def __init__(self, ptr, n, nnz, stream):
        self._ptr = ptr
        self.n = n
        self.nnz = nnz
        self.stream = stream

    @property
    def ptr(self):
        if not self._ptr:
            raise RuntimeError("handle destroyed")
        return self._ptr

    def stats(self) -> dict:
        s = _Stats()
        _check(load().gs2_get_stats(self.ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _Stats._fields_}

    def set_stream(self, stream):
        self.stream = stream
        _check(load().gs2_set_stream(self.ptr, stream or None))

    def profile(self, enable: bool):
        _check(load().gs2_profile_enable(self.ptr, 1 if enable else 0))

    def autotune_gmres(self, restart: int = 30, precond: Params | None = None) -> int:
        """Time one restart cycle per solve structure (separate launches,
        cycle graphs, one launch) and make the fastest the automatic
        choice; returns it (gs2_autotune_gmres)."""
        mode = ctypes.c_int()
        _check(load().gs2_autotune_gmres(self.ptr, restart,
                                         ctypes.byref(precond) if precond is not None else None,
                                         ctypes.byref(mode)))
        return int(mode.value)

    def autotune(self):
        """Pick the fastest tile shape of each matrix (cached by matrix class)."""
        _check(load().gs2_autotune(self.ptr))

    def amg_setup(self, theta: float = 0.25, max_levels: int = 10, coarse_size: int = 64):
        """Build the smoothed-aggregation hierarchy used by the AMG
        preconditioner kinds (host setup, device-resident levels)."""
        _check(load().gs2_amg_setup(self.ptr, ctypes.byref(_AmgCfg(theta, max_levels,
                                                                    coarse_size))))

    def amg_info(self) -> list:
        """[(rows, matrix entries, prolongator entries)] per level."""
        lv = ctypes.c_int()
        arr = [(ctypes.c_int64 * AMG_MAX_LEVELS)() for _ in range(3)]
        _check(load().gs2_amg_info(self.ptr, ctypes.byref(lv), *arr))
        return [(arr[0][i], arr[1][i], arr[2][i]) for i in range(lv.value)]

    def set_graph_mode(self, mode: int):
        """0: automatic (one thread-block cluster for a small system that fits
        its shared memory, else one launch for small systems, else graphs), 1:
        restart cycles as CUDA graphs, 2: separate launches, 3: one launch, 4:
        one thread-block cluster (GMRES, CG, or a pack: one cluster a system)."""
        _check(load().gs2_set_graph_mode(self.ptr, mode))

    def test_stall_barrier(self):
        """Test hook: the next one-launch solve's barrier never opens."""
        _check(load().gs2_test_stall_barrier(self.ptr))

    def check(self):
        """Synchronise and raise if a kernel reported a device-side error."""
        _check(load().gs2_check(self.ptr))

    def profile_filter(self, name: str | None):
        """Time only kernels called `name` (None: all)."""
        _check(load().gs2_profile_filter(self.ptr, name.encode() if name else None))

    def profile_read(self) -> dict:
        arr = (_KStat * 64)()
        cnt = ctypes.c_int(0)
        _check(load().gs2_profile_read(self.ptr, arr, 64, ctypes.byref(cnt)))
        return {arr[i].name.decode(): dict(launches=arr[i].launches, total_ms=arr[i].total_ms,
                                           bytes=arr[i].bytes) for i in range(cnt.value)}

    def profile_reset(self):
        _check(load().gs2_profile_reset(self.ptr))

    def close(self):
        if self._ptr:
            load().gs2_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _current_stream():
    try:
        torch = _torch()
        if torch.cuda.is_available():
            return torch.cuda.current_stream().cuda_stream
    except Exception:
        pass
    return 0


def gs2_setup(A, precisions=(), stream=None) -> Handle:
    """Create a handle for CSR A = (rowptr int64, col int32, val float64);
    arrays may be numpy (host) or torch tensors (host or CUDA)."""
    rp, ci, va = A
    keep = []
    on_dev = 0
    ptrs = []
    for arr, dt in ((rp, "int64"), (ci, "int32"), (va, "float64")):
        if isinstance(arr, np.ndarray):
            arr = np.ascontiguousarray(arr, dtype=dt)
            keep.append(arr)
            ptrs.append(arr.ctypes.data)
        else:
            torch = _torch()
            t = arr.to(getattr(torch, dt)).contiguous()
            keep.append(t)
            ptrs.append(t.data_ptr())
            on_dev = 1 if t.is_cuda else 0
    n = len(rp) - 1
    nnz = int(rp[-1])
    mask = 0
    for p in precisions:
        mask |= 1 << (_PREC[p] if isinstance(p, str) else int(p))
    s = _current_stream() if stream is None else stream
    out = ctypes.c_void_p()
    _check(load().gs2_setup(n, nnz, ptrs[0], ptrs[1], ptrs[2], on_dev, mask, s or None,
                            ctypes.byref(out)))
    return Handle(out.value, n, nnz, s)


class PackHandle(Handle):
    """A pack: independent systems held as one block-diagonal handle.
    `offsets[s]` is the first row of system s in the concatenated vectors."""

    def __init__(self, ptr, n, nnz, stream, offsets):
        super().__init__(ptr, n, nnz, stream)
        self.offsets = offsets
        self.count = len(offsets) - 1

    def split(self, v) -> list:
        """The per-system pieces of a concatenated vector."""
        return [v[self.offsets[s]:self.offsets[s + 1]] for s in range(self.count)]


def pack_setup(As, precisions=(), stream=None) -> PackHandle:
    """Create a pack from a list of host CSR matrices (rowptr int64, col
    int32, val float64), each indexed from 0 within its own system."""
    cnt = len(As)
    keep = []
    N = (ctypes.c_int64 * cnt)()
    R, C, V = (ctypes.c_void_p * cnt)(), (ctypes.c_void_p * cnt)(), (ctypes.c_void_p * cnt)()
    nnz = 0
    for s, (rp, ci, va) in enumerate(As):
        rp = np.ascontiguousarray(rp, dtype=np.int64)
        ci = np.ascontiguousarray(ci, dtype=np.int32)
        va = np.ascontiguousarray(va, dtype=np.float64)
        keep += [rp, ci, va]
        N[s] = len(rp) - 1
        R[s], C[s], V[s] = rp.ctypes.data, ci.ctypes.data, va.ctypes.data
        nnz += int(rp[-1])
    mask = 0
    for p in precisions:
        mask |= 1 << (_PREC[p] if isinstance(p, str) else int(p))
    st = _current_stream() if stream is None else stream
    out = ctypes.c_void_p()
    _check(load().gs2_pack_setup(cnt, N, R, C, V, mask, st or None, ctypes.byref(out)))
    cnt_out = ctypes.c_int()
    off = (ctypes.c_int64 * (cnt + 1))()
    _check(load().gs2_pack_info(out.value, ctypes.byref(cnt_out), off))
    offsets = [int(off[i]) for i in range(cnt_out.value + 1)]
    return PackHandle(out.value, offsets[-1], nnz, st, offsets)


def pack_gmres(h: PackHandle, b, x, restart=30, tol=1e-8, max_iters=10000,
               precond: Params | None = None) -> list:
    """GMRES on every system of a pack (b, x concatenated); a SolveInfo per
    system."""
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    infos = (_Info * h.count)()
    st = load().gs2_pack_gmres(h.ptr, pb, px, restart, tol, max_iters,
                               ctypes.byref(precond) if precond is not None else None, infos)
    if st not in _SOLVER_STATUSES:
        _err(st)
    return [SolveInfo(i.iters, i.cycles, i.status, i.true_relres) for i in infos]


def gs2_apply(h, b, x, outer_sweeps=1, inner_sweeps=1, damping=1.0, direction=FORWARD):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    d = _DIR[direction] if isinstance(direction, str) else direction
    _check(load().gs2_apply(h.ptr, pb, px, outer_sweeps, inner_sweeps, damping, d))
    return x


def gs2_apply_ex(h, b, x, p: Params):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    _check(load().gs2_apply_ex(h.ptr, pb, px, ctypes.byref(p)))
    return x


def relax_apply(h, b, x, p: Params):
    """The relaxation of p's kind (GS2, JR, GS, MTGS), global or hybrid, from x."""
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    _check(load().relax_apply(h.ptr, pb, px, ctypes.byref(p)))


def gs_apply(h, b, x, sweeps=1, omega=1.0, direction=FORWARD):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    d = _DIR[direction] if isinstance(direction, str) else direction
    _check(load().gs_apply(h.ptr, pb, px, sweeps, omega, d))
    return x


def mtgs_apply(h, b, x, sweeps=1, omega=1.0, direction=FORWARD):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    d = _DIR[direction] if isinstance(direction, str) else direction
    _check(load().mtgs_apply(h.ptr, pb, px, sweeps, omega, d))
    return x


def amg_vcycle(h, b, x, params):
    """x = M^{-1} b, one V-cycle (params.kind PC_AMG or PC_AMG_JR)."""
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    _check(load().gs2_amg_vcycle(h.ptr, pb, px, ctypes.byref(params)))
    return x


def jr_apply(h, b, x, sweeps=1, omega=1.0):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    _check(load().jr_apply(h.ptr, pb, px, sweeps, omega))
    return x


def gs2_spmv(h, x, y):
    px, _kx = _ptr(x)
    py, _ky = _ptr(y, True)
    _check(load().gs2_spmv(h.ptr, px, py))
    return y


_SOLVER_STATUSES = (0, 5, 6, 7)


def gmres_solve(h, b, x, restart=30, tol=1e-8, max_iters=10000, precond: Params | None = None):
    """Restarted right-preconditioned GMRES; returns SolveInfo (the solver
    statuses NOT_CONVERGED / BREAKDOWN / NAN are returned, not raised)."""
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    info = _Info()
    st = load().gmres_solve(h.ptr, pb, px, restart, tol, max_iters,
                            ctypes.byref(precond) if precond is not None else None,
                            ctypes.byref(info))
    if st not in _SOLVER_STATUSES:
        _err(st)
    return SolveInfo(info.iters, info.cycles, info.status, info.true_relres)


def cg_solve(h, b, x, tol=1e-8, max_iters=10000, precond: Params | None = None):
    pb, _kb = _ptr(b)
    px, _kx = _ptr(x, True)
    info = _Info()
    st = load().cg_solve(h.ptr, pb, px, tol, max_iters,
                         ctypes.byref(precond) if precond is not None else None,
                         ctypes.byref(info))
    if st not in _SOLVER_STATUSES:
        _err(st)
    return SolveInfo(info.iters, info.cycles, info.status, info.true_relres)


def gs2_batch_solve(handles, bs, xs, restart=30, tol=1e-8, max_iters=10000,
                    precond: Params | None = None):
    """Solve independent systems together; returns a list of SolveInfo."""
    cnt = len(handles)
    H = (ctypes.c_void_p * cnt)(*[h.ptr for h in handles])
    keep = []
    B = (ctypes.c_void_p * cnt)()
    X = (ctypes.c_void_p * cnt)()
    for i in range(cnt):
        pb, kb = _ptr(bs[i])
        px, kx = _ptr(xs[i], True)
        keep += [kb, kx]
        B[i], X[i] = pb, px
    infos = (_Info * cnt)()
    st = load().gs2_batch_solve(H, B, X, cnt, restart, tol, max_iters,
                                ctypes.byref(precond) if precond is not None else None, infos)
    if st not in _SOLVER_STATUSES:
        _err(st)
    return [SolveInfo(i.iters, i.cycles, i.status, i.true_relres) for i in infos]


class Server:
    """Continuous-batching solve server on the current CUDA device (see
    gs2_server_* in include/gs2.h).  Matrices and vectors are host numpy."""

    def __init__(self, restart=30, tol=1e-8, max_iters=10000, precond: Params | None = None,
                 max_slots=4, prep_threads=2, hbm_budget_bytes=0, fail_ticket=0,
                 pack_rows=0, pack_max=0, small_rows=0, small_slots=0):
        """pack_rows > 0: requests of at most that many rows are admitted
        together (up to pack_max, 0 = 64) and solved as one pack.
        small_slots > 0: that many of the max_slots slots are kept for
        requests of at most small_rows rows, which pass larger ones waiting
        for a slot."""
        self._cfg = _ServerCfg(hbm_budget_bytes, max_slots, prep_threads, restart, tol,
                               max_iters, 1 if precond is not None else 0,
                               precond if precond is not None else Params(), fail_ticket,
                               pack_rows, pack_max, small_rows, small_slots)
        out = ctypes.c_void_p()
        _check(load().gs2_server_create(ctypes.byref(self._cfg), ctypes.byref(out)))
        self._ptr = out.value

    def footprint(self, n: int, nnz: int) -> int:
        return int(load().gs2_server_footprint(ctypes.byref(self._cfg), n, nnz))

    def submit(self, A, b, x0=None) -> int:
        rp = np.ascontiguousarray(A[0], dtype=np.int64)
        ci = np.ascontiguousarray(A[1], dtype=np.int32)
        va = np.ascontiguousarray(A[2], dtype=np.float64)
        b = np.ascontiguousarray(b, dtype=np.float64)
        x0 = None if x0 is None else np.ascontiguousarray(x0, dtype=np.float64)
        q = _Request(len(rp) - 1, int(rp[-1]), rp.ctypes.data, ci.ctypes.data, va.ctypes.data,
                     b.ctypes.data, x0.ctypes.data if x0 is not None else None)
        t = ctypes.c_uint64()
        _check(load().gs2_server_submit(self._ptr, ctypes.byref(q), ctypes.byref(t)))
        return int(t.value)

    def _collect(self, fn, ticket, n, *extra):
        info = _Info()
        x = np.empty(n) if n else None
        lat = ctypes.c_double()
        st = fn(self._ptr, ticket, *extra, ctypes.byref(info),
                x.ctypes.data if x is not None else None, ctypes.byref(lat))
        return st, SolveInfo(info.iters, info.cycles, info.status, info.true_relres), x, lat.value

    def poll(self, ticket: int, n: int = 0):
        """None while busy, else (SolveInfo, x or None, latency_ms)."""
        st, info, x, lat = self._collect(load().gs2_server_poll, ticket, n)
        if st == 9:
            return None
        if st == 10:
            _err(st)
        return info, x, lat

    def wait(self, ticket: int, n: int = 0, timeout: float = 600.0):
        """Block until done: (SolveInfo, x or None, latency_ms)."""
        st, info, x, lat = self._collect(load().gs2_server_wait, ticket, n,
                                         ctypes.c_double(timeout))
        if st in (8, 10):
            _err(st)
        return info, x, lat

    def stats(self) -> dict:
        s = _ServerStats()
        _check(load().gs2_server_get_stats(self._ptr, ctypes.byref(s)))
        return {f: getattr(s, f) for f, _ in _ServerStats._fields_}

    def close(self):
        if self._ptr:
            load().gs2_server_destroy(self._ptr)
            self._ptr = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def server_footprint(n: int, nnz: int, restart: int = 30, precond: Params | None = None) -> int:
    """Device bytes the server reserves for a request of this size."""
    cfg = _ServerCfg(0, 1, 1, restart, 1e-8, 100, 1 if precond is not None else 0,
                     precond if precond is not None else Params(), 0)
    return int(load().gs2_server_footprint(ctypes.byref(cfg), n, nnz))


def version() -> str:
    return load().gs2_version().decode()


def launch_count() -> int:
    """Kernel launches made by the library in this process so far."""
    return int(load().gs2_launch_count())
