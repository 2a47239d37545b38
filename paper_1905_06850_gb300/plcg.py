"""Python binding of libplcg.so (the C ABI in include/plcg.h).

Argument marshalling only: every step of a solve runs in the library's CUDA
kernels.  There is no CPU fallback -- if the library cannot be loaded, every
call raises.  Device vectors are torch CUDA tensors (float64, contiguous);
torch supplies device memory and the stream, nothing else.

The ctypes names mirror the C names (``plcg_create_stencil``,
``plcg_create_csr``, ``plcg_solve``, ``plcg_solve_host``,
``plcg_solve_batched``, ``plcg_destroy`` ...); ``Matrix`` and ``solve`` are
conveniences on top of them.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "libplcg.so")

PLCG_OK = 0
PLCG_PENDING = 1
PLCG_ERR_INVALID = -1
PLCG_ERR_NOMEM = -2
PLCG_ERR_CUDA = -3
PLCG_ERR_BREAKDOWN = -4
PLCG_ERR_MAXIT = -5
PLCG_ERR_NONFINITE = -6
PLCG_ERR_TIMEOUT = -7
PLCG_ERR_UNIMPL = -8
STATUS_NAMES = {0: "OK", 1: "PENDING", -1: "INVALID", -2: "NOMEM", -3: "CUDA", -4: "BREAKDOWN",
                -5: "MAXIT", -6: "NONFINITE", -7: "TIMEOUT", -8: "UNIMPL"}

PLCG_FP64 = 0
PLCG_FP32_FP64DOT = 1
PLCG_FP32_MATRIX = 2
PLCG_METHOD_PLCG = 0
PLCG_METHOD_CG = 1
PLCG_PRECOND_NONE = 0
PLCG_PRECOND_JACOBI = 1


class plcg_stencil_desc(C.Structure):
    _fields_ = [("dim", C.c_int), ("points", C.c_int), ("nx", C.c_int64), ("ny", C.c_int64),
                ("nz", C.c_int64), ("center", C.c_double), ("off", C.c_double),
                ("diag_shift", C.c_double)]


class plcg_params(C.Structure):
    _fields_ = [("method", C.c_int), ("l", C.c_int), ("shifts", C.POINTER(C.c_double)),
                ("lmin", C.c_double), ("lmax", C.c_double), ("rtol", C.c_double),
                ("maxit", C.c_int64), ("prec", C.c_int), ("dots_2l1", C.c_int),
                ("max_restarts", C.c_int), ("inner_rtol_floor", C.c_double),
                ("grid_ctas", C.c_int), ("precond", C.c_int)]


class plcg_result(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int64), ("spmvs", C.c_int64),
                ("restarts", C.c_int64), ("refinements", C.c_int64),
                ("recursive_relres", C.c_double), ("true_relres", C.c_double),
                ("seconds", C.c_double), ("latency", C.c_double)]


class plcg_launch_info(C.Structure):
    _fields_ = [("kernel", C.c_uint64), ("grid_ctas", C.c_int), ("dyn_smem", C.c_uint),
                ("lookahead", C.c_int), ("staged", C.c_int), ("poll_limit", C.c_uint64),
                ("force_timeout", C.c_int), ("cluster", C.c_int)]


# every symbol include/plcg.h declares, with (restype, argtypes)
_VP = C.c_void_p
SIGNATURES = {
    "plcg_params_default": (None, [C.POINTER(plcg_params)]),
    "plcg_create_stencil": (C.c_int, [C.POINTER(plcg_stencil_desc), _VP, C.POINTER(_VP)]),
    "plcg_create_csr": (C.c_int, [C.c_int64, C.c_int64, _VP, _VP, _VP, C.c_int, C.c_int, _VP,
                                  C.POINTER(_VP)]),
    "plcg_create_var27": (C.c_int, [C.c_int64, C.c_int64, C.c_int64, _VP, C.c_int, C.c_int, _VP,
                                    C.POINTER(_VP)]),
    "plcg_estimate_interval": (C.c_int, [_VP, C.POINTER(plcg_params), C.c_int, C.POINTER(C.c_double),
                                         C.POINTER(C.c_double)]),
    "plcg_destroy": (None, [_VP]),
    "plcg_solve": (C.c_int, [_VP, _VP, _VP, C.POINTER(plcg_params), C.POINTER(plcg_result)]),
    "plcg_solve_host": (C.c_int, [_VP, _VP, _VP, C.POINTER(plcg_params), C.POINTER(plcg_result)]),
    "plcg_solve_batched": (C.c_int, [C.c_int, _VP, _VP, _VP, _VP, _VP, C.POINTER(plcg_params),
                                     _VP]),
    "plcg_solve_stencil_noalloc": (C.c_int, [C.POINTER(plcg_stencil_desc), _VP, _VP,
                                             C.POINTER(plcg_params), C.POINTER(plcg_result), _VP]),
    "plcg_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(_VP)]),
    "plcg_submit": (C.c_int, [_VP, _VP, _VP, _VP, C.POINTER(plcg_params), C.POINTER(C.c_uint64)]),
    "plcg_poll": (C.c_int, [_VP, C.c_uint64, C.POINTER(plcg_result)]),
    "plcg_wait": (C.c_int, [_VP, C.c_uint64, C.POINTER(plcg_result)]),
    "plcg_server_destroy": (None, [_VP]),
    "plcg_set_batched_schedule": (C.c_int, [C.c_int, C.c_double, C.c_double]),
    "plcg_set_batched_launch": (C.c_int, [C.c_int, C.c_int, C.c_int]),
    "plcg_set_cluster_rows": (C.c_int, [C.c_int64]),
    "plcg_last_error": (C.c_char_p, []),
    "plcg_version": (C.c_char_p, []),
    "plcg_debug_set_poll_limit": (None, [C.c_uint64]),
    "plcg_debug_force_barrier_timeout": (None, [C.c_int]),
    "plcg_debug_last_launch": (None, [C.POINTER(plcg_launch_info)]),
    "plcg_debug_server_admission": (C.c_int, [C.c_int, _VP, _VP, _VP, C.c_uint64, C.c_double, C.c_int,
                                              C.c_int, _VP]),
    "plcg_measure_fp64_fma_rate": (C.c_int, [C.POINTER(C.c_double)]),
}

_lib = None


def load(path: str = LIB_PATH):
    """Load libplcg.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: build it with "
                               "python -m paper_1905_06850_gb300.build")
        lib = C.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def last_error() -> str:
    return load().plcg_last_error().decode()


CLUSTER_ROWS_DEFAULT = 12288


def set_cluster_rows(max_rows: int = CLUSTER_ROWS_DEFAULT):
    """plcg_set_cluster_rows: small systems run on one thread-block cluster
    (p(l >= 2)-CG and CG up to max_rows rows, p(1)-CG up to half; 0: never;
    no argument: the library's default)."""
    _check(load().plcg_set_cluster_rows(int(max_rows)))


def measure_fp64_fma_rate() -> float:
    """plcg_measure_fp64_fma_rate: the device's FP64 FMA throughput (FLOP/s)."""
    v = C.c_double()
    _check(load().plcg_measure_fp64_fma_rate(C.byref(v)))
    return v.value


def last_launch() -> dict:
    """plcg_debug_last_launch: shape and flags of this thread's last solve launch."""
    info = plcg_launch_info()
    load().plcg_debug_last_launch(C.byref(info))
    return {name: getattr(info, name) for name, _ in info._fields_}


def server_admission(bytes_, share, waited_s, mem_free, sm_used, num_sms, free_slots):
    """plcg_debug_server_admission: the indices the server's admission pass
    would start, in order, for a queue described by the three lists."""
    n = len(bytes_)
    b = (C.c_uint64 * max(n, 1))(*bytes_)
    sh = (C.c_double * max(n, 1))(*share)
    w = (C.c_double * max(n, 1))(*waited_s)
    out = (C.c_int * max(n, 1))()
    k = load().plcg_debug_server_admission(n, b, sh, w, int(mem_free), float(sm_used), int(num_sms),
                                           int(free_slots), out)
    return list(out[:k])


class PlcgError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"plcg status {STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


def _check(st: int, allow=(PLCG_OK,)):
    if st not in allow:
        raise PlcgError(st, last_error())
    return st


def _stream_ptr(stream):
    if stream is None:
        import torch
        return torch.cuda.current_stream().cuda_stream
    return getattr(stream, "cuda_stream", stream)


@dataclass
class Result:
    status: int
    iters: int
    spmvs: int
    restarts: int
    refinements: int
    recursive_relres: float
    true_relres: float
    seconds: float
    latency: float = 0.0

    @property
    def ok(self) -> bool:
        return self.status == PLCG_OK


def _result(r: plcg_result) -> Result:
    return Result(r.status, r.iters, r.spmvs, r.restarts, r.refinements, r.recursive_relres,
                  r.true_relres, r.seconds, r.latency)


def _prec_code(prec) -> int:
    """Solve precision: "fp64", "fp32" (FP32 vectors and values, FP64 dots,
    scalars and refinement) or "fp32_matrix" (FP32 values, FP64 vectors)."""
    if prec in ("fp32", PLCG_FP32_FP64DOT):
        return PLCG_FP32_FP64DOT
    if prec in ("fp32_matrix", PLCG_FP32_MATRIX):
        return PLCG_FP32_MATRIX
    if prec in ("fp64", PLCG_FP64):
        return PLCG_FP64
    raise ValueError(f"unknown precision {prec!r}")


def make_params(method="plcg", l=1, shifts=None, interval=(0.0, 8.0), rtol=1e-8, maxit=100000,
                prec="fp64", dots_2l1=False, max_restarts=8, inner_rtol_floor=1e-4,
                grid_ctas=0, precond=None):
    p = plcg_params()
    load().plcg_params_default(C.byref(p))
    p.method = PLCG_METHOD_CG if method == "cg" else PLCG_METHOD_PLCG
    p.l = int(l)
    keep = None
    if shifts is not None:
        keep = (C.c_double * len(shifts))(*[float(s) for s in shifts])
        p.shifts = C.cast(keep, C.POINTER(C.c_double))
    p.lmin, p.lmax = float(interval[0]), float(interval[1])
    p.rtol = float(rtol)
    p.maxit = int(maxit)
    p.prec = _prec_code(prec)
    p.dots_2l1 = int(bool(dots_2l1))
    p.max_restarts = int(max_restarts)
    p.inner_rtol_floor = float(inner_rtol_floor)
    p.grid_ctas = int(grid_ctas)
    if precond not in (None, "none", "jacobi"):
        raise ValueError(f"unknown preconditioner {precond!r}")
    p.precond = PLCG_PRECOND_JACOBI if precond == "jacobi" else PLCG_PRECOND_NONE
    return p, keep


class Matrix:
    """A device operator (stencil, CSR or structured 27-point) owned by the library."""

    def __init__(self, op: dict, prec="fp64", stream=None):
        """prec: "fp64" keeps FP64 matrix values; "fp32" and "fp32_matrix"
        store them rounded to FP32 (solvable with prec "fp32" or "fp32_matrix")."""
        lib = load()
        self.op = op
        if op["kind"] == "csr":
            self.n = int(op["n"])
        elif op["kind"] == "var27":
            self.n = int(op["nx"]) * int(op["ny"]) * int(op["nz"])
        else:
            self.n = int(op["nx"]) * int(op["ny"]) * (int(op["nz"]) if op["dim"] == 3 else 1)
        h = _VP()
        if op["kind"] == "var27":
            coef = np.ascontiguousarray(op["coef"], dtype=np.float64)
            if coef.shape != (14, self.n):
                raise ValueError("var27 coef must have shape (14, n)")
            pc = PLCG_FP64 if _prec_code(prec) == PLCG_FP64 else PLCG_FP32_FP64DOT
            _check(lib.plcg_create_var27(int(op["nx"]), int(op["ny"]), int(op["nz"]), coef.ctypes.data,
                                         0, pc, _VP(_stream_ptr(stream)), C.byref(h)))
        elif op["kind"] == "stencil":
            d = plcg_stencil_desc(dim=int(op["dim"]), points=5 if op["dim"] == 2 else 7,
                                  nx=int(op["nx"]), ny=int(op["ny"]),
                                  nz=int(op["nz"]) if op["dim"] == 3 else 1,
                                  center=float(op["center"]), off=float(op["off"]), diag_shift=0.0)
            _check(lib.plcg_create_stencil(C.byref(d), _VP(_stream_ptr(stream)), C.byref(h)))
        else:
            rowptr = np.ascontiguousarray(op["rowptr"], dtype=np.int64)
            col = np.ascontiguousarray(op["col"], dtype=np.int32)
            val = np.ascontiguousarray(op["val"], dtype=np.float64)
            pc = PLCG_FP64 if _prec_code(prec) == PLCG_FP64 else PLCG_FP32_FP64DOT
            _check(lib.plcg_create_csr(self.n, int(col.size), rowptr.ctypes.data, col.ctypes.data,
                                       val.ctypes.data, 0, pc, _VP(_stream_ptr(stream)), C.byref(h)))
        self.handle = h

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            load().plcg_destroy(self.handle)
            self.handle = _VP()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def solve(self, b, x, check=True, **kw) -> Result:
        """plcg_solve on torch CUDA float64 tensors b (in) and x (in: x0, out)."""
        import torch
        if not (b.is_cuda and x.is_cuda and b.dtype == torch.float64 and x.dtype == torch.float64):
            raise TypeError("b and x must be float64 CUDA tensors")
        if not (b.is_contiguous() and x.is_contiguous()) or b.numel() != self.n or x.numel() != self.n:
            raise ValueError("b and x must be contiguous with n elements")
        p, keep = make_params(**kw)
        r = plcg_result()
        st = load().plcg_solve(self.handle, b.data_ptr(), x.data_ptr(), C.byref(p), C.byref(r))
        del keep
        if check:
            _check(st)
        return _result(r)

    def estimate_interval(self, steps=30, **kw):
        """plcg_estimate_interval: (lmin, lmax) Ritz values of `steps` CG steps
        (kw: prec, precond)."""
        p, keep = make_params(**kw)
        lo, hi = C.c_double(), C.c_double()
        _check(load().plcg_estimate_interval(self.handle, C.byref(p), int(steps), C.byref(lo), C.byref(hi)))
        del keep
        return lo.value, hi.value

    def solve_host(self, b: np.ndarray, x: np.ndarray, check=True, **kw) -> Result:
        """plcg_solve_host on host float64 arrays (x in: x0, out: solution)."""
        if b.dtype != np.float64 or x.dtype != np.float64 or not b.flags.c_contiguous \
                or not x.flags.c_contiguous or b.size != self.n or x.size != self.n:
            raise ValueError("b and x must be contiguous float64 arrays of length n")
        p, keep = make_params(**kw)
        r = plcg_result()
        st = load().plcg_solve_host(self.handle, b.ctypes.data, x.ctypes.data, C.byref(p),
                                    C.byref(r))
        del keep
        if check:
            _check(st)
        return _result(r)


def solve_batched(mats, bs, xs, lmins=None, lmaxs=None, check=True, **kw):
    """plcg_solve_batched: mats (list of stencil Matrix), bs/xs (lists of
    float64 CUDA tensors; xs in: x0, out: solutions), optional per-system
    shift intervals.  Returns (status, list of Result)."""
    count = len(mats)
    VP = C.c_void_p
    hA = (VP * count)(*[m.handle.value for m in mats])
    hb = (VP * count)(*[b.data_ptr() for b in bs])
    hx = (VP * count)(*[x.data_ptr() for x in xs])
    lo = None if lmins is None else (C.c_double * count)(*[float(v) for v in lmins])
    hi = None if lmaxs is None else (C.c_double * count)(*[float(v) for v in lmaxs])
    p, keep = make_params(**kw)
    res = (plcg_result * count)()
    st = load().plcg_solve_batched(count, hA, hb, hx, lo, hi, C.byref(p), res)
    del keep
    if check:
        _check(st)
    return st, [_result(r) for r in res]


class Server:
    """plcg_server_*: continuous batching of solves (see include/plcg.h)."""

    def __init__(self, mem_budget_bytes=0, max_inflight=0):
        h = _VP()
        _check(load().plcg_server_create(int(mem_budget_bytes), int(max_inflight), C.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, mat: Matrix, b, x, **kw) -> int:
        p, keep = make_params(**kw)
        t = C.c_uint64()
        _check(load().plcg_submit(self.handle, mat.handle, b.data_ptr(), x.data_ptr(), C.byref(p),
                                  C.byref(t)))
        self._keep[t.value] = (mat, b, x)
        del keep
        return t.value

    def poll(self, ticket: int):
        """None while pending, else the Result."""
        r = plcg_result()
        st = load().plcg_poll(self.handle, ticket, C.byref(r))
        if st == PLCG_PENDING:
            return None
        if st == PLCG_ERR_INVALID and r.status == 0 and r.iters == 0:
            raise PlcgError(st, last_error())
        self._keep.pop(ticket, None)
        return _result(r)

    def wait(self, ticket: int) -> Result:
        r = plcg_result()
        st = load().plcg_wait(self.handle, ticket, C.byref(r))
        if st == PLCG_ERR_INVALID and r.status == 0 and r.iters == 0:
            raise PlcgError(st, last_error())
        self._keep.pop(ticket, None)
        return _result(r)

    def close(self):
        if getattr(self, "handle", None) and self.handle.value:
            load().plcg_server_destroy(self.handle)
            self.handle = _VP()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def solve(op: dict, b, x0=None, **kw):
    """Convenience: build the operator, solve on the GPU, return (x, Result)."""
    import torch
    A = Matrix(op, prec=kw.get("prec", "fp64"))
    bt = torch.as_tensor(b, dtype=torch.float64).cuda().contiguous()
    xt = torch.zeros_like(bt) if x0 is None else torch.as_tensor(x0, dtype=torch.float64).cuda().clone()
    res = A.solve(bt, xt, **kw)
    A.close()
    return xt, res
