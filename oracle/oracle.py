"""ctypes front end of the FP64 CPU oracle (``plcg_oracle.c``).

THIS IS TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and
``bench.py`` (its CPU-baseline leg, and the statement of each FP32 result's
error against the FP64 oracle, outside every timed region) may import it.  It does not import the
CUDA library or its binding, and the CUDA library does not import it.

The operator is described by a plain dict, the same description the seeded
input generators produce:

* stencil: ``{"kind": "stencil", "dim": 2|3, "nx", "ny", "nz", "center", "off"}``
  (Dirichlet 5-/7-point, lexicographic order with x fastest; ``center``
  already includes any diagonal shift);
* CSR: ``{"kind": "csr", "n", "rowptr" (int64), "col" (int32), "val" (float64)}``;
* structured 27-point: ``{"kind": "var27", "nx", "ny", "nz", "coef" (14, n)}``
  (diagonal, then the weights to the 13 forward neighbours).

The method's arithmetic lives in the C file; this module only marshals arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "plcg_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")

ORC_OK = 0
ORC_ERR_INVALID = -1
ORC_ERR_NOMEM = -2
ORC_ERR_BREAKDOWN = -4
ORC_ERR_MAXIT = -5
ORC_ERR_NONFINITE = -6


class _Op(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("dim", C.c_int),
        ("nx", C.c_int64), ("ny", C.c_int64), ("nz", C.c_int64),
        ("center", C.c_double), ("off", C.c_double),
        ("n", C.c_int64),
        ("rowptr", C.c_void_p), ("col", C.c_void_p), ("val", C.c_void_p),
        ("coef", C.c_void_p),
    ]


class _Params(C.Structure):
    _fields_ = [
        ("l", C.c_int), ("sigma", C.c_void_p), ("rtol", C.c_double),
        ("maxit", C.c_int64), ("dots_2l1", C.c_int), ("max_restarts", C.c_int),
        ("precond", C.c_int),
    ]


class _Result(C.Structure):
    _fields_ = [
        ("status", C.c_int),
        ("iters", C.c_int64), ("spmvs", C.c_int64), ("dots", C.c_int64),
        ("restarts", C.c_int64), ("segments", C.c_int64),
        ("recursive_relres", C.c_double), ("true_relres", C.c_double),
        ("trace_cap", C.c_int64), ("trace_len", C.c_int64),
        ("x_hist", C.c_void_p), ("zeta_hist", C.c_void_p),
        ("gamma_hist", C.c_void_p), ("delta_hist", C.c_void_p),
        ("g_hist", C.c_void_p), ("z_hist", C.c_void_p), ("graw_hist", C.c_void_p),
    ]


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liboracle.so`` (plain gcc, -O2, serial)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"],
                       check=True)
        os.replace(tmp, _LIB)
    return _LIB


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = C.CDLL(build())
        for name in ("orc_cg", "orc_plcg"):
            fn = getattr(lib, name)
            fn.restype = C.c_int
            fn.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p, C.POINTER(_Params),
                           C.POINTER(_Result)]
        lib.orc_apply.restype = None
        lib.orc_apply.argtypes = [C.POINTER(_Op), C.c_void_p, C.c_void_p]
        lib.orc_chebyshev_shifts.restype = None
        lib.orc_chebyshev_shifts.argtypes = [C.c_int, C.c_double, C.c_double, C.c_void_p]
        for name, st in (("orc_sizeof_op", _Op), ("orc_sizeof_params", _Params),
                         ("orc_sizeof_result", _Result)):
            fn = getattr(lib, name)
            fn.restype = C.c_int
            if fn() != C.sizeof(st):
                raise RuntimeError(f"oracle struct layout mismatch for {st.__name__}")
        _lib = lib
    return _lib


def _ptr(a: np.ndarray | None):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


class _OpHolder:
    """Keeps the arrays referenced by an ``_Op`` alive."""

    def __init__(self, op: dict):
        o = _Op()
        if op["kind"] == "stencil":
            o.kind = 0
            o.dim = int(op["dim"])
            o.nx, o.ny = int(op["nx"]), int(op["ny"])
            o.nz = int(op.get("nz", 1)) if o.dim == 3 else 1
            o.center, o.off = float(op["center"]), float(op["off"])
            o.n = o.nx * o.ny * o.nz
            self.keep = ()
        elif op["kind"] == "csr":
            o.kind = 1
            rowptr = np.ascontiguousarray(op["rowptr"], dtype=np.int64)
            col = np.ascontiguousarray(op["col"], dtype=np.int32)
            val = np.ascontiguousarray(op["val"], dtype=np.float64)
            o.n = int(op["n"])
            if rowptr.shape != (o.n + 1,) or col.shape != val.shape or rowptr[-1] != col.size:
                raise ValueError("inconsistent CSR arrays")
            o.rowptr, o.col, o.val = _ptr(rowptr), _ptr(col), _ptr(val)
            self.keep = (rowptr, col, val)
        elif op["kind"] == "var27":
            o.kind = 2
            o.dim = 3
            o.nx, o.ny, o.nz = int(op["nx"]), int(op["ny"]), int(op["nz"])
            o.n = o.nx * o.ny * o.nz
            coef = np.ascontiguousarray(op["coef"], dtype=np.float64)
            if coef.shape != (14, o.n):
                raise ValueError("var27 coef must have shape (14, n)")
            o.coef = _ptr(coef)
            self.keep = (coef,)
        else:
            raise ValueError(f"unknown operator kind {op['kind']!r}")
        self.op = o
        self.n = int(o.n)


def apply(op: dict, x: np.ndarray) -> np.ndarray:
    """y = A x in FP64."""
    h = _OpHolder(op)
    x = np.ascontiguousarray(x, dtype=np.float64)
    if x.shape != (h.n,):
        raise ValueError("x has the wrong length")
    y = np.empty(h.n, dtype=np.float64)
    _load().orc_apply(C.byref(h.op), _ptr(x), _ptr(y))
    return y


def chebyshev_shifts(l: int, lmin: float, lmax: float) -> np.ndarray:
    """Sec. 2.2, Eq. (chebyshev): the l shifts on [lmin, lmax]."""
    s = np.empty(l, dtype=np.float64)
    _load().orc_chebyshev_shifts(int(l), float(lmin), float(lmax), _ptr(s))
    return s


@dataclass
class Result:
    x: np.ndarray
    status: int
    iters: int
    spmvs: int
    dots: int
    restarts: int
    segments: int
    recursive_relres: float
    true_relres: float
    trace: dict = field(default_factory=dict)


_PRECONDS = {None: 0, "none": 0, "jacobi": 1}


def _solve(fn_name, op, b, x0, l, sigma, rtol, maxit, dots_2l1, max_restarts, trace_cap,
           precond=None):
    lib = _load()
    h = _OpHolder(op)
    n = h.n
    b = np.ascontiguousarray(b, dtype=np.float64)
    if b.shape != (n,):
        raise ValueError("b has the wrong length")
    x = np.zeros(n) if x0 is None else np.array(x0, dtype=np.float64, copy=True)
    sig = None if sigma is None else np.ascontiguousarray(sigma, dtype=np.float64)
    p = _Params(l=int(l), sigma=_ptr(sig), rtol=float(rtol), maxit=int(maxit),
                dots_2l1=int(bool(dots_2l1)), max_restarts=int(max_restarts),
                precond=_PRECONDS[precond])
    r = _Result()
    tr = {}
    if trace_cap > 0:
        W = 2 * l + 1
        tr = {
            "x": np.zeros((trace_cap, n)), "zeta": np.zeros(trace_cap),
            "gamma": np.zeros(trace_cap), "delta": np.zeros(trace_cap),
            "g": np.zeros((trace_cap, W)), "graw": np.zeros((trace_cap, W)),
        }
        if fn_name == "orc_plcg":
            tr["z"] = np.zeros((l + 1, trace_cap, n))
        r.trace_cap = trace_cap
        r.x_hist, r.zeta_hist = _ptr(tr["x"]), _ptr(tr["zeta"])
        r.gamma_hist, r.delta_hist = _ptr(tr["gamma"]), _ptr(tr["delta"])
        r.g_hist, r.graw_hist = _ptr(tr["g"]), _ptr(tr["graw"])
        r.z_hist = _ptr(tr.get("z"))
    getattr(lib, fn_name)(C.byref(h.op), _ptr(b), _ptr(x), C.byref(p), C.byref(r))
    if trace_cap > 0:
        tr["len"] = int(r.trace_len)
    return Result(x=x, status=r.status, iters=r.iters, spmvs=r.spmvs, dots=r.dots,
                  restarts=r.restarts, segments=r.segments,
                  recursive_relres=r.recursive_relres, true_relres=r.true_relres, trace=tr)


def cg(op, b, x0=None, rtol=1e-8, maxit=100000, max_restarts=8, trace_cap=0,
       precond=None) -> Result:
    """Classic Hestenes-Stiefel CG in FP64 (textbook; Sec. 1 cites it).

    ``precond="jacobi"``: the textbook preconditioned CG with M = diag(A);
    the tolerance then applies to natural norms ||.||_{M^{-1}} (Sec. 2.2,
    "Residual norm in p(l)-CG")."""
    return _solve("orc_cg", op, b, x0, 1, None, rtol, maxit, 0, max_restarts, trace_cap,
                  precond)


def plcg(op, b, x0=None, l=1, sigma=None, rtol=1e-8, maxit=100000, dots_2l1=True,
         max_restarts=8, trace_cap=0, precond=None) -> Result:
    """Algorithm 1 in FP64.  ``sigma`` defaults to zero shifts.

    ``precond=None``: M = I.  ``precond="jacobi"``: M = diag(A), with u and
    z^(l) kept apart and natural-norm stopping (Sec. 2.2)."""
    if sigma is None:
        sigma = np.zeros(l)
    sigma = np.asarray(sigma, dtype=np.float64)
    if sigma.shape != (l,):
        raise ValueError("need exactly l shifts")
    return _solve("orc_plcg", op, b, x0, l, sigma, rtol, maxit, dots_2l1, max_restarts,
                  trace_cap, precond)


def refined(op, b, method="plcg", l=1, sigma=None, rtol=1e-8, floor=1e-4, maxit=100000,
            dots_2l1=False, max_restarts=8) -> Result:
    """The FP32 path's outer refinement loop (the paper has none; it is the
    reading the FP32-with-FP64-correction path follows), restated in FP64
    around the FP64 solvers: r = b - A x; stop when ||r|| < rtol ||b||;
    otherwise solve A d = r from d = 0 to the absolute tolerance
    max(floor ||r||, rtol ||b|| / 2) and set x += d.  Every inner solve
    starts a new Krylov space (a restart in the sense of Sec. 2.2), so this
    gives the iteration count of the FP32 path's segment structure without
    its FP32 rounding.  M = I.  Returns a Result whose iters sums the inner
    solves and whose segments counts them."""
    x = np.zeros_like(np.asarray(b, dtype=np.float64))
    nb = float(np.linalg.norm(b))
    iters = segments = restarts = 0
    while True:
        r = np.asarray(b, dtype=np.float64) - apply(op, x)
        rn = float(np.linalg.norm(r))
        if rn < rtol * nb or iters >= maxit or nb == 0.0:
            status = ORC_OK if (rn < rtol * nb or nb == 0.0) else ORC_ERR_MAXIT
            return Result(x=x, status=status, iters=iters, spmvs=0, dots=0, restarts=restarts,
                          segments=segments, recursive_relres=rn / nb if nb else 0.0,
                          true_relres=rn / nb if nb else 0.0, trace={})
        inner = max(floor * rn, 0.5 * rtol * nb) / rn
        if method == "cg":
            s = cg(op, r, rtol=inner, maxit=maxit - iters, max_restarts=max_restarts)
        else:
            s = plcg(op, r, l=l, sigma=sigma, rtol=inner, maxit=maxit - iters, dots_2l1=dots_2l1,
                     max_restarts=max_restarts)
        x = x + s.x
        iters += s.iters
        restarts += s.restarts
        segments += 1
        if s.status not in (ORC_OK, ORC_ERR_MAXIT):
            return Result(x=x, status=s.status, iters=iters, spmvs=0, dots=0, restarts=restarts,
                          segments=segments, recursive_relres=0.0, true_relres=rn / nb, trace={})
