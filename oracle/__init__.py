"""CPU oracle for the reproducible (pipelined) PBiCGStab hot path.

TEST INFRASTRUCTURE ONLY: the plain, slow, obviously correct CPU statement of
what the GPU library must return bit for bit. Only ``tests/``, the smoke check
in ``__graft_entry__`` and the CPU-baseline leg of ``bench.py`` may import it;
the product package never does. It shares no code with the CUDA library.

The arithmetic lives in ``exact.c`` (TwoSum/TwoProd, Alg. 1-2; the exact dot of
Sec. 2 / Sec. 3.2 via a Kulisch accumulator, rounded once) and ``solver.c``
(fma SpMV and Jacobi of Sec. 4.1, classic PBiCGStab of Fig. 2, pipelined
p-PBiCGStab of Fig. 4). This module only builds the shared object with gcc
(``-O2 -ffp-contract=off``, no fast-math) and marshals numpy arrays.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_SRCS = ["exact.c", "solver.c"]
_lock = threading.Lock()
_lib = None

DIGITS = 136
HIST_W = 12
OK, EINVAL, EBREAKDOWN, ENAN = 0, 1, 4, 5
CLASSIC, PIPELINED = 0, 1

CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC",
          "-shared", "-Wall", "-Wextra"]


def build(force: bool = False) -> str:
    """Compile liboracle.so in-tree (oracle/_build) if it is missing or stale."""
    os.makedirs(os.path.join(_HERE, "_build"), exist_ok=True)
    srcs = [os.path.join(_HERE, s) for s in _SRCS]
    deps = srcs + [os.path.join(_HERE, "oracle.h")]
    if not force and os.path.exists(_SO):
        so_t = os.path.getmtime(_SO)
        if all(os.path.getmtime(d) <= so_t for d in deps):
            return _SO
    tmp = _SO + f".tmp{os.getpid()}"
    # OpenMP for the threaded oracle (set_threads); without it the oracle is
    # sequential and the thread count is ignored
    r = subprocess.run(["gcc", *CFLAGS, "-fopenmp", "-o", tmp, *srcs, "-lm"], cwd=_HERE,
                       capture_output=True, text=True)
    if r.returncode != 0:
        subprocess.run(["gcc", *CFLAGS, "-o", tmp, *srcs, "-lm"], check=True, cwd=_HERE)
    os.replace(tmp, _SO)
    return _SO


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32),
                ("status", C.c_int32), ("tau0", C.c_double),
                ("tau_final", C.c_double), ("rho0", C.c_double),
                ("tau_max", C.c_double), ("alpha0", C.c_double),
                ("mu0", C.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            lp = C.POINTER(C.c_int64)
            ip = C.POINTER(C.c_int32)
            lib.orc_exdot.restype = C.c_double
            lib.orc_exdot.argtypes = [dp, dp, C.c_int64]
            lib.orc_exsum.restype = C.c_double
            lib.orc_exsum.argtypes = [dp, C.c_int64]
            lib.orc_exdot_limbs.restype = None
            lib.orc_exdot_limbs.argtypes = [dp, dp, C.c_int64, lp, ip]
            lib.orc_round_limbs.restype = C.c_double
            lib.orc_round_limbs.argtypes = [lp, C.c_int32]
            lib.orc_twosum.restype = None
            lib.orc_twosum.argtypes = [C.c_double, C.c_double, dp, dp]
            lib.orc_twoprod.restype = None
            lib.orc_twoprod.argtypes = [C.c_double, C.c_double, dp, dp]
            lib.orc_mul_add_unfused.restype = C.c_double
            lib.orc_mul_add_unfused.argtypes = [C.c_double] * 3
            lib.orc_spmv.restype = None
            lib.orc_spmv.argtypes = [C.c_int64, lp, ip, dp, dp, dp]
            lib.orc_jacobi_invd.restype = C.c_int
            lib.orc_jacobi_invd.argtypes = [C.c_int64, lp, ip, dp, dp, dp]
            lib.orc_jacobi_apply.restype = None
            lib.orc_jacobi_apply.argtypes = [C.c_int64, dp, dp, dp]
            lib.orc_fma_vec.restype = None
            lib.orc_fma_vec.argtypes = [C.c_int64, C.c_double, dp, dp, dp]
            lib.orc_set_threads.restype = None
            lib.orc_set_threads.argtypes = [C.c_int]
            lib.orc_get_threads.restype = C.c_int
            lib.orc_get_threads.argtypes = []
            lib.orc_solve.restype = C.c_int
            lib.orc_solve.argtypes = [C.c_int64, lp, ip, dp, dp, dp, dp,
                                      C.c_double, C.c_int32, C.c_int32, dp,
                                      C.POINTER(_Info), dp]
            _lib = lib
    return _lib


def _d(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    return a, a.ctypes.data_as(C.POINTER(C.c_double))


def _dn(a):
    if a is None:
        return None, None
    return _d(a)


def twosum(a: float, b: float):
    r, s = C.c_double(), C.c_double()
    _load().orc_twosum(a, b, C.byref(r), C.byref(s))
    return r.value, s.value


def twoprod(a: float, b: float):
    r, s = C.c_double(), C.c_double()
    _load().orc_twoprod(a, b, C.byref(r), C.byref(s))
    return r.value, s.value


def mul_add_unfused(a: float, b: float, c: float) -> float:
    return _load().orc_mul_add_unfused(a, b, c)


def fma_vec(a: float, x, y):
    """fma(a, x_i, y_i) element-wise, one rounding each."""
    x, xp = _d(x)
    y, yp = _d(y)
    out = np.empty_like(x)
    _load().orc_fma_vec(x.size, float(a), xp, yp, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def set_threads(n: int) -> None:
    """Threads of the oracle's loops and exact dots (1: sequential; results do
    not depend on it)."""
    _load().orc_set_threads(int(n))


def get_threads() -> int:
    return int(_load().orc_get_threads())


def exdot(x, y) -> float:
    x, xp = _d(x)
    y, yp = _d(y)
    assert x.shape == y.shape and x.ndim == 1
    return _load().orc_exdot(xp, yp, x.size)


def exsum(x) -> float:
    x, xp = _d(x)
    return _load().orc_exsum(xp, x.size)


def exdot_limbs(x, y):
    """The exact accumulator of one rank: (int64[DIGITS] digit values, flags)."""
    x, xp = _d(x)
    y, yp = _d(y)
    limbs = np.zeros(DIGITS, dtype=np.int64)
    flags = C.c_int32()
    _load().orc_exdot_limbs(xp, yp, x.size,
                            limbs.ctypes.data_as(C.POINTER(C.c_int64)),
                            C.byref(flags))
    return limbs, flags.value


def round_limbs(limbs, flags: int) -> float:
    limbs = np.ascontiguousarray(limbs, dtype=np.int64)
    assert limbs.size == DIGITS
    return _load().orc_round_limbs(limbs.ctypes.data_as(C.POINTER(C.c_int64)),
                                   int(flags))


def _csr(A):
    rowptr = np.ascontiguousarray(A.rowptr, dtype=np.int64)
    col = np.ascontiguousarray(A.col, dtype=np.int32)
    val = np.ascontiguousarray(A.val, dtype=np.float64)
    return (rowptr, col, val, rowptr.ctypes.data_as(C.POINTER(C.c_int64)),
            col.ctypes.data_as(C.POINTER(C.c_int32)),
            val.ctypes.data_as(C.POINTER(C.c_double)))


def spmv(A, x):
    rowptr, col, val, rp, cp, vp = _csr(A)
    x, xp = _d(x)
    y = np.empty(A.n, dtype=np.float64)
    _load().orc_spmv(A.n, rp, cp, vp, xp, y.ctypes.data_as(C.POINTER(C.c_double)))
    return y


def jacobi_invd(A, diag=None):
    rowptr, col, val, rp, cp, vp = _csr(A)
    diag, dgp = _dn(diag)
    invd = np.empty(A.n, dtype=np.float64)
    st = _load().orc_jacobi_invd(A.n, rp, cp, vp, dgp,
                                 invd.ctypes.data_as(C.POINTER(C.c_double)))
    if st != OK:
        raise ValueError("zero or missing diagonal entry")
    return invd


def jacobi_apply(invd, p):
    invd, ip_ = _d(invd)
    p, pp = _d(p)
    out = np.empty_like(p)
    _load().orc_jacobi_apply(p.size, ip_, pp, out.ctypes.data_as(C.POINTER(C.c_double)))
    return out


def solve(A, b, x0=None, diag=None, tol=1e-8, maxit=1000, variant=CLASSIC,
          history=True):
    """Run Fig. 2 (variant 0) or Fig. 4 (variant 1); returns a dict with x,
    iters, converged, status, tau0, tau_final, rho0, tau_max, alpha0, mu0 and
    hist (iters x HIST_W float64, or None)."""
    rowptr, col, val, rp, cp, vp = _csr(A)
    b, bp = _d(b)
    x0, x0p = _dn(x0)
    diag, dgp = _dn(diag)
    x = np.empty(A.n, dtype=np.float64)
    info = _Info()
    hist = np.empty((max(int(maxit), 1), HIST_W), dtype=np.float64) if history else None
    hp = hist.ctypes.data_as(C.POINTER(C.c_double)) if history else None
    _load().orc_solve(A.n, rp, cp, vp, bp, x0p, dgp, float(tol), int(maxit),
                      int(variant), x.ctypes.data_as(C.POINTER(C.c_double)),
                      C.byref(info), hp)
    return {
        "x": x, "iters": info.iters, "converged": info.converged,
        "status": info.status, "tau0": info.tau0, "tau_final": info.tau_final,
        "rho0": info.rho0, "tau_max": info.tau_max, "alpha0": info.alpha0,
        "mu0": info.mu0,
        "hist": hist[: info.iters].copy() if history else None,
    }
