"""Python binding of librbs.so, the GB300 reproducible PBiCGStab library.

Argument marshalling only: every step of the computation runs in the CUDA
kernels behind the C ABI of include/rbs.h, under the same names. PyTorch
provides device memory and streams; numpy arrays are passed as host pointers
(the library stages them itself). If the compiled library is missing, every
call raises: there is no CPU fallback.

Method: Iakymchuk & Aliaga, arXiv 2302.04180 -- exact dot (Sec. 2, Sec. 3.2),
fma SpMV, Jacobi and axpy-like updates (Sec. 3.3, Sec. 4.1), PBiCGStab (Fig. 2)
and pipelined PBiCGStab (Fig. 4).
"""
from __future__ import annotations

import ctypes as C
import os
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librbs.so")

RBS_OK, RBS_EINVAL, RBS_ENOMEM, RBS_ECUDA, RBS_EBREAKDOWN, RBS_ENAN, RBS_ETIMEOUT = range(7)
RBS_CLASSIC, RBS_PIPELINED = 0, 1
RBS_DOT_EXACT, RBS_DOT_PLAIN = 0, 1
RBS_LOOP_GRAPH, RBS_LOOP_HOST = 0, 1
RBS_LIMBS = 136
RBS_NOALLOC_MAX_DOTS = 6
RBS_HIST_W = 12
RBS_PROF_KINDS = 8
PROF_KIND_NAMES = ("k1_spmv_dot", "vec", "setup", "spmv", "pipe_vec_dot", "k3_spmv_dot2", "k4_vec_dot2")

# every symbol include/rbs.h declares
EXPORTS = ("rbs_exdot", "rbs_exdot_multi", "rbs_exdot_noalloc", "rbs_exdot_partial", "rbs_round_limbs",
           "rbs_spmv_csr", "rbs_jacobi_invd", "rbs_jacobi_apply", "rbs_solve",
           "rbs_solve_ex", "rbs_solve_batched", "rbs_solve_batched_ex", "rbs_batch_tune", "rbs_fpe_dot",
           "rbs_server_create", "rbs_server_submit", "rbs_server_poll", "rbs_server_wait",
           "rbs_server_request_stats", "rbs_server_stats", "rbs_server_destroy", "rbs_stream_status", "rbs_release", "rbs_set_param",
           "rbs_get_param", "rbs_last_error", "rbs_version")


class RbsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"rbs error {code}: {msg}")
        self.code = code


class _Csr(C.Structure):
    _fields_ = [("n", C.c_int64), ("nnz", C.c_int64), ("rowptr", C.c_void_p),
                ("col", C.c_void_p), ("val", C.c_void_p)]


class _Opts(C.Structure):
    _fields_ = [("dot_mode", C.c_int32), ("check_every", C.c_int32),
                ("profile", C.c_int32), ("loop_mode", C.c_int32)]


class _Info(C.Structure):
    _fields_ = [("iters", C.c_int32), ("converged", C.c_int32), ("status", C.c_int32),
                ("reserved", C.c_int32), ("tau0", C.c_double), ("tau_final", C.c_double),
                ("rho0", C.c_double), ("tau_max", C.c_double), ("alpha0", C.c_double),
                ("mu0", C.c_double)]


class _System(C.Structure):
    _fields_ = [("A", _Csr), ("b", C.c_void_p), ("x0", C.c_void_p), ("jacobi_diag", C.c_void_p),
                ("x", C.c_void_p), ("tol", C.c_double), ("maxit", C.c_int32), ("variant", C.c_int32)]


class _ReqStats(C.Structure):
    _fields_ = [("admit_step", C.c_int64), ("finish_step", C.c_int64), ("active_at_admit", C.c_int32),
                ("done", C.c_int32)]


class _SrvCounters(C.Structure):
    _fields_ = [(k, C.c_int64) for k in ("steps", "completed", "peak_active", "pending", "budget_in_use",
                                         "pool_reserved", "pool_reserved_peak")]


class _Hist(C.Structure):
    _fields_ = [("cap", C.c_int32), ("len", C.c_int32), ("rec", C.c_void_p)]


class _Prof(C.Structure):
    _fields_ = [("launches", C.c_int64 * RBS_PROF_KINDS), ("ms", C.c_double * RBS_PROF_KINDS),
                ("trace_cap", C.c_int32), ("trace_len", C.c_int32), ("trace_kind", C.c_void_p),
                ("trace_iter", C.c_void_p), ("trace_ms", C.c_void_p)]


_lock = threading.Lock()
_lib = None


def load(path: str | None = None):
    """Load librbs.so (built by paper_2302_04180_gb300.build). Raises if absent."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        p = path or LIB_PATH
        if not os.path.exists(p):
            raise RuntimeError(f"librbs.so not found at {p}: build it with "
                               "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(p)
        vp, i64, i32, dbl = C.c_void_p, C.c_int64, C.c_int32, C.c_double
        sig = {
            "rbs_exdot": [vp, vp, i64, vp, vp],
            "rbs_exdot_multi": [C.c_int, vp, vp, i64, vp, vp],
            "rbs_exdot_noalloc": [C.c_int, vp, vp, i64, vp, vp],
            "rbs_exdot_partial": [vp, vp, i64, vp, vp, vp],
            "rbs_round_limbs": [vp, vp, vp, vp],
            "rbs_spmv_csr": [C.POINTER(_Csr), vp, vp, vp],
            "rbs_jacobi_invd": [C.POINTER(_Csr), vp, vp, vp],
            "rbs_jacobi_apply": [i64, vp, vp, vp, vp],
            "rbs_solve": [C.POINTER(_Csr), vp, vp, vp, dbl, i32, i32, vp, C.POINTER(_Info),
                          C.POINTER(_Hist), vp],
            "rbs_solve_ex": [C.POINTER(_Csr), vp, vp, vp, dbl, i32, i32, C.POINTER(_Opts), vp,
                             C.POINTER(_Info), C.POINTER(_Hist), C.POINTER(_Prof), vp],
            "rbs_fpe_dot": [vp, vp, i64, vp, vp, vp],
            "rbs_server_create": [i32, i32, i64, i64, C.POINTER(vp)],
            "rbs_server_submit": [vp, C.POINTER(_System), C.POINTER(i64)],
            "rbs_server_poll": [vp, i64, C.POINTER(i32), C.POINTER(_Info), C.POINTER(dbl), C.POINTER(dbl)],
            "rbs_server_wait": [vp, i64, C.POINTER(_Info), C.POINTER(dbl), C.POINTER(dbl)],
            "rbs_server_request_stats": [vp, i64, C.POINTER(_ReqStats)],
            "rbs_server_stats": [vp, C.POINTER(_SrvCounters)],
            "rbs_server_destroy": [vp],
            "rbs_solve_batched": [C.c_int32, C.POINTER(_System), C.POINTER(_Info), C.POINTER(_Hist), vp],
            "rbs_solve_batched_ex": [C.c_int32, C.POINTER(_System), C.POINTER(_Info), C.POINTER(_Hist),
                                     C.POINTER(_Schedule), vp],
            "rbs_batch_tune": [C.c_int32, C.POINTER(_System), C.POINTER(_Info), C.c_int32,
                               C.POINTER(_Schedule), vp],
            "rbs_stream_status": [vp],
            "rbs_release": [],
            "rbs_set_param": [C.c_char_p, i64],
            "rbs_get_param": [C.c_char_p],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = C.c_int
        lib.rbs_get_param.restype = C.c_int64
        lib.rbs_last_error.restype = C.c_char_p
        lib.rbs_last_error.argtypes = []
        lib.rbs_version.restype = C.c_char_p
        lib.rbs_version.argtypes = []
        _lib = lib
        return lib


def _check(rc):
    if rc != RBS_OK:
        raise RbsError(rc, load().rbs_last_error().decode())
    return rc


def _ptr(a):
    """Raw address of a torch tensor or numpy array (None -> NULL)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        assert a.flags["C_CONTIGUOUS"]
        return a.ctypes.data
    assert a.is_contiguous()
    return a.data_ptr()


def _stream(stream, *tensors):
    if stream is not None:
        return stream if isinstance(stream, int) else stream.cuda_stream
    for t in tensors:
        if t is not None and not isinstance(t, np.ndarray) and t.is_cuda:
            import torch
            return torch.cuda.current_stream(t.device).cuda_stream
    return None


@dataclass
class DeviceCSR:
    """CSR on the device as torch tensors (int64 rowptr, int32 col, float64 val)."""
    n: int
    rowptr: object
    col: object
    val: object

    @property
    def nnz(self) -> int:
        return int(self.col.numel())


def to_device(A, device="cuda") -> DeviceCSR:
    import torch
    return DeviceCSR(int(A.n), torch.as_tensor(np.asarray(A.rowptr, np.int64)).to(device),
                     torch.as_tensor(np.asarray(A.col, np.int32)).to(device),
                     torch.as_tensor(np.asarray(A.val, np.float64)).to(device))


def _csr(A):
    return _Csr(int(A.n), int(A.nnz), _ptr(A.rowptr), _ptr(A.col), _ptr(A.val))


# ---- entry points (same names as the C ABI) ----------------------------------------

def rbs_version() -> str:
    return load().rbs_version().decode()


def rbs_set_param(name: str, value: int) -> None:
    _check(load().rbs_set_param(name.encode(), int(value)))


def rbs_get_param(name: str) -> int:
    return int(load().rbs_get_param(name.encode()))


def rbs_release() -> None:
    _check(load().rbs_release())


def rbs_stream_status(stream=None) -> None:
    _check(load().rbs_stream_status(_stream(stream)))


def rbs_exdot(x, y, out=None, stream=None):
    """RN(sum x*y), exact. Torch tensors: returns a 1-element device tensor
    (asynchronous) unless `out` is given. numpy arrays: returns a float."""
    n = int(x.shape[0])
    if isinstance(x, np.ndarray) and isinstance(y, np.ndarray) and out is None:
        res = np.zeros(1, dtype=np.float64)
        _check(load().rbs_exdot(_ptr(x), _ptr(y), n, res.ctypes.data, _stream(stream)))
        return float(res[0])
    if out is None:
        import torch
        dev = x.device if not isinstance(x, np.ndarray) else y.device
        out = torch.empty(1, dtype=torch.float64, device=dev)
    _check(load().rbs_exdot(_ptr(x), _ptr(y), n, _ptr(out), _stream(stream, x, y, out)))
    return out


def rbs_exdot_multi(xs, ys, out=None, stream=None):
    k = len(xs)
    n = int(xs[0].shape[0])
    xa = (C.c_void_p * k)(*[_ptr(t) for t in xs])
    ya = (C.c_void_p * k)(*[_ptr(t) for t in ys])
    if out is None:
        import torch
        out = torch.empty(k, dtype=torch.float64, device=xs[0].device)
    _check(load().rbs_exdot_multi(k, xa, ya, n, _ptr(out), _stream(stream, xs[0], out)))
    return out


def rbs_fpe_dot(x, y, stream=None):
    """Lightweight FPE-8 dot: returns (value, fell_back). The value is always
    the correctly rounded dot (the exact path is taken when the expansions
    cannot hold every bit)."""
    res = np.zeros(1, dtype=np.float64)
    fb = C.c_int32(0)
    _check(load().rbs_fpe_dot(_ptr(x), _ptr(y), int(x.shape[0]), res.ctypes.data, C.byref(fb),
                              _stream(stream, x, y)))
    return float(res[0]), bool(fb.value)


def rbs_exdot_noalloc(xs, ys, out, stream=None):
    """Allocation-free k exact dots: `out` (k float64) and all operands must be
    device tensors; nothing is allocated on any path of this call."""
    k = len(xs)
    xa = (C.c_void_p * k)(*[_ptr(t) for t in xs])
    ya = (C.c_void_p * k)(*[_ptr(t) for t in ys])
    _check(load().rbs_exdot_noalloc(k, xa, ya, int(xs[0].shape[0]), _ptr(out),
                                    _stream(stream, xs[0], out)))
    return out


def rbs_exdot_partial(x, y, limbs=None, flags=None, stream=None):
    import torch
    if limbs is None:
        limbs = torch.empty(RBS_LIMBS, dtype=torch.int64, device=x.device)
    if flags is None:
        flags = torch.empty(1, dtype=torch.int32, device=x.device)
    _check(load().rbs_exdot_partial(_ptr(x), _ptr(y), int(x.shape[0]), _ptr(limbs), _ptr(flags),
                                    _stream(stream, x)))
    return limbs, flags


def rbs_round_limbs(limbs, flags, out=None, stream=None):
    import torch
    if out is None:
        out = torch.empty(1, dtype=torch.float64, device=limbs.device)
    _check(load().rbs_round_limbs(_ptr(limbs), _ptr(flags), _ptr(out), _stream(stream, limbs)))
    return out


def rbs_spmv_csr(A, x, y=None, stream=None):
    if y is None:
        import torch
        y = torch.empty(A.n, dtype=torch.float64, device=x.device)
    csr = _csr(A)
    _check(load().rbs_spmv_csr(C.byref(csr), _ptr(x), _ptr(y), _stream(stream, x, y)))
    return y


def rbs_jacobi_invd(A, diag=None, invd=None, stream=None):
    import torch
    if invd is None:
        invd = torch.empty(A.n, dtype=torch.float64, device=A.val.device)
    csr = _csr(A)
    _check(load().rbs_jacobi_invd(C.byref(csr), _ptr(diag), _ptr(invd), _stream(stream, invd)))
    return invd


def rbs_jacobi_apply(invd, p, phat=None, stream=None):
    import torch
    if phat is None:
        phat = torch.empty_like(p)
    _check(load().rbs_jacobi_apply(int(p.shape[0]), _ptr(invd), _ptr(p), _ptr(phat),
                                   _stream(stream, p)))
    return phat


def rbs_solve(A, b, x0=None, jacobi_diag=None, tol=1e-8, maxit=1000, variant=RBS_CLASSIC,
              x_out=None, history=True, dot_mode=RBS_DOT_EXACT, check_every=0,
              profile=False, loop_mode=0, stream=None, raise_on_status=False, trace=0):
    """Reproducible PBiCGStab (variant 0, Fig. 2) or p-PBiCGStab (variant 1, Fig. 4).
    Returns a dict: x, iters, converged, status, tau0, tau_final, rho0, tau_max,
    alpha0, mu0, hist (iters x 12 float64) and prof (per kernel kind: launches
    and milliseconds of the launches that ran). With profile and trace = N > 0,
    also trace: up to N per-launch (kind name, iteration, ms) tuples in enqueue
    order."""
    n = int(A.n)
    if x_out is None:
        if isinstance(b, np.ndarray):
            x_out = np.empty(n, dtype=np.float64)
        else:
            import torch
            x_out = torch.empty(n, dtype=torch.float64, device=b.device)
    cap = max(int(maxit), 1) if history else 0
    rec = np.empty((max(cap, 1), RBS_HIST_W), dtype=np.float64)
    h = _Hist(cap, 0, rec.ctypes.data)
    info = _Info()
    opts = _Opts(int(dot_mode), int(check_every), 1 if profile else 0, int(loop_mode))
    prof = _Prof()
    tcap = int(trace) if profile else 0
    t_kind = np.zeros(max(tcap, 1), dtype=np.int32)
    t_iter = np.zeros(max(tcap, 1), dtype=np.int32)
    t_ms = np.zeros(max(tcap, 1), dtype=np.float32)
    if tcap > 0:
        prof.trace_cap = tcap
        prof.trace_kind, prof.trace_iter, prof.trace_ms = t_kind.ctypes.data, t_iter.ctypes.data, t_ms.ctypes.data
    csr = _csr(A)
    rc = load().rbs_solve_ex(C.byref(csr), _ptr(b), _ptr(x0), _ptr(jacobi_diag), float(tol),
                             int(maxit), int(variant), C.byref(opts), _ptr(x_out),
                             C.byref(info), C.byref(h) if history else None, C.byref(prof),
                             _stream(stream, b, x_out, A.val if hasattr(A.val, "is_cuda") else None))
    if rc not in (RBS_OK, RBS_EBREAKDOWN, RBS_ENAN) or (raise_on_status and rc != RBS_OK):
        _check(rc)
    return {
        "x": x_out, "iters": info.iters, "converged": info.converged, "status": info.status,
        "tau0": info.tau0, "tau_final": info.tau_final, "rho0": info.rho0,
        "tau_max": info.tau_max, "alpha0": info.alpha0, "mu0": info.mu0,
        "hist": rec[: h.len].copy() if history else None,
        "prof": {PROF_KIND_NAMES[k]: (int(prof.launches[k]), float(prof.ms[k]))
                 for k in range(len(PROF_KIND_NAMES))} if profile else None,
        "trace": [(PROF_KIND_NAMES[int(t_kind[j])] if 0 <= t_kind[j] < len(PROF_KIND_NAMES) else str(int(t_kind[j])),
                   int(t_iter[j]), float(t_ms[j])) for j in range(prof.trace_len)] if tcap > 0 else None,
    }


class _Schedule(C.Structure):
    _fields_ = [("cluster", C.c_int32), ("pad", C.c_int32), ("split", C.c_int64), ("ms", C.c_double)]


def _systems(systems, history):
    nsys = len(systems)
    arr = (_System * nsys)()
    hists = (_Hist * nsys)()
    recs = []
    for i, sd in enumerate(systems):
        A = sd["A"]
        arr[i] = _System(_csr(A), _ptr(sd["b"]), _ptr(sd.get("x0")), _ptr(sd.get("jacobi_diag")),
                         _ptr(sd.get("x")), float(sd.get("tol", 1e-8)), int(sd.get("maxit", 1000)),
                         int(sd.get("variant", RBS_CLASSIC)))
        cap = max(int(sd.get("maxit", 1000)), 1) if history else 0
        rec = np.empty((max(cap, 1), RBS_HIST_W), dtype=np.float64)
        recs.append(rec)
        hists[i] = _Hist(cap, 0, rec.ctypes.data)
    return arr, hists, recs


def rbs_solve_batched(systems, history=True, stream=None, schedule=None):
    """Solve many independent systems in one persistent launch. `systems` is a
    list of dicts with keys A (DeviceCSR), b, x (device tensors), and optional
    x0, jacobi_diag, tol (1e-8), maxit (1000), variant (0). `schedule`: a dict
    {"cluster", "split"} (see rbs_batch_schedule), None for the tuned or default
    one. Returns a list of per-system dicts like rbs_solve's (x is the caller's
    tensor)."""
    nsys = len(systems)
    arr, hists, recs = _systems(systems, history)
    infos = (_Info * nsys)()
    first = systems[0]["b"] if nsys else None
    sch = None
    if schedule is not None:
        sch = _Schedule(int(schedule["cluster"]), 0, int(schedule.get("split", 0)), 0.0)
    rc = load().rbs_solve_batched_ex(nsys, arr, infos, hists if history else None,
                                     C.byref(sch) if sch is not None else None, _stream(stream, first))
    # RBS_EINVAL with per-system statuses marks invalid systems (the others are
    # solved); without any, the call itself was rejected (e.g. its schedule)
    if rc not in (RBS_OK, RBS_EINVAL) or (rc == RBS_EINVAL and
                                          not any(infos[i].status == RBS_EINVAL for i in range(nsys))):
        _check(rc)
    out = []
    for i in range(nsys):
        I = infos[i]
        out.append({"x": systems[i]["x"], "iters": I.iters, "converged": I.converged,
                    "status": I.status, "tau0": I.tau0, "tau_final": I.tau_final, "rho0": I.rho0,
                    "tau_max": I.tau_max, "alpha0": I.alpha0, "mu0": I.mu0,
                    "hist": recs[i][: hists[i].len].copy() if history else None})
    return out


def rbs_batch_tune(systems, prev=None, proxy_iters=24, stream=None):
    """Autotune the batched schedule (see rbs_batch_tune in include/rbs.h).
    prev: the result list of an earlier rbs_solve_batched of the same systems
    (its iteration counts weight the proxy solves). Returns {"cluster",
    "split", "ms"}; later rbs_solve_batched calls on this device use it."""
    nsys = len(systems)
    arr, _, _ = _systems(systems, False)
    pinfo = None
    if prev is not None:
        pinfo = (_Info * nsys)()
        for i, r in enumerate(prev):
            pinfo[i].iters = int(r["iters"])
    best = _Schedule()
    first = systems[0]["b"] if nsys else None
    _check(load().rbs_batch_tune(nsys, arr, pinfo, int(proxy_iters), C.byref(best), _stream(stream, first)))
    return {"cluster": best.cluster, "split": best.split, "ms": best.ms}


class RbsServer:
    """Per-iteration continuous-batching solve server (see rbs_server_create in
    include/rbs.h). submit(system_dict) -> ticket; wait(ticket) / poll(ticket) ->
    result dict with latency_s and queue_s; request_stats(ticket) and stats()
    report where requests ran and the server's counters. Keep each system's
    tensors alive until it is done."""

    def __init__(self, engines=1, max_active=64, budget_bytes=16 << 30, rows_per_block=0):
        self._h = C.c_void_p()
        _check(load().rbs_server_create(int(engines), int(max_active), int(budget_bytes),
                                        int(rows_per_block), C.byref(self._h)))
        self._keep = {}

    def submit(self, sd) -> int:
        sysc = _System(_csr(sd["A"]), _ptr(sd["b"]), _ptr(sd.get("x0")), _ptr(sd.get("jacobi_diag")),
                       _ptr(sd["x"]), float(sd.get("tol", 1e-8)), int(sd.get("maxit", 1000)),
                       int(sd.get("variant", RBS_CLASSIC)))
        t = C.c_int64()
        _check(load().rbs_server_submit(self._h, C.byref(sysc), C.byref(t)))
        self._keep[t.value] = sd
        return t.value

    def _result(self, ticket, info, lat, que):
        sd = self._keep.pop(ticket, None)
        err = load().rbs_last_error().decode() if info.status != RBS_OK else ""
        return {"x": sd["x"] if sd else None, "iters": info.iters, "converged": info.converged,
                "status": info.status, "latency_s": lat.value, "queue_s": que.value, "error": err}

    def wait(self, ticket):
        info, lat, que = _Info(), C.c_double(), C.c_double()
        _check(load().rbs_server_wait(self._h, int(ticket), C.byref(info), C.byref(lat), C.byref(que)))
        return self._result(ticket, info, lat, que)

    def poll(self, ticket):
        done, info, lat, que = C.c_int32(), _Info(), C.c_double(), C.c_double()
        _check(load().rbs_server_poll(self._h, int(ticket), C.byref(done), C.byref(info),
                                      C.byref(lat), C.byref(que)))
        return self._result(ticket, info, lat, que) if done.value else None

    def request_stats(self, ticket):
        r = _ReqStats()
        _check(load().rbs_server_request_stats(self._h, int(ticket), C.byref(r)))
        return {"admit_step": r.admit_step, "finish_step": r.finish_step,
                "active_at_admit": r.active_at_admit, "done": bool(r.done)}

    def stats(self):
        c = _SrvCounters()
        _check(load().rbs_server_stats(self._h, C.byref(c)))
        return {k: int(getattr(c, k)) for k, _ in _SrvCounters._fields_}

    def close(self):
        if self._h:
            load().rbs_server_destroy(self._h)
            self._h = C.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()
