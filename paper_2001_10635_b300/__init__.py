"""Interval reachability on one B300 GPU: Python binding of libreach.so.

A thin ctypes layer over the C ABI declared in ``include/reach.h``; every
function here has the name of the C entry point it calls and only marshals
arguments.  All computation happens in the CUDA kernels of ``csrc/``.  Arrays
may be numpy float64 arrays (host memory, copied by the library) or contiguous
float64 CUDA tensors (device memory, used in place).

Methods (Devonport, Khaled, Arcak, Zamani, "PIRK", 2020, Sec. 2.1):
``reach_mm`` (mixed monotonicity, Algorithm 3), ``reach_cgb`` (contraction /
growth bound, Algorithm 2), ``reach_mc`` (Monte Carlo, Algorithm 4), all over
fixed-step RK4 (Algorithm 1).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libreach.so")

TRAFFIC, KS, OSC, LINEAR, HEAT3D, QUAD = 0, 1, 2, 3, 4, 5
KINDS = {"traffic": TRAFFIC, "ks": KS, "osc": OSC, "linear": LINEAR, "heat": HEAT3D, "quad": QUAD}
OPT_KERNEL, OPT_STEPS_PER_LAUNCH, OPT_BLOCK, OPT_BATCH_CPT, OPT_TILE, OPT_MC_SB, OPT_MC_LAYOUT = 1, 2, 3, 4, 5, 6, 7
OPT_SERVE_QUEUE_BLOCKS, OPT_SERVE_QUEUE_N, OPT_SERVE_MAX_WIDE, OPT_BATCH_CLUSTER_FROM, OPT_ONE_LAUNCH = 8, 9, 10, 11, 12
OPT_SERVE_PRIORITY, OPT_SERVE_WIDE_EXCLUSIVE, OPT_SERVE_LIGHT = 13, 14, 15
BATCH_NO_AUTOTUNE = 1
STATUS = {0: "REACH_OK", -1: "REACH_EINVAL", -2: "REACH_ENOMEM", -3: "REACH_EADMIT",
          -4: "REACH_ENONFINITE", -5: "REACH_ETIMEOUT", -6: "REACH_ECUDA", -7: "REACH_ENODEV"}

_lib = None


class _TrafficParams(ctypes.Structure):
    _fields_ = [("cap", ctypes.c_double), ("v", ctypes.c_double), ("w", ctypes.c_double),
                ("xbar", ctypes.c_double), ("cgb_local", ctypes.c_int), ("sound", ctypes.c_int)]


class _HeatParams(ctypes.Structure):
    _fields_ = [("alpha", ctypes.c_double), ("l", ctypes.c_int64), ("open_face", ctypes.c_int)]


class _Query(ctypes.Structure):
    """reach_query (include/reach.h)."""
    _fields_ = [("sys", ctypes.c_void_p), ("method", ctypes.c_int), ("x0_lo", ctypes.c_void_p),
                ("x0_hi", ctypes.c_void_p), ("w_lo", ctypes.c_void_p), ("w_hi", ctypes.c_void_p),
                ("t_final", ctypes.c_double), ("dt", ctypes.c_double), ("lo", ctypes.c_void_p),
                ("hi", ctypes.c_void_p)]


class _Request(ctypes.Structure):
    """reach_request (include/reach.h)."""
    _fields_ = [("sys", ctypes.c_void_p), ("method", ctypes.c_int), ("x0_lo", ctypes.c_void_p),
                ("x0_hi", ctypes.c_void_p), ("w_lo", ctypes.c_void_p), ("w_hi", ctypes.c_void_p),
                ("t_final", ctypes.c_double), ("dt", ctypes.c_double), ("m", ctypes.c_int64),
                ("seed", ctypes.c_uint64), ("precision", ctypes.c_int), ("lo", ctypes.c_void_p),
                ("hi", ctypes.c_void_p)]


class ReachError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = int(code)
        super().__init__(f"{where}: {STATUS.get(self.code, self.code)} ({strerror(self.code)})")


def lib() -> ctypes.CDLL:
    """Load libreach.so; there is no fallback when it is missing."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is not built: run python -m paper_2001_10635_b300.build")
        try:   # share the CUDA runtime PyTorch loads, when it is present
            import torch  # noqa: F401
        except Exception:
            pass
        L = ctypes.CDLL(LIB_PATH)
        vp, i64, dbl = ctypes.c_void_p, ctypes.c_int64, ctypes.c_double
        L.reach_system_create.argtypes = [ctypes.c_int, i64, vp, ctypes.c_size_t, ctypes.POINTER(vp)]
        L.reach_system_destroy.argtypes = [vp]
        L.reach_system_dim.argtypes = [vp]
        L.reach_system_dim.restype = i64
        L.reach_input_dim.argtypes = [vp]
        L.reach_input_dim.restype = i64
        box = [vp, vp, vp, vp, vp, dbl, dbl]
        L.reach_mm.argtypes = box + [vp, vp, vp]
        L.reach_cgb.argtypes = box + [vp, vp, vp]
        L.reach_mc.argtypes = box + [i64, ctypes.c_uint64, ctypes.c_int, vp, vp, vp]
        L.reach_pipe.argtypes = [vp, ctypes.c_int, vp, vp, vp, vp, dbl, dbl, i64, vp, vp, vp]
        L.reach_mc_samples.argtypes = [i64, dbl, dbl]
        L.reach_mc_samples.restype = i64
        L.reach_set_option.argtypes = [ctypes.c_int, i64]
        L.reach_get_option.argtypes = [ctypes.c_int]
        L.reach_get_option.restype = i64
        L.reach_strerror.argtypes = [ctypes.c_int]
        L.reach_strerror.restype = ctypes.c_char_p
        L.reach_kernel_launches.restype = i64
        L.reach_batch_create.argtypes = [ctypes.POINTER(_Query), i64, ctypes.c_int, ctypes.POINTER(vp)]
        L.reach_batch_run.argtypes = [vp, vp, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dbl)]
        L.reach_batch_info.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(dbl)]
        L.reach_batch_layout.argtypes = [vp, ctypes.POINTER(i64), ctypes.POINTER(i64), ctypes.POINTER(dbl),
                                         ctypes.POINTER(dbl)]
        L.reach_batch_destroy.argtypes = [vp]
        L.reach_queue_create.argtypes = [ctypes.c_int, dbl, i64, ctypes.POINTER(vp)]
        L.reach_queue_submit.argtypes = [vp, ctypes.POINTER(_Query), ctypes.POINTER(i64)]
        L.reach_queue_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(ctypes.c_int)]
        L.reach_queue_start.argtypes = [vp, ctypes.c_int, ctypes.c_int]
        L.reach_queue_join.argtypes = [vp, dbl, ctypes.POINTER(ctypes.c_int)]
        L.reach_queue_stats.argtypes = [vp] + [ctypes.POINTER(i64)] * 3
        L.reach_queue_destroy.argtypes = [vp]
        L.reach_request_footprint.argtypes = [ctypes.POINTER(_Request)]
        L.reach_request_footprint.restype = i64
        L.reach_server_create.argtypes = [ctypes.c_int, i64, ctypes.POINTER(vp)]
        L.reach_server_submit.argtypes = [vp, ctypes.POINTER(_Request), ctypes.POINTER(i64)]
        L.reach_server_wait.argtypes = [vp, i64, dbl, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(dbl),
                                        ctypes.POINTER(dbl)]
        L.reach_server_stats.argtypes = [vp] + [ctypes.POINTER(i64)] * 5
        L.reach_server_destroy.argtypes = [vp]
        L.reach_server_queued.argtypes = [vp]
        L.reach_server_queued.restype = i64
        _lib = L
    return _lib


def strerror(code: int) -> str:
    return lib().reach_strerror(int(code)).decode()


def _check(rc: int, where: str):
    if rc != 0:
        raise ReachError(rc, where)


# ------------------------------------------------------------------ arrays
def _is_torch(a) -> bool:
    return type(a).__module__.startswith("torch")


def _ptr(a, n: int, name: str):
    """Address and keep-alive reference of a float64 contiguous vector."""
    if a is None:
        if n:
            raise ValueError(f"{name} is required")
        return None, None
    if _is_torch(a):
        import torch
        if a.dtype != torch.float64 or not a.is_contiguous() or a.numel() != n:
            raise ValueError(f"{name}: need a contiguous float64 tensor of {n} values")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if arr.size != n:
        raise ValueError(f"{name}: need {n} values, got {arr.size}")
    return arr.ctypes.data, arr


def _out(like, given, n: int, name: str):
    if given is not None:
        return given
    if _is_torch(like):
        import torch
        return torch.empty(n, dtype=torch.float64, device=like.device)
    return np.empty(n, dtype=np.float64)


def _stream(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return int(stream.cuda_stream)
    return int(stream)


# ------------------------------------------------------------------ systems
class System:
    """reach_system_create / reach_system_destroy."""

    _PARAM_FIELDS = {TRAFFIC: 4, KS: 4, OSC: 3, QUAD: 6}

    def __init__(self, kind, n: int, params=None, A=None):
        self.kind = KINDS[kind] if isinstance(kind, str) else int(kind)
        self.handle = ctypes.c_void_p()
        buf, nbytes = None, 0
        if self.kind == LINEAR:
            self._A = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(n, n))
            buf = (ctypes.c_void_p * 1)(self._A.ctypes.data)
            nbytes = ctypes.sizeof(ctypes.c_void_p)
        elif self.kind == TRAFFIC and params is not None and len(params) in (5, 6):
            cap, v, w, xbar, local = params[:5]
            sound = params[5] if len(params) == 6 else 0
            buf = ctypes.pointer(_TrafficParams(float(cap), float(v), float(w), float(xbar), int(bool(local)),
                                                int(bool(sound))))
            nbytes = ctypes.sizeof(_TrafficParams)
        elif self.kind == HEAT3D and params is not None:
            alpha, l, open_face = params
            buf = _HeatParams(float(alpha), int(l), int(bool(open_face)))
            nbytes = ctypes.sizeof(buf)
            buf = ctypes.pointer(buf)
        elif params is not None:
            vals = [float(v) for v in params]
            if len(vals) != self._PARAM_FIELDS[self.kind]:
                raise ValueError("wrong number of parameters")
            buf = (ctypes.c_double * len(vals))(*vals)
            nbytes = ctypes.sizeof(buf)
        rc = lib().reach_system_create(self.kind, int(n), ctypes.cast(buf, ctypes.c_void_p) if buf is not None
                                       else None, nbytes, ctypes.byref(self.handle))
        _check(rc, "reach_system_create")
        self.n = int(lib().reach_system_dim(self.handle))
        self.nw = int(lib().reach_input_dim(self.handle))

    def close(self):
        if self.handle:
            lib().reach_system_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def _box_args(sys: System, x0_lo, x0_hi, w_lo, w_hi):
    a = _ptr(x0_lo, sys.n, "x0_lo")
    b = _ptr(x0_hi, sys.n, "x0_hi")
    c = _ptr(w_lo, sys.nw, "w_lo") if sys.nw else (None, None)
    d = _ptr(w_hi, sys.nw, "w_hi") if sys.nw else (None, None)
    return a, b, c, d


def reach_mm(sys: System, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final: float, dt: float,
             lo=None, hi=None, stream=None):
    """Mixed-monotonicity box (Algorithm 3).  Returns (lo, hi)."""
    a, b, c, d = _box_args(sys, x0_lo, x0_hi, w_lo, w_hi)
    lo = _out(x0_lo, lo, sys.n, "lo")
    hi = _out(x0_lo, hi, sys.n, "hi")
    pl, _ = _ptr(lo, sys.n, "lo")
    ph, _ = _ptr(hi, sys.n, "hi")
    rc = lib().reach_mm(sys.handle, a[0], b[0], c[0], d[0], float(t_final), float(dt), pl, ph, _stream(stream))
    _check(rc, "reach_mm")
    return lo, hi


def reach_cgb(sys: System, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final: float, dt: float,
              lo=None, hi=None, stream=None):
    """Contraction / growth-bound box (Algorithm 2).  Returns (lo, hi)."""
    a, b, c, d = _box_args(sys, x0_lo, x0_hi, w_lo, w_hi)
    lo = _out(x0_lo, lo, sys.n, "lo")
    hi = _out(x0_lo, hi, sys.n, "hi")
    pl, _ = _ptr(lo, sys.n, "lo")
    ph, _ = _ptr(hi, sys.n, "hi")
    rc = lib().reach_cgb(sys.handle, a[0], b[0], c[0], d[0], float(t_final), float(dt), pl, ph, _stream(stream))
    _check(rc, "reach_cgb")
    return lo, hi


def reach_mc(sys: System, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final: float, dt: float, m: int,
             seed: int = 0, precision: int = 64, lo=None, hi=None, stream=None):
    """Monte Carlo box of m Philox samples (Algorithm 4).  Returns (lo, hi)."""
    a, b, c, d = _box_args(sys, x0_lo, x0_hi, w_lo, w_hi)
    lo = _out(x0_lo, lo, sys.n, "lo")
    hi = _out(x0_lo, hi, sys.n, "hi")
    pl, _ = _ptr(lo, sys.n, "lo")
    ph, _ = _ptr(hi, sys.n, "hi")
    rc = lib().reach_mc(sys.handle, a[0], b[0], c[0], d[0], float(t_final), float(dt), int(m),
                        int(seed) & (2**64 - 1), int(precision), pl, ph, _stream(stream))
    _check(rc, "reach_mc")
    return lo, hi


def reach_pipe(sys: System, method: str, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final: float, dt: float,
               every: int, stream=None):
    """The reach pipe (Sec. 5.5): boxes after every `every` steps, as two
    (rows, n) arrays (numpy for host inputs, CUDA tensors for device inputs)."""
    a, b, c, d = _box_args(sys, x0_lo, x0_hi, w_lo, w_hi)
    rows = int(round(t_final / dt)) // int(every)
    if _is_torch(x0_lo):
        import torch
        plo = torch.empty((rows, sys.n), dtype=torch.float64, device=x0_lo.device)
        phi = torch.empty_like(plo)
        pl, ph = plo.data_ptr(), phi.data_ptr()
    else:
        plo = np.empty((rows, sys.n))
        phi = np.empty((rows, sys.n))
        pl, ph = plo.ctypes.data, phi.ctypes.data
    rc = lib().reach_pipe(sys.handle, {"mm": 0, "cgb": 1}[method], a[0], b[0], c[0], d[0], float(t_final),
                          float(dt), int(every), pl, ph, _stream(stream))
    _check(rc, "reach_pipe")
    return plo, phi


def reach_mc_samples(n: int, eps: float, delta: float) -> int:
    return int(lib().reach_mc_samples(int(n), float(eps), float(delta)))


def reach_set_option(key: int, value: int):
    _check(lib().reach_set_option(int(key), int(value)), "reach_set_option")


def reach_get_option(key: int) -> int:
    return int(lib().reach_get_option(int(key)))


def reach_kernel_launches() -> int:
    return int(lib().reach_kernel_launches())


# ------------------------------------------------------------------ batches
class Batch:
    """reach_batch_create / _run / _info / _destroy.

    queries: sequence of dicts with keys sys (System), method ("mm" | "cgb"),
    x0_lo, x0_hi, w_lo, w_hi, t_final, dt, and optionally lo, hi (allocated like
    x0_lo when absent).  The arrays are kept alive by the batch; update input
    contents in place between runs."""

    def __init__(self, queries, autotune: bool = True):
        self._keep = []
        arr = (_Query * len(queries))()
        self.outputs = []
        for k, q in enumerate(queries):
            sys_ = q["sys"]
            a = _ptr(q["x0_lo"], sys_.n, "x0_lo")
            b = _ptr(q["x0_hi"], sys_.n, "x0_hi")
            c = _ptr(q.get("w_lo"), sys_.nw, "w_lo") if sys_.nw else (None, None)
            d = _ptr(q.get("w_hi"), sys_.nw, "w_hi") if sys_.nw else (None, None)
            lo = _out(q["x0_lo"], q.get("lo"), sys_.n, "lo")
            hi = _out(q["x0_lo"], q.get("hi"), sys_.n, "hi")
            pl, _ = _ptr(lo, sys_.n, "lo")
            ph, _ = _ptr(hi, sys_.n, "hi")
            self._keep += [sys_, a[1], b[1], c[1], d[1], lo, hi]
            self.outputs.append((lo, hi))
            method = {"mm": 0, "cgb": 1}[q["method"]] if isinstance(q["method"], str) else int(q["method"])
            arr[k] = _Query(sys_.handle.value, method, a[0], b[0], c[0], d[0], float(q["t_final"]),
                            float(q["dt"]), pl, ph)
        self.count = len(queries)
        self.handle = ctypes.c_void_p()
        rc = lib().reach_batch_create(arr, self.count, 0 if autotune else BATCH_NO_AUTOTUNE,
                                      ctypes.byref(self.handle))
        _check(rc, "reach_batch_create")

    def run(self, stream=None, check: bool = True):
        """Run once; returns (status per query, completion seconds per query)."""
        st = np.zeros(self.count, dtype=np.int32)
        fin = np.zeros(self.count, dtype=np.float64)
        rc = lib().reach_batch_run(self.handle, _stream(stream),
                                   st.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                                   fin.ctypes.data_as(ctypes.POINTER(ctypes.c_double)))
        if check:
            _check(rc, "reach_batch_run")
        return st, fin

    def info(self):
        cpt = ctypes.c_int64()
        kern = ctypes.c_int64()
        tune = (ctypes.c_double * 4)()
        _check(lib().reach_batch_info(self.handle, ctypes.byref(cpt), ctypes.byref(kern), tune), "reach_batch_info")
        return {"cpt": cpt.value, "kernels": kern.value, "tune_ms": dict(zip((2, 4, 8, 16), list(tune)))}

    def layout(self):
        """The tuned layout: cpt, cluster_from (components), create_s, and the
        candidates' timings (ms)."""
        cpt, cf = ctypes.c_int64(), ctypes.c_int64()
        cs = ctypes.c_double()
        tune = (ctypes.c_double * 6)()
        _check(lib().reach_batch_layout(self.handle, ctypes.byref(cpt), ctypes.byref(cf), ctypes.byref(cs), tune),
               "reach_batch_layout")
        names = ("cpt2", "cpt4", "cpt8", "cpt16", "cluster_from_4096", "cluster_from_2048")
        return {"cpt": cpt.value, "cluster_from": cf.value, "create_s": cs.value,
                "tune_ms": {k: v for k, v in zip(names, list(tune)) if v > 0}}

    def close(self):
        if self.handle:
            lib().reach_batch_destroy(self.handle)
            self.handle = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ device work queue
QUEUE_MAX_N = 4096
_KIND_IDS = {"traffic": 0, "ks": 1, "osc": 2, "linear": 3, "heat": 4}


class Queue:
    """reach_queue_create / _submit / _wait / _start / _join / _stats / _destroy."""

    def __init__(self, max_blocks: int = 64, idle_s: float = 0.005, arena_bytes: int = 256 << 20):
        self.handle = ctypes.c_void_p()
        _check(lib().reach_queue_create(int(max_blocks), float(idle_s), int(arena_bytes), ctypes.byref(self.handle)),
               "reach_queue_create")
        self._keep = {}

    def submit(self, sys_, method, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final, dt, lo=None, hi=None):
        """Returns (ticket, (lo, hi)); the outputs are complete after wait(ticket)."""
        a = _ptr(x0_lo, sys_.n, "x0_lo")
        b = _ptr(x0_hi, sys_.n, "x0_hi")
        c = _ptr(w_lo, sys_.nw, "w_lo") if sys_.nw else (None, None)
        d = _ptr(w_hi, sys_.nw, "w_hi") if sys_.nw else (None, None)
        lo = _out(x0_lo, lo, sys_.n, "lo")
        hi = _out(x0_lo, hi, sys_.n, "hi")
        q = _Query(sys_.handle.value, _METHOD_IDS[method] if isinstance(method, str) else int(method), a[0], b[0],
                   c[0], d[0], float(t_final), float(dt), _ptr(lo, sys_.n, "lo")[0], _ptr(hi, sys_.n, "hi")[0])
        t = ctypes.c_int64()
        _check(lib().reach_queue_submit(self.handle, ctypes.byref(q), ctypes.byref(t)), "reach_queue_submit")
        self._keep[t.value] = (sys_, lo, hi)
        return t.value, (lo, hi)

    def wait(self, ticket: int, timeout_s: float = 600.0) -> int:
        """Returns the query's status; raises ReachError(REACH_ETIMEOUT) on timeout."""
        st = ctypes.c_int()
        _check(lib().reach_queue_wait(self.handle, int(ticket), float(timeout_s), ctypes.byref(st)),
               "reach_queue_wait")
        self._keep.pop(ticket, None)
        return st.value

    def start(self, kind: str, blocks: int):
        _check(lib().reach_queue_start(self.handle, _KIND_IDS[kind], int(blocks)), "reach_queue_start")

    def join(self, timeout_s: float = 60.0) -> int:
        """Waits for every block to leave; returns the last launch's exit status."""
        st = ctypes.c_int()
        _check(lib().reach_queue_join(self.handle, float(timeout_s), ctypes.byref(st)), "reach_queue_join")
        return st.value

    def stats(self):
        v = [ctypes.c_int64() for _ in range(3)]
        _check(lib().reach_queue_stats(self.handle, *[ctypes.byref(x) for x in v]), "reach_queue_stats")
        return dict(zip(("in_flight", "alive_blocks", "launched_blocks"), [x.value for x in v]))

    def close(self):
        if self.handle:
            lib().reach_queue_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ------------------------------------------------------------------ serving
_METHOD_IDS = {"mm": 0, "cgb": 1, "mc": 2}


class Server:
    """reach_server_create / _submit / _wait / _stats / _destroy."""

    def __init__(self, slots: int = 8, hbm_budget_bytes: int = 64 << 30):
        self.handle = ctypes.c_void_p()
        _check(lib().reach_server_create(int(slots), int(hbm_budget_bytes), ctypes.byref(self.handle)),
               "reach_server_create")
        self._keep = {}

    @staticmethod
    def _request(sys_, method, x0_lo, x0_hi, w_lo, w_hi, t_final, dt, m, seed, precision, lo, hi):
        a = _ptr(x0_lo, sys_.n, "x0_lo")
        b = _ptr(x0_hi, sys_.n, "x0_hi")
        c = _ptr(w_lo, sys_.nw, "w_lo") if sys_.nw else (None, None)
        d = _ptr(w_hi, sys_.nw, "w_hi") if sys_.nw else (None, None)
        lo = _out(x0_lo, lo, sys_.n, "lo")
        hi = _out(x0_lo, hi, sys_.n, "hi")
        r = _Request(sys_.handle.value, _METHOD_IDS.get(method, method), a[0], b[0], c[0], d[0], float(t_final),
                     float(dt), int(m), int(seed) & (2**64 - 1), int(precision), _ptr(lo, sys_.n, "lo")[0],
                     _ptr(hi, sys_.n, "hi")[0])
        return r, (sys_, a[1], b[1], c[1], d[1], lo, hi)

    def submit(self, sys_, method, x0_lo, x0_hi, w_lo=None, w_hi=None, *, t_final, dt, m=0, seed=0,
               precision=64, lo=None, hi=None):
        """Returns (ticket, (lo, hi)); the outputs are complete after wait(ticket)."""
        r, keep = self._request(sys_, method, x0_lo, x0_hi, w_lo, w_hi, t_final, dt, m, seed, precision, lo, hi)
        t = ctypes.c_int64()
        _check(lib().reach_server_submit(self.handle, ctypes.byref(r), ctypes.byref(t)), "reach_server_submit")
        self._keep[t.value] = keep
        return t.value, (keep[5], keep[6])

    def wait(self, ticket: int, timeout_s: float = 600.0):
        """Returns (status, queue_s, run_s); raises ReachError(REACH_ETIMEOUT) on timeout."""
        st = ctypes.c_int()
        q = ctypes.c_double()
        r = ctypes.c_double()
        rc = lib().reach_server_wait(self.handle, int(ticket), float(timeout_s), ctypes.byref(st), ctypes.byref(q),
                                     ctypes.byref(r))
        _check(rc, "reach_server_wait")
        self._keep.pop(ticket, None)
        return st.value, q.value, r.value

    def queued(self) -> int:
        """Requests that went to the server's device work queue."""
        return int(lib().reach_server_queued(self.handle))

    def stats(self):
        v = [ctypes.c_int64() for _ in range(5)]
        _check(lib().reach_server_stats(self.handle, *[ctypes.byref(x) for x in v]), "reach_server_stats")
        return dict(zip(("waiting", "running", "done", "bytes_in_use", "bytes_peak"), [x.value for x in v]))

    def close(self):
        if self.handle:
            lib().reach_server_destroy(self.handle)
            self.handle = ctypes.c_void_p()
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def reach_request_footprint(sys_, method, m=0, precision=64) -> int:
    r = _Request(sys_.handle.value, _METHOD_IDS.get(method, method), None, None, None, None, 1.0, 1.0, int(m), 0,
                 int(precision), None, None)
    return int(lib().reach_request_footprint(ctypes.byref(r)))
