"""Plain FP64 CPU oracle for the PIRK interval-reachability methods.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers.  The product library
never imports this package and shares no code with it.

The arithmetic lives in ``oracle.c`` (single-threaded C, ``-O2
-ffp-contract=off``); this module only marshals numpy arrays through ctypes.
Every function of ``oracle.c`` cites the passage of the paper it follows and
lists the readings taken where the paper is garbled or silent.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
# a test may point the wrapper at a separately compiled copy (mutation tests)
_LIB_OVERRIDE = os.environ.get("REACH_ORACLE_LIB")

MM, CGB, MC = 0, 1, 2
TRAFFIC, KS, OSC, LINEAR, HEAT, QUAD = 0, 1, 2, 3, 4, 5
METHODS = {"mm": MM, "cgb": CGB, "mc": MC}
KINDS = {"traffic": TRAFFIC, "ks": KS, "osc": OSC, "linear": LINEAR, "heat": HEAT, "quad": QUAD}

# default parameters of the benchmark workloads: traffic (c, v, w, xbar); KS (dx, g_nl,
# g_2, g_4); oscillator (ka, kb, kc)
TRAFFIC_PRM = (40.0, 0.5, 1.0 / 6.0, 320.0)
# the same with the box-evaluated CGB contraction matrix (reading R14)
TRAFFIC_LOCAL_PRM = TRAFFIC_PRM + (1.0,)
# outward-rounded MM / CGB (reading R15)
TRAFFIC_SOUND_PRM = TRAFFIC_PRM + (0.0, 1.0)
KS_PRM = (math.pi / 4.0, 1.0, 1.0, 1.0)
OSC_PRM = (1.0, 0.1, 0.5)
# heat: (alpha, l, open face); l is set from n by default_params
HEAT_ALPHA = 8e-6
# quadrotor: (m, g, F, Jx, Jy, Jz), hover thrust F = m g
QUAD_PRM = (1.4, 9.81, 1.4 * 9.81, 0.054, 0.054, 0.104)


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so beside it (no threads, no FMA)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        subprocess.check_call([
            "gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c11",
            "-fPIC", "-shared", "-Wall", "-o", _LIB, _SRC, "-lm"])
    return _LIB


_lib = None


def lib():
    global _lib
    if _lib is None:
        if _LIB_OVERRIDE:
            L = ctypes.CDLL(_LIB_OVERRIDE)
        else:
            build()
            L = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        L.orc_reach.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int64,
                                dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                ctypes.c_int64, ctypes.c_uint64, ctypes.c_int, dp, dp, dp]
        L.orc_reach.restype = ctypes.c_int
        L.orc_reach_pipe.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int64,
                                     dp, dp, dp, dp, ctypes.c_double, ctypes.c_double,
                                     ctypes.c_int64, dp, dp, dp, dp]
        L.orc_reach_pipe.restype = ctypes.c_int
        L.orc_flow.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp,
                               ctypes.c_double, ctypes.c_double, dp]
        L.orc_flow.restype = ctypes.c_int
        L.orc_nsteps.argtypes = [ctypes.c_double, ctypes.c_double, ctypes.POINTER(ctypes.c_int64)]
        L.orc_nsteps.restype = ctypes.c_int
        L.orc_input_dim.argtypes = [ctypes.c_int, ctypes.c_int64]
        L.orc_input_dim.restype = ctypes.c_int64
        L.orc_philox4x32_10.argtypes = [ctypes.POINTER(ctypes.c_uint32)] * 3
        L.orc_philox4x32_10.restype = None
        L.orc_uniform.argtypes = [ctypes.c_uint64, ctypes.c_int64, ctypes.c_int64, ctypes.c_uint32]
        L.orc_uniform.restype = ctypes.c_double
        L.orc_mc_samples.argtypes = [ctypes.c_int64, ctypes.c_double, ctypes.c_double]
        L.orc_mc_samples.restype = ctypes.c_int64
        L.orc_rhs.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp, dp]
        L.orc_rhs.restype = ctypes.c_int
        L.orc_decomp.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp, dp, dp, dp]
        L.orc_decomp.restype = ctypes.c_int
        pd = ctypes.POINTER(ctypes.c_double)
        L.orc_sound_op.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double, pd]
        L.orc_sound_op.restype = ctypes.c_int
        L.orc_sound_mul_pos.argtypes = [ctypes.c_double] * 4 + [pd, pd]
        L.orc_sound_mul_pos.restype = ctypes.c_int
        L.orc_traffic_sound_rhs.argtypes = [dp, ctypes.c_int64, dp, dp, ctypes.c_double, ctypes.c_double, dp, dp]
        L.orc_traffic_sound_rhs.restype = ctypes.c_int
        L.orc_traffic_sound_radius_rhs.argtypes = [dp, ctypes.c_int64, dp, ctypes.c_double, dp]
        L.orc_traffic_sound_radius_rhs.restype = ctypes.c_int
        L.orc_growth.argtypes = [ctypes.c_int, dp, dp, ctypes.c_int64, dp, dp, dp, dp]
        L.orc_growth.restype = ctypes.c_int
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, rc):
        super().__init__(f"oracle returned {rc}")
        self.rc = rc


def _p(a):
    if a is None:
        return None
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _vec(a, n=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64)).reshape(-1)
    if n is not None and a.size != n:
        raise ValueError(f"expected {n} values, got {a.size}")
    return a


def default_params(kind: str, n: int = 0):
    if kind == "heat":
        return (HEAT_ALPHA, float(round(n ** (1.0 / 3.0))), 1.0)
    return {"traffic": TRAFFIC_PRM, "ks": KS_PRM, "osc": OSC_PRM, "linear": (), "quad": QUAD_PRM}[kind]


def input_dim(kind: str, n: int) -> int:
    return int(lib().orc_input_dim(KINDS[kind], n))


def _prep(kind, n, params, A, w_lo, w_hi):
    prm = _vec(default_params(kind, n) if params is None else params)
    if kind == "traffic" and prm.size < 6:
        # defaults: CGB with the bounds valid for every state; round to nearest
        prm = np.concatenate([prm, np.zeros(6 - prm.size)])
    if prm.size == 0:
        prm = np.zeros(1)
    Aa = None
    if kind == "linear":
        Aa = np.ascontiguousarray(np.asarray(A, dtype=np.float64).reshape(n, n))
    nw = input_dim(kind, n)
    wl = _vec(np.zeros(nw) if w_lo is None else w_lo, nw)
    wh = _vec(np.zeros(nw) if w_hi is None else w_hi, nw)
    if nw == 0:
        wl = np.zeros(1)
        wh = np.zeros(1)
    return prm, Aa, wl, wh


def reach(method: str, kind: str, x_lo, x_hi, w_lo=None, w_hi=None, *, t_final: float,
          dt: float, params=None, A=None, m: int = 0, seed: int = 0, prec: int = 64,
          return_finals: bool = False):
    """Interval reachable set of one method (Algorithms 2-4).  Returns (lo, hi)
    [, finals (m x n) for MC]."""
    x_lo = _vec(x_lo)
    n = x_lo.size
    x_hi = _vec(x_hi, n)
    prm, Aa, wl, wh = _prep(kind, n, params, A, w_lo, w_hi)
    lo = np.empty(n)
    hi = np.empty(n)
    finals = np.empty((m, n)) if (return_finals and method == "mc") else None
    rc = lib().orc_reach(METHODS[method], KINDS[kind], _p(prm), _p(Aa), n, _p(x_lo), _p(x_hi),
                         _p(wl), _p(wh), float(t_final), float(dt), int(m), int(seed) & (2**64 - 1),
                         int(prec), _p(lo), _p(hi), _p(finals))
    if rc != 0:
        raise OracleError(rc)
    if return_finals and method == "mc":
        return lo, hi, finals
    return lo, hi


def reach_pipe(method: str, kind: str, x_lo, x_hi, w_lo=None, w_hi=None, *, t_final: float,
               dt: float, every: int, params=None, A=None):
    """Boxes after every `every` RK4 steps (the reach pipe, Sec. 5.5)."""
    x_lo = _vec(x_lo)
    n = x_lo.size
    x_hi = _vec(x_hi, n)
    prm, Aa, wl, wh = _prep(kind, n, params, A, w_lo, w_hi)
    N = nsteps(t_final, dt)
    rows = N // every if every > 0 else 0
    plo = np.empty((max(rows, 1), n))
    phi = np.empty((max(rows, 1), n))
    lo = np.empty(n)
    hi = np.empty(n)
    rc = lib().orc_reach_pipe(METHODS[method], KINDS[kind], _p(prm), _p(Aa), n, _p(x_lo), _p(x_hi),
                              _p(wl), _p(wh), float(t_final), float(dt), int(every),
                              _p(plo), _p(phi), _p(lo), _p(hi))
    if rc != 0:
        raise OracleError(rc)
    return plo[:rows], phi[:rows]


def flow(kind: str, x0, w=None, *, t_final: float, dt: float, params=None, A=None):
    """One trajectory Phi(t_final; 0, x0, w) of the plain system under RK4."""
    x0 = _vec(x0)
    n = x0.size
    prm, Aa, wl, _ = _prep(kind, n, params, A, w, w)
    out = np.empty(n)
    rc = lib().orc_flow(KINDS[kind], _p(prm), _p(Aa), n, _p(x0), _p(wl), float(t_final),
                        float(dt), _p(out))
    if rc != 0:
        raise OracleError(rc)
    return out


def sound_op(op: str, a: float, b: float) -> float:
    """One directed operation of reading R15: op in add_dn, add_up, mul_dn,
    mul_up, div_dn, div_up."""
    code = ["add_dn", "add_up", "mul_dn", "mul_up", "div_dn", "div_up"].index(op)
    out = ctypes.c_double(0.0)
    rc = lib().orc_sound_op(code, float(a), float(b), ctypes.byref(out))
    if rc != 0:
        raise OracleError(rc)
    return out.value


def sound_mul_pos(cl, cu, ql, qu):
    """[ql, qu] times a constant in [cl, cu] (cl >= 0), rounded outward."""
    rl, ru = ctypes.c_double(0.0), ctypes.c_double(0.0)
    rc = lib().orc_sound_mul_pos(float(cl), float(cu), float(ql), float(qu), ctypes.byref(rl), ctypes.byref(ru))
    if rc != 0:
        raise OracleError(rc)
    return rl.value, ru.value


def traffic_sound_rhs(yl, yu, dl, du, params=None):
    """Interval right-hand side of the traffic chain, rounded outward (R15)."""
    yl = _vec(yl)
    n = yl.size
    yu = _vec(yu, n)
    prm, _, _, _ = _prep("traffic", n, params, None, [dl], [du])
    kl, ku = np.empty(n), np.empty(n)
    rc = lib().orc_traffic_sound_rhs(_p(prm), n, _p(yl), _p(yu), float(dl), float(du), _p(kl), _p(ku))
    if rc != 0:
        raise OracleError(rc)
    return kl, ku


def traffic_sound_radius_rhs(r, hp, params=None):
    """Upper bound of the traffic CGB radius right-hand side C r + [p] (R15)."""
    r = _vec(r)
    n = r.size
    prm, _, _, _ = _prep("traffic", n, params, None, [0.0], [0.0])
    dr = np.empty(n)
    rc = lib().orc_traffic_sound_radius_rhs(_p(prm), n, _p(r), float(hp), _p(dr))
    if rc != 0:
        raise OracleError(rc)
    return dr


def nsteps(t_final: float, dt: float) -> int:
    N = ctypes.c_int64(0)
    rc = lib().orc_nsteps(float(t_final), float(dt), ctypes.byref(N))
    if rc != 0:
        raise OracleError(rc)
    return int(N.value)


def philox4x32_10(ctr, key):
    c = (ctypes.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (ctypes.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (ctypes.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return tuple(int(v) for v in o)


def uniform(seed: int, j: int, i: int, tag: int) -> float:
    return float(lib().orc_uniform(int(seed) & (2**64 - 1), int(j), int(i), int(tag)))


def mc_samples(n: int, eps: float, delta: float) -> int:
    return int(lib().orc_mc_samples(int(n), float(eps), float(delta)))


def rhs(kind: str, x, p=None, *, params=None, A=None):
    """f(x, p) of the plain system (Sec. 2)."""
    x = _vec(x)
    n = x.size
    prm, Aa, pl, _ = _prep(kind, n, params, A, p, p)
    out = np.empty(n)
    rc = lib().orc_rhs(KINDS[kind], _p(prm), _p(Aa), n, _p(x), _p(pl), _p(out))
    if rc != 0:
        raise OracleError(rc)
    return out


def decomp(kind: str, x, p, xh, ph, *, params=None, A=None):
    """Decomposition function d(x, p, xh, ph) (Sec. 2.1, MM)."""
    x = _vec(x)
    n = x.size
    xh = _vec(xh, n)
    prm, Aa, pl, ph_ = _prep(kind, n, params, A, p, ph)
    out = np.empty(n)
    rc = lib().orc_decomp(KINDS[kind], _p(prm), _p(Aa), n, _p(x), _p(pl), _p(xh), _p(ph_), _p(out))
    if rc != 0:
        raise OracleError(rc)
    return out


def growth(kind: str, c, r, hp=None, *, params=None, A=None):
    """Growth dynamics g = C(c, r) r + [p] (Sec. 2.1, CGB)."""
    c = _vec(c)
    n = c.size
    r = _vec(r, n)
    prm, Aa, hpl, _ = _prep(kind, n, params, A, hp, hp)
    out = np.empty(n)
    rc = lib().orc_growth(KINDS[kind], _p(prm), _p(Aa), n, _p(c), _p(r), _p(hpl), _p(out))
    if rc != 0:
        raise OracleError(rc)
    return out
