"""reach_mm_noalloc, the entry point for callers that cannot let the library
allocate device memory (their device memory is held by another allocator, or
their loop must not enter the driver's allocator).

It must give the same boxes as reach_mm, whose scratch comes from the memory
pool, on two calls in a row (the second call finds the first call's contents
in the shared fixed buffer).  This file is collected last so that a run that
stops at the first failure has run every other test before it.
"""
import ctypes

import numpy as np
import pytest

import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

MAX_N = 1048576   # REACH_NOALLOC_MAX_N in include/reach.h


def _noalloc():
    f = R.lib().reach_mm_noalloc
    vp = ctypes.c_void_p
    f.argtypes = [vp, vp, vp, vp, vp, ctypes.c_double, ctypes.c_double, vp, vp, vp]
    f.restype = ctypes.c_int
    return f


def _traffic_case(n, seed):
    import torch
    wl = W.traffic_large(n, seed=seed)
    d = {k: torch.tensor(wl[k], dtype=torch.float64, device="cuda") for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    return wl, d


def _call(f, s, d, T, dt):
    import torch
    lo = torch.empty(s.n, dtype=torch.float64, device="cuda")
    hi = torch.empty_like(lo)
    w = (d["w_lo"].data_ptr(), d["w_hi"].data_ptr()) if "w_lo" in d else (None, None)
    rc = f(s.handle, d["x_lo"].data_ptr(), d["x_hi"].data_ptr(), w[0], w[1], T, dt,
           lo.data_ptr(), hi.data_ptr(), None)
    return rc, lo, hi


def test_noalloc_matches_reach_mm_on_two_calls():
    f = _noalloc()
    n, T, dt = 300_001, 0.5, 0.01
    with R.System("traffic", n) as s:
        for seed in (1, 2):   # two calls in a row on the shared buffer
            wl, d = _traffic_case(n, seed)
            rc, lo, hi = _call(f, s, d, T, dt)
            assert rc == 0, R.strerror(rc)
            ref = R.reach_mm(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=T, dt=dt)
            assert_close(lo.cpu().numpy(), ref[0].cpu().numpy(), TOL64, f"call {seed} lo")
            assert_close(hi.cpu().numpy(), ref[1].cpu().numpy(), TOL64, f"call {seed} hi")


def test_noalloc_host_inflow_short_grid_and_zero_horizon():
    # the traffic inflow box from host memory, a grid short enough for several
    # RK4 steps per launch, and a zero horizon (the box itself)
    import torch
    f = _noalloc()
    n, T, dt = 5000, 0.37, 0.01
    with R.System("traffic", n) as s:
        wl, d = _traffic_case(n, 6)
        lo = torch.empty(n, dtype=torch.float64, device="cuda")
        hi = torch.empty_like(lo)
        for _ in range(2):
            rc = f(s.handle, d["x_lo"].data_ptr(), d["x_hi"].data_ptr(), wl["w_lo"].ctypes.data,
                   wl["w_hi"].ctypes.data, T, dt, lo.data_ptr(), hi.data_ptr(), None)
            assert rc == 0, R.strerror(rc)
            ref = R.reach_mm(s, wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T, dt=dt)
            assert_close(lo.cpu().numpy(), ref[0], TOL64, "lo")
            assert_close(hi.cpu().numpy(), ref[1], TOL64, "hi")
        rc, lo0, hi0 = _call(f, s, d, 0.0, dt)
        assert rc == 0
        assert torch.equal(lo0, d["x_lo"]) and torch.equal(hi0, d["x_hi"])


def test_noalloc_ks_at_the_size_limit():
    import torch
    f = _noalloc()
    wl = W.ks_grid(MAX_N, t_final=0.002)
    d = {k: torch.tensor(wl[k], dtype=torch.float64, device="cuda") for k in ("x_lo", "x_hi")}
    with R.System("ks", MAX_N) as s:
        rc, lo, hi = _call(f, s, d, wl["t_final"], wl["dt"])
        assert rc == 0, R.strerror(rc)
        ref = R.reach_mm(s, d["x_lo"], d["x_hi"], t_final=wl["t_final"], dt=wl["dt"])
    assert_close(lo.cpu().numpy(), ref[0].cpu().numpy(), TOL64, "ks lo")
    assert_close(hi.cpu().numpy(), ref[1].cpu().numpy(), TOL64, "ks hi")


def test_noalloc_rejects_what_it_cannot_run():
    import torch
    f = _noalloc()
    with R.System("traffic", MAX_N + 1) as s:   # one cell beyond the fixed buffer
        _, d = _traffic_case(MAX_N + 1, 3)
        rc, _, _ = _call(f, s, d, 0.1, 0.01)
        assert rc == -1
    with R.System("traffic", 1000) as s:        # host state vectors are not staged
        wl = W.traffic_large(1000, seed=4)
        lo, hi = np.empty(1000), np.empty(1000)
        rc = f(s.handle, wl["x_lo"].ctypes.data, wl["x_hi"].ctypes.data, wl["w_lo"].ctypes.data,
               wl["w_hi"].ctypes.data, 0.1, 0.01, lo.ctypes.data, hi.ctypes.data, None)
        assert rc == -1
    with R.System("traffic", 1000) as s:        # inverted inflow box
        _, d = _traffic_case(1000, 5)
        d["w_lo"], d["w_hi"] = d["w_hi"], d["w_lo"]
        rc, _, _ = _call(f, s, d, 0.1, 0.01)
        assert rc == -1
    with R.System("traffic", 1000, params=(40.0, 0.5, 1 / 6, 320.0, 0, 1)) as s:   # outward rounding
        _, d = _traffic_case(1000, 5)
        rc, _, _ = _call(f, s, d, 0.1, 0.01)
        assert rc == -1
    A = np.eye(3) * -1.0
    with R.System("linear", 3, A=A) as s:       # no streaming kernel for this kind
        d = {k: torch.zeros(3, dtype=torch.float64, device="cuda") for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        rc, _, _ = _call(f, s, d, 0.1, 0.01)
        assert rc == -1
