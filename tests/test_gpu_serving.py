"""The continuous-batching server (reach_server_*): results in the mix equal
results alone, admission keeps within the memory budget, and bounded waits
time out on the host without touching the GPU."""
import numpy as np
import pytest

import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL32, TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


def _systems(trace):
    cache = {}
    for q in trace:
        key = (q.kind, q.n)
        if key not in cache:
            cache[key] = R.System(q.kind, q.n)
    return cache


def _alone(s, q):
    kw = dict(t_final=q.steps * q.dt, dt=q.dt)
    w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
    if q.method == "mm":
        return R.reach_mm(s, q.x_lo, q.x_hi, *w, **kw)
    if q.method == "cgb":
        return R.reach_cgb(s, q.x_lo, q.x_hi, *w, **kw)
    return R.reach_mc(s, q.x_lo, q.x_hi, *w, **kw, m=q.m, seed=q.seed, precision=q.prec)


def test_results_in_the_mix_equal_results_alone():
    trace = W.serving_trace(count=48, seed=3, traffic_n=(100, 200_000), ks_k=(10, 15), steps=(100, 2000),
                            scale_steps=0.2)
    cache = _systems(trace)
    with R.Server(slots=6, hbm_budget_bytes=8 << 30) as srv:
        tickets = []
        for q in trace:   # all at once: the server must overlap and admit them as slots free up
            w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
            tickets.append(srv.submit(cache[(q.kind, q.n)], q.method, q.x_lo, q.x_hi, *w, t_final=q.steps * q.dt,
                                      dt=q.dt, m=q.m, seed=q.seed, precision=q.prec))
        for (t, (lo, hi)), q in zip(tickets, trace):
            st, qs, rs = srv.wait(t, timeout_s=300)
            assert st == 0, (q.kind, q.method, q.n, st)
            a = _alone(cache[(q.kind, q.n)], q)
            tol = TOL32 if q.method == "mc" and q.prec == 32 else TOL64
            assert_close(lo, a[0], tol, f"{q.kind} {q.method} n={q.n} lo")
            assert_close(hi, a[1], tol, f"{q.kind} {q.method} n={q.n} hi")
        st = srv.stats()
        assert st["done"] == len(trace) and st["waiting"] == 0 and st["bytes_in_use"] == 0
    for s in cache.values():
        s.close()


def test_admission_keeps_within_the_budget():
    n = 1 << 18
    wl = W.traffic_large(n, seed=1, t_final=0.5)
    with R.System("traffic", n) as s:
        need = R.reach_request_footprint(s, "mm")
        assert need > 48 * n
        budget = int(2.5 * need)   # at most two at a time
        with R.Server(slots=8, hbm_budget_bytes=budget) as srv:
            ts = [srv.submit(s, "mm", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=0.5, dt=0.01)
                  for _ in range(6)]
            outs = []
            for t, (lo, hi) in ts:
                assert srv.wait(t, timeout_s=300)[0] == 0
                outs.append(lo)
            assert srv.stats()["bytes_peak"] <= budget
            assert all(np.array_equal(outs[0], o) for o in outs)
        with R.Server(slots=2, hbm_budget_bytes=need - 1) as srv:
            with pytest.raises(R.ReachError) as e:
                srv.submit(s, "mm", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=0.5, dt=0.01)
            assert e.value.code == -3


def test_bounded_wait_times_out_and_the_request_still_completes():
    n = 1 << 22
    wl = W.traffic_large(n, seed=2, t_final=4.0)
    with R.System("traffic", n) as s, R.Server(slots=1, hbm_budget_bytes=4 << 30) as srv:
        t, (lo, hi) = srv.submit(s, "mm", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=4.0, dt=0.01)
        with pytest.raises(R.ReachError) as e:
            srv.wait(t, timeout_s=0.001)
        assert e.value.code == -5
        st, _, run_s = srv.wait(t, timeout_s=300)
        assert st == 0 and run_s > 0 and np.isfinite(lo).all()


def test_heat_quad_and_outward_rounded_requests_in_the_mix():
    # the other kinds through the server, submitted together: each result
    # equals the same call made alone (bit for bit: same kernels, same inputs)
    hc = W.heat_cube(20, t_final=0.2)
    qs = W.quad_swarm(300, seed=2, t_final=0.3)
    tr = W.traffic_large(9000, seed=4, t_final=0.3)
    systems = {"heat": R.System("heat", 20 ** 3), "quad": R.System("quad", 3600),
               "sound": R.System("traffic", 9000, params=(40.0, 0.5, 1 / 6, 320.0, 0, 1)),
               "local": R.System("traffic", 9000, params=(40.0, 0.5, 1 / 6, 320.0, 1, 0))}
    jobs = []
    for method in ("mm", "cgb"):
        jobs.append(("heat", method, (hc["x_lo"], hc["x_hi"], None, None), 0.2, 0.02))
        jobs.append(("quad", method, (qs["x_lo"], qs["x_hi"], qs["w_lo"], qs["w_hi"]), 0.3, 0.01))
        jobs.append(("sound", method, (tr["x_lo"], tr["x_hi"], tr["w_lo"], tr["w_hi"]), 0.3, 0.01))
    jobs.append(("local", "cgb", (tr["x_lo"], tr["x_hi"], tr["w_lo"], tr["w_hi"]), 0.3, 0.01))
    jobs.append(("quad", "mc", (qs["x_lo"], qs["x_hi"], qs["w_lo"], qs["w_hi"]), 0.3, 0.01))
    with R.Server(slots=4, hbm_budget_bytes=4 << 30) as srv:
        tickets = [srv.submit(systems[k], m, *args, t_final=T, dt=dt, m=64, seed=9, precision=64)
                   for k, m, args, T, dt in jobs]
        for (t, (lo, hi)), (k, m, args, T, dt) in zip(tickets, jobs):
            st, _, _ = srv.wait(t, timeout_s=300)
            assert st == 0, (k, m, st)
            s = systems[k]
            if m == "mm":
                a = R.reach_mm(s, *args, t_final=T, dt=dt)
            elif m == "cgb":
                a = R.reach_cgb(s, *args, t_final=T, dt=dt)
            else:
                a = R.reach_mc(s, *args, t_final=T, dt=dt, m=64, seed=9, precision=64)
            np.testing.assert_array_equal(lo, a[0])
            np.testing.assert_array_equal(hi, a[1])
    for s in systems.values():
        s.close()
