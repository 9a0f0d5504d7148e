"""The continuous-batching server (reach_server_*): every result in the mix is
the oracle's (or, for queries too large for the oracle, the same call made
alone), small requests run on the device work queue, admission keeps within
the memory budget, and bounded waits time out on the host."""
import numpy as np
import pytest

import oracle as O
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


# oracle work per query (comp-steps) up to which the mix is checked against
# the oracle; larger queries are checked against the same call made alone
ORACLE_WORK = 3e7


def _oracle(q):
    kw = dict(t_final=q.steps * q.dt, dt=q.dt, params=q.params or None)
    w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
    if q.method == "mc":
        return O.reach("mc", q.kind, q.x_lo, q.x_hi, *w, **kw, m=q.m, seed=q.seed, prec=q.prec)
    return O.reach(q.method, q.kind, q.x_lo, q.x_hi, *w, **kw)


def _work(q):
    return (q.m * q.n if q.method == "mc" else 2 * q.n) * q.steps


@pytest.mark.parametrize("exclusive", [0, 1])
def test_results_in_the_mix_match_the_oracle(exclusive):
    # all submitted at once: the server must overlap them, send the small MM /
    # CGB requests to its device work queue and admit the rest as slots free up
    # (with exclusive wide requests, a wide one computes alone)
    trace = W.serving_trace(count=48, seed=3, traffic_n=(100, 600_000), ks_k=(10, 15), steps=(100, 2000),
                            scale_steps=0.2)
    cache = _systems(trace)
    checked = 0
    R.reach_set_option(R.OPT_SERVE_WIDE_EXCLUSIVE, exclusive)
    try:
        srv = R.Server(slots=6, hbm_budget_bytes=8 << 30)
    finally:
        R.reach_set_option(R.OPT_SERVE_WIDE_EXCLUSIVE, 1)
    with srv:
        tickets = []
        for q in trace:
            w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
            tickets.append(srv.submit(cache[(q.kind, q.n)], q.method, q.x_lo, q.x_hi, *w, t_final=q.steps * q.dt,
                                      dt=q.dt, m=q.m, seed=q.seed, precision=q.prec))
        for (t, (lo, hi)), q in zip(tickets, trace):
            st, qs, rs = srv.wait(t, timeout_s=300)
            assert st == 0, (q.kind, q.method, q.n, st)
            tol = TOL32 if q.method == "mc" and q.prec == 32 else TOL64
            if _work(q) <= ORACLE_WORK:
                ref = _oracle(q)
                checked += 1
            else:
                ref = _alone(cache[(q.kind, q.n)], q)
            assert_close(lo, ref[0], tol, f"{q.kind} {q.method} n={q.n} lo")
            assert_close(hi, ref[1], tol, f"{q.kind} {q.method} n={q.n} hi")
        st = srv.stats()
        assert st["done"] == len(trace) and st["waiting"] == 0 and st["bytes_in_use"] == 0
        assert srv.queued() > 0   # some requests ran on the device work queue
    assert checked >= len(trace) // 2
    for s in cache.values():
        s.close()


def test_small_requests_alone_and_in_the_mix_through_the_queue():
    # small MM / CGB requests (always queued) submitted one at a time and all
    # together give the same boxes, and they are the oracle's
    g = np.random.default_rng(12)
    reqs = []
    for i in range(24):
        kind = ("traffic", "ks")[i % 2]
        n = int(g.integers(10, 500))
        if kind == "traffic":
            c = g.uniform(60, 200, n)
            args = (c - 2, c + 2, np.array([35.0]), np.array([45.0]))
            T, dt = 1.0, 0.01
        else:
            u = W.ks_profile(n) + g.uniform(-0.01, 0.01, n)
            args = (u - 1e-3, u + 1e-3, None, None)
            T, dt = 0.01, 1e-4
        reqs.append((kind, n, ("mm", "cgb")[(i // 2) % 2], args, T, dt))
    systems = {(k, n): R.System(k, n) for k, n, *_ in reqs}
    with R.Server(slots=2, hbm_budget_bytes=1 << 30) as srv:
        alone = []
        for k, n, m, args, T, dt in reqs:
            t, out = srv.submit(systems[(k, n)], m, *args, t_final=T, dt=dt)
            assert srv.wait(t, timeout_s=120)[0] == 0
            alone.append(out)
        mix = [srv.submit(systems[(k, n)], m, *args, t_final=T, dt=dt) for k, n, m, args, T, dt in reqs]
        for (t, out), a, (k, n, m, args, T, dt) in zip(mix, alone, reqs):
            assert srv.wait(t, timeout_s=120)[0] == 0
            np.testing.assert_array_equal(out[0], a[0])
            np.testing.assert_array_equal(out[1], a[1])
            o = O.reach(m, k, *args, t_final=T, dt=dt)
            assert_close(out[0], o[0], TOL64, f"{k}{n} {m} lo")
            assert_close(out[1], o[1], TOL64, f"{k}{n} {m} hi")
        assert srv.queued() == 2 * len(reqs)
    for s in systems.values():
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
