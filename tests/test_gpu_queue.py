"""The device work queue (reach_queue_*): queries published to a ring in
mapped host memory and run by the blocks of a persistent kernel as they
arrive.  Results must equal the FP64 oracle (and, bit for bit, the on-chip
kernel of reach_mm / reach_cgb); every device-side wait is bounded, so idle
blocks leave by themselves with REACH_ETIMEOUT as their exit status."""
import threading

import numpy as np
import pytest

import oracle as O
import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


@pytest.fixture(autouse=True)
def _reset_options():
    yield
    R.reach_set_option(R.OPT_KERNEL, 0)


def _problem(kind, n, seed):
    g = np.random.default_rng(seed)
    if kind == "traffic":
        c = g.uniform(60, 200, n)
        return dict(x_lo=c - 4, x_hi=c + 4, w_lo=np.array([35.0]), w_hi=np.array([45.0]), T=0.5, dt=0.01)
    if kind == "ks":
        u = W.ks_profile(n) + g.uniform(-0.01, 0.01, n)
        return dict(x_lo=u - 1e-3, x_hi=u + 1e-3, w_lo=None, w_hi=None, T=0.005, dt=1e-4)
    if kind == "osc":
        q = W.osc_query(n // 2, seed=seed, half_width=1e-3, t_final=0.5)
        return dict(x_lo=q["x_lo"], x_hi=q["x_hi"], w_lo=q["w_lo"], w_hi=q["w_hi"], T=0.5, dt=0.005)
    if kind == "heat":
        lo, hi = W.random_box(n, seed=seed, centre=(0.0, 1.0), width=(0.0, 0.1))
        return dict(x_lo=lo, x_hi=hi, w_lo=None, w_hi=None, T=0.2, dt=0.02)
    lo, hi = W.random_box(n, seed=seed + 1)
    plo, phi = W.random_box(n, seed=seed + 2, centre=(-0.1, 0.1), width=(0.0, 0.05))
    return dict(x_lo=lo, x_hi=hi, w_lo=plo, w_hi=phi, T=0.5, dt=0.01, A=W.linear_general(n, seed=seed, scale=0.5))


# (kind, n): one item per block at 1, 4 and 16 components per thread
MIX = [("traffic", 16), ("traffic", 200), ("traffic", 1000), ("traffic", 4096), ("ks", 64), ("ks", 700),
       ("ks", 4096), ("osc", 40), ("osc", 2000), ("heat", 125), ("heat", 4096), ("linear", 7), ("linear", 100)]


def test_queued_queries_match_the_oracle_and_the_on_chip_kernel():
    systems, jobs = {}, []
    with R.Queue(max_blocks=8, idle_s=0.01) as q:
        for i, (kind, n) in enumerate(MIX):
            p = _problem(kind, n, seed=50 + i)
            s = systems[(kind, n)] = R.System(kind, n, A=p.get("A"))
            for method in ("mm", "cgb"):
                t, out = q.submit(s, method, p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
                jobs.append((kind, n, method, p, t, out))
        for kind, n, method, p, t, (lo, hi) in jobs:
            assert q.wait(t, timeout_s=120) == 0, (kind, n, method)
            o = O.reach(method, kind, p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"],
                        A=p.get("A"))
            assert_close(lo, o[0], TOL64, f"{kind}{n} {method} lo")
            assert_close(hi, o[1], TOL64, f"{kind}{n} {method} hi")
            R.reach_set_option(R.OPT_KERNEL, 2)
            f = R.reach_mm if method == "mm" else R.reach_cgb
            a = f(systems[(kind, n)], p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
            R.reach_set_option(R.OPT_KERNEL, 0)
            np.testing.assert_array_equal(lo, a[0])
            np.testing.assert_array_equal(hi, a[1])
        assert q.stats()["in_flight"] == 0
    for s in systems.values():
        s.close()


def test_device_buffers_and_device_side_box_check():
    import torch
    p = _problem("traffic", 3000, seed=3)
    d = {k: torch.tensor(p[k], dtype=torch.float64, device="cuda") for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    with R.System("traffic", 3000) as s, R.Queue(max_blocks=2, idle_s=0.01) as q:
        t, (lo, hi) = q.submit(s, "mm", d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=p["T"], dt=p["dt"])
        assert q.wait(t, timeout_s=60) == 0
        o = O.reach("mm", "traffic", p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
        assert_close(lo.cpu().numpy(), o[0], TOL64, "lo")
        assert_close(hi.cpu().numpy(), o[1], TOL64, "hi")
        # an inverted box in device memory is seen by the kernel: REACH_EINVAL as the query's status
        t, _ = q.submit(s, "cgb", d["x_hi"], d["x_lo"], d["w_lo"], d["w_hi"], t_final=p["T"], dt=p["dt"])
        assert q.wait(t, timeout_s=60) == -1


def test_idle_blocks_leave_when_their_bounded_wait_runs_out():
    # no producer: the launched blocks poll the empty ring for idle_s and
    # leave; the launch's exit status is REACH_ETIMEOUT and the GPU stays usable
    with R.Queue(max_blocks=4, idle_s=0.05) as q:
        q.start("traffic", 4)
        assert q.join(timeout_s=30) == -5
        assert q.stats()["alive_blocks"] == 0
        # a query submitted afterwards starts new blocks and completes
        p = _problem("traffic", 100, seed=4)
        with R.System("traffic", 100) as s:
            t, (lo, hi) = q.submit(s, "mm", p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
            assert q.wait(t, timeout_s=60) == 0
            o = O.reach("mm", "traffic", p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
            assert_close(lo, o[0], TOL64, "lo")
        assert q.join(timeout_s=30) == -5


def test_host_wait_times_out_and_the_query_still_completes():
    p = _problem("ks", 4096, seed=6)
    with R.System("ks", 4096) as s, R.Queue(max_blocks=1, idle_s=0.01) as q:
        t, (lo, hi) = q.submit(s, "mm", p["x_lo"], p["x_hi"], t_final=0.05, dt=1e-4)   # 500 steps
        with pytest.raises(R.ReachError) as e:
            q.wait(t, timeout_s=0.0)
        assert e.value.code == -5
        assert q.wait(t, timeout_s=120) == 0
        assert np.isfinite(lo).all() and (lo <= hi).all()


def test_more_queries_than_blocks_arrive_while_a_streaming_kernel_runs():
    # arrivals join the running blocks (continuous batching) while another
    # thread runs a GPU-wide streaming call; every result is the oracle's
    big = W.traffic_large(1 << 22, seed=1, t_final=1.0)
    sb = R.System("traffic", 1 << 22)
    done = {}

    def run_big():
        done["big"] = R.reach_mm(sb, big["x_lo"], big["x_hi"], big["w_lo"], big["w_hi"], t_final=1.0, dt=0.01)

    th = threading.Thread(target=run_big)
    th.start()
    systems, jobs = {}, []
    with R.Queue(max_blocks=3, idle_s=0.01) as q:
        g = np.random.default_rng(8)
        for i in range(40):
            kind = ("traffic", "ks")[i % 2]
            n = int(g.integers(8, 600)) if kind == "traffic" else int(g.integers(5, 600))
            p = _problem(kind, n, seed=100 + i)
            s = systems.setdefault((kind, n), R.System(kind, n))
            method = ("mm", "cgb")[(i // 2) % 2]
            t, out = q.submit(s, method, p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
            jobs.append((kind, n, method, p, t, out))
        for kind, n, method, p, t, (lo, hi) in jobs:
            assert q.wait(t, timeout_s=120) == 0
            o = O.reach(method, kind, p["x_lo"], p["x_hi"], p["w_lo"], p["w_hi"], t_final=p["T"], dt=p["dt"])
            assert_close(lo, o[0], TOL64, f"{kind}{n} {method} lo")
            assert_close(hi, o[1], TOL64, f"{kind}{n} {method} hi")
        st = q.stats()
        assert st["in_flight"] == 0 and 1 <= st["launched_blocks"]
    th.join()
    assert np.isfinite(done["big"][0]).all()
    sb.close()
    for s in systems.values():
        s.close()


def test_queue_rejects_what_it_cannot_run():
    p = _problem("traffic", 20, seed=9)
    with R.Queue(max_blocks=1, idle_s=0.01) as q:
        cases = [(R.System("traffic", 5000), p["x_lo"].repeat(250), p["x_hi"].repeat(250), 0.5),   # n > 4096
                 (R.System("traffic", 20, params=(40.0, 0.5, 1 / 6, 320.0, 0, 1)), p["x_lo"], p["x_hi"], 0.5),
                 (R.System("traffic", 20), p["x_lo"], p["x_hi"], 0.0),                               # zero horizon
                 (R.System("traffic", 20), p["x_hi"], p["x_lo"], 0.5)]                               # lo > hi on host
        for s, lo, hi, T in cases:
            with pytest.raises(R.ReachError) as e:
                q.submit(s, "mm", lo, hi, p["w_lo"], p["w_hi"], t_final=T, dt=0.01)
            assert e.value.code == -1
            s.close()
        with R.System("quad", 24) as s:
            qs = W.quad_swarm(2, seed=1, t_final=0.1)
            with pytest.raises(R.ReachError):
                q.submit(s, "mm", qs["x_lo"], qs["x_hi"], qs["w_lo"], qs["w_hi"], t_final=0.1, dt=0.01)
