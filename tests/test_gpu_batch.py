"""Batched persistent launch (reach_batch_*) and the cluster path of single
queries: parity with the oracle and with per-query calls."""
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
    R.reach_set_option(R.OPT_BATCH_CPT, 0)
    R.reach_set_option(R.OPT_KERNEL, 0)
    R.reach_set_option(R.OPT_BATCH_CLUSTER_FROM, 0)


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_single_query_on_a_cluster_matches_oracle(method):
    m = 3000   # 2n = 12000 components: more than one block holds
    q = W.osc_query(m, seed=21, t_final=0.1)
    with R.System("osc", 2 * m) as s:
        fn = R.reach_mm if method == "mm" else R.reach_cgb
        g = fn(s, q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=q["t_final"], dt=q["dt"])
    o = O.reach(method, "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=q["t_final"], dt=q["dt"])
    assert_close(g[0], o[0], TOL64, "lo")
    assert_close(g[1], o[1], TOL64, "hi")


def _osc_batch(sizes, T, seed0=100):
    systems, queries, raw = {}, [], []
    for k, m in enumerate(sizes):
        q = W.osc_query(int(m), seed=seed0 + k, t_final=T)
        s = systems.setdefault(int(m), R.System("osc", 2 * int(m)))
        for method in ("mm", "cgb"):
            queries.append(dict(sys=s, method=method, x0_lo=q["x_lo"], x0_hi=q["x_hi"], w_lo=q["w_lo"],
                                w_hi=q["w_hi"], t_final=T, dt=q["dt"]))
            raw.append((method, q))
    return systems, queries, raw


@pytest.mark.parametrize("autotune", [True, False])
def test_osc_batch_matches_oracle_and_solo(autotune):
    sizes = [4, 5, 9, 17, 40, 77, 150, 333, 600, 1100, 2047, 2048, 2600, 4096]
    T = 0.1
    systems, queries, raw = _osc_batch(sizes, T)
    with R.Batch(queries, autotune=autotune) as b:
        st, fin = b.run()
        info = b.info()
        assert (st == 0).all() and (fin > 0).all()
        assert info["cpt"] in (2, 4, 8, 16) and info["kernels"] >= 2
        for (lo, hi), (method, q), qq in zip(b.outputs, raw, queries):
            o = O.reach(method, "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=q["dt"])
            assert_close(lo, o[0], TOL64, f"{method} m={qq['sys'].n // 2} lo")
            assert_close(hi, o[1], TOL64, f"{method} m={qq['sys'].n // 2} hi")
            fn = R.reach_mm if method == "mm" else R.reach_cgb
            solo = fn(qq["sys"], q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=q["dt"])
            assert np.array_equal(solo[0], lo) and np.array_equal(solo[1], hi)
    for s in systems.values():
        s.close()


@pytest.mark.parametrize("cluster_from", [0, 2048, 4096])
def test_mid_size_items_on_clusters_give_the_same_boxes(cluster_from):
    # the layout's second tuned dimension: items from cluster_from components
    # run on a two-block cluster instead of a bin slot; a component's
    # arithmetic does not depend on where it runs, so the boxes are the same
    # bit for bit, and they are the oracle's
    sizes = [9, 300, 520, 700, 1000, 1500, 2048]
    T = 0.05
    R.reach_set_option(R.OPT_BATCH_CPT, 16)
    R.reach_set_option(R.OPT_BATCH_CLUSTER_FROM, cluster_from)
    systems, queries, raw = _osc_batch(sizes, T, seed0=300)
    with R.Batch(queries) as b:
        st, _ = b.run()
        lay = b.layout()
        assert (st == 0).all()
        assert lay["cpt"] == 16 and lay["cluster_from"] == cluster_from and lay["create_s"] > 0
        for (lo, hi), (method, q), qq in zip(b.outputs, raw, queries):
            o = O.reach(method, "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=q["dt"])
            assert_close(lo, o[0], TOL64, f"{method} m={qq['sys'].n // 2} lo")
            assert_close(hi, o[1], TOL64, f"{method} m={qq['sys'].n // 2} hi")
            fn = R.reach_mm if method == "mm" else R.reach_cgb
            solo = fn(qq["sys"], q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=q["dt"])
            assert np.array_equal(solo[0], lo) and np.array_equal(solo[1], hi)
    for s in systems.values():
        s.close()


def test_tuner_reports_its_candidates():
    sizes = [4, 40, 600, 1100, 1500]
    systems, queries, _ = _osc_batch(sizes, 0.05, seed0=400)
    with R.Batch(queries) as b:
        lay = b.layout()
        assert lay["cpt"] in (2, 4, 8, 16) and lay["cluster_from"] in (0, 2048, 4096)
        assert {"cpt2", "cpt4", "cpt8", "cpt16"} <= set(lay["tune_ms"])
    for s in systems.values():
        s.close()


def test_mixed_kind_batch_with_device_buffers_and_replay():
    import torch
    T = 0.05
    qs, expect = [], []
    tr = W.traffic_small(16)
    s_tr = R.System("traffic", 16)
    s_ks = R.System("ks", 64)
    A = W.linear_general(6, seed=5, scale=0.5)
    s_li = R.System("linear", 6, A=A)
    ks = W.ks_grid(64, t_final=T)
    llo, lhi = W.random_box(6, seed=6)
    plo, phi = W.random_box(6, seed=7, centre=(-0.1, 0.1), width=(0.0, 0.05))
    dev = lambda v: torch.tensor(v, dtype=torch.float64, device="cuda")
    for method in ("mm", "cgb"):
        qs.append(dict(sys=s_tr, method=method, x0_lo=dev(tr["x_lo"]), x0_hi=dev(tr["x_hi"]),
                       w_lo=dev(tr["w_lo"]), w_hi=dev(tr["w_hi"]), t_final=T, dt=tr["dt"]))
        expect.append(O.reach(method, "traffic", tr["x_lo"], tr["x_hi"], tr["w_lo"], tr["w_hi"], t_final=T,
                              dt=tr["dt"]))
        qs.append(dict(sys=s_ks, method=method, x0_lo=ks["x_lo"], x0_hi=ks["x_hi"], t_final=T, dt=ks["dt"]))
        expect.append(O.reach(method, "ks", ks["x_lo"], ks["x_hi"], t_final=T, dt=ks["dt"], params=ks["params"]))
        qs.append(dict(sys=s_li, method=method, x0_lo=llo, x0_hi=lhi, w_lo=plo, w_hi=phi, t_final=T, dt=0.01))
        expect.append(O.reach(method, "linear", llo, lhi, plo, phi, t_final=T, dt=0.01, A=A))
    with R.Batch(qs) as b:
        st, _ = b.run()
        assert (st == 0).all()
        for (lo, hi), o in zip(b.outputs, expect):
            lo = lo.cpu().numpy() if hasattr(lo, "cpu") else lo
            hi = hi.cpu().numpy() if hasattr(hi, "cpu") else hi
            assert_close(lo, o[0], TOL64, "lo")
            assert_close(hi, o[1], TOL64, "hi")
        # replay after changing a host input in place: the graph reads it again
        new_lo = ks["x_lo"] - 1e-3
        qs[1]["x0_lo"][:] = new_lo
        st, _ = b.run()
        o = O.reach("mm", "ks", new_lo, ks["x_hi"], t_final=T, dt=ks["dt"], params=ks["params"])
        assert_close(b.outputs[1][0], o[0], TOL64, "replayed lo")
    for s in (s_tr, s_ks, s_li):
        s.close()


def test_batch_rejects_invalid_queries():
    with R.System("osc", 8) as s:
        q = W.osc_query(4, seed=1, t_final=0.1)
        good = dict(sys=s, method="mm", x0_lo=q["x_lo"], x0_hi=q["x_hi"], w_lo=q["w_lo"], w_hi=q["w_hi"],
                    t_final=0.1, dt=q["dt"])
        for bad in (dict(t_final=0.0), dict(dt=0.03), dict(x0_lo=q["x_hi"], x0_hi=q["x_lo"])):
            with pytest.raises(R.ReachError):
                R.Batch([good, dict(good, **bad)])


@pytest.mark.parametrize("cpt", [2, 4, 8, 16])
def test_every_batch_layout_matches_solo(cpt):
    sizes = [4, 31, 64, 200, 513, 1024, 3000]
    T = 0.05
    R.reach_set_option(R.OPT_BATCH_CPT, cpt)
    systems, queries, raw = _osc_batch(sizes, T, seed0=300)
    with R.Batch(queries) as b:
        st, _ = b.run()
        assert (st == 0).all() and b.info()["cpt"] == cpt
        for (lo, hi), (method, q), qq in zip(b.outputs, raw, queries):
            fn = R.reach_mm if method == "mm" else R.reach_cgb
            solo = fn(qq["sys"], q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=q["dt"])
            assert np.array_equal(solo[0], lo) and np.array_equal(solo[1], hi)
    for s in systems.values():
        s.close()


def test_full_osc_batch_sampled_queries_match_oracle():
    """The benchmark's batch as it runs there: 4096 queries x (MM to T = 5,
    CGB to T = 4), autotuned; sampled queries against the oracle."""
    sizes = W.osc_sizes(4096, seed=0)
    systems, queries, raw = {}, [], []
    for k, m in enumerate(sizes):
        q = W.osc_query(int(m), seed=1000003 + k, t_final=W.OSC_T)
        s = systems.setdefault(int(m), R.System("osc", 2 * int(m)))
        for method, T in (("mm", W.OSC_T), ("cgb", W.OSC_T_CGB)):
            queries.append(dict(sys=s, method=method, x0_lo=q["x_lo"], x0_hi=q["x_hi"], w_lo=q["w_lo"],
                                w_hi=q["w_hi"], t_final=T, dt=W.OSC_DT))
            raw.append((method, T, q))
    with R.Batch(queries) as b:
        st, fin = b.run()
        assert (st == 0).all() and (fin > 0).all()
        big = int(np.argmax(sizes))
        small = int(np.argmin(sizes))
        picks = sorted({2 * big, 2 * big + 1, 2 * small, 2 * small + 1, 1, 2 * 1234, 2 * 4095 + 1, 2 * 777 + 1})
        for i in picks:
            method, T, q = raw[i]
            lo, hi = b.outputs[i]
            o = O.reach(method, "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=T, dt=W.OSC_DT)
            assert_close(lo, o[0], TOL64, f"query {i} {method} lo")
            assert_close(hi, o[1], TOL64, f"query {i} {method} hi")
    for s in systems.values():
        s.close()


def test_heat_cubes_in_a_batch():
    # heat cubes of several sides (one block, and l = 18: 2n = 11664 on a
    # cluster) in one batch, both methods, against the oracle; the quadrotor
    # swarm is rejected (one call already runs every agent in one launch)
    qs, expect, systems = [], [], []
    T, dt = 0.2, 0.02
    for l, seed in ((3, 1), (7, 2), (12, 3), (18, 4)):
        lo, hi = W.random_box(l ** 3, seed=seed, centre=(0.0, 1.0), width=(0.0, 0.1))
        prm = (0.3 / (6 * dt * l * l), l, 1)
        s = R.System("heat", l ** 3, params=prm)
        systems.append(s)
        for method in ("mm", "cgb"):
            qs.append(dict(sys=s, method=method, x0_lo=lo, x0_hi=hi, t_final=T, dt=dt))
            expect.append(O.reach(method, "heat", lo, hi, t_final=T, dt=dt, params=prm))
    with R.Batch(qs) as b:
        st, _ = b.run()
        assert (st == 0).all()
        for (lo, hi), o in zip(b.outputs, expect):
            assert_close(lo, o[0], TOL64, "lo")
            assert_close(hi, o[1], TOL64, "hi")
    q = W.quad_swarm(2, seed=1)
    with R.System("quad", 24) as sq:
        with pytest.raises(R.ReachError):
            R.Batch([dict(sys=sq, method="mm", x0_lo=q["x_lo"], x0_hi=q["x_hi"], w_lo=q["w_lo"], w_hi=q["w_hi"],
                          t_final=0.1, dt=0.01)])
    for s in systems:
        s.close()
