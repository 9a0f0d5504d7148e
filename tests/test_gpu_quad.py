"""Parity of the quadrotor-swarm path (Sec. 5.2) with the FP64 oracle.

The agents are independent, so the 1.2e8-state swarm (10^7 agents, the
largest the paper reports on a GPU) is checked on sampled agents, each
recomputed by the oracle on its own; smaller swarms are compared whole,
including a ragged last block of threads.
"""
import numpy as np
import pytest

import oracle as O
import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL32, TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

PRM = (1.4, 9.81, 1.4 * 9.81, 0.054, 0.061, 0.104)


def gpu(method, n, wl, T, dt, params=PRM, **kw):
    with R.System("quad", n, params=params) as s:
        args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
        if method == "mm":
            return R.reach_mm(s, *args, t_final=T, dt=dt)
        if method == "cgb":
            return R.reach_cgb(s, *args, t_final=T, dt=dt)
        return R.reach_mc(s, *args, t_final=T, dt=dt, **kw)


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("K", [1, 3, 130])
def test_swarm_matches_oracle(method, K):
    wl = W.quad_swarm(K, seed=K)
    T, dt = 1.0, 0.01
    olo, ohi = O.reach(method, "quad", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T, dt=dt,
                       params=PRM)
    glo, ghi = gpu(method, 12 * K, wl, T, dt)
    assert_close(glo, olo, TOL64, f"{method} K={K} lo")
    assert_close(ghi, ohi, TOL64, f"{method} K={K} hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_wide_yaw_intervals(method):
    # yaw boxes wide enough to hold extrema of sine and cosine, and one of
    # more than a full turn
    wl = W.quad_swarm(4, seed=9)
    wl["x_lo"][8::12] = [-0.5, 1.0, 2.9, -4.0]
    wl["x_hi"][8::12] = [0.5, 2.2, 3.4, 3.0]
    T, dt = 0.5, 0.01
    olo, ohi = O.reach(method, "quad", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T, dt=dt,
                       params=PRM)
    glo, ghi = gpu(method, 48, wl, T, dt)
    assert_close(glo, olo, TOL64, f"{method} lo")
    assert_close(ghi, ohi, TOL64, f"{method} hi")


@pytest.mark.parametrize("prec,tol", [(64, TOL64), (32, TOL32)])
@pytest.mark.parametrize("m", [1, 100])
def test_mc_matches_oracle(prec, tol, m):
    K = 5
    wl = W.quad_swarm(K, seed=21)
    T, dt = 1.0, 0.01
    olo, ohi = O.reach("mc", "quad", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T, dt=dt,
                       params=PRM, m=m, seed=77, prec=prec)
    glo, ghi = gpu("mc", 12 * K, wl, T, dt, m=m, seed=77, precision=prec)
    assert_close(glo, olo, tol, f"mc{prec} lo")
    assert_close(ghi, ohi, tol, f"mc{prec} hi")


@pytest.mark.parametrize("prec,tol", [(64, TOL64), (32, TOL32)])
def test_mc_fast_rotation(prec, tol):
    # angular rates around the point where a stage's angle increment h/2 w
    # passes 1/16 (12.5 rad/s at dt = 0.01): above it the stages halve the
    # increment into the range of its sine and cosine series and double the
    # values back, below it they take the series directly; rates of
    # 12.4..12.6 rad/s split one warp's samples between the two, 150 rad/s
    # takes four halvings, and 50 steps take the step-start values afresh once
    # after the first step
    wl = W.quad_swarm(5, seed=41)
    for k, (lo, hi) in enumerate([(19.9, 20.1), (4.9, 5.1), (12.4, 12.6), (-30.1, -29.9), (149.9, 150.1)]):
        for d in range(3):
            wl["x_lo"][12 * k + 9 + d] = lo * (1 - 0.2 * d)
            wl["x_hi"][12 * k + 9 + d] = hi * (1 - 0.2 * d)
    T, dt = 0.5, 0.01
    olo, ohi = O.reach("mc", "quad", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T, dt=dt,
                       params=PRM, m=100, seed=3, prec=prec)
    glo, ghi = gpu("mc", 60, wl, T, dt, m=100, seed=3, precision=prec)
    assert_close(glo, olo, tol, f"mc{prec} lo")
    assert_close(ghi, ohi, tol, f"mc{prec} hi")


def test_point_box_and_containment():
    K = 8
    wl = W.quad_swarm(K, seed=31)
    T, dt = 1.0, 0.01
    with R.System("quad", 12 * K, params=PRM) as s:
        args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
        mlo, mhi = R.reach_mm(s, *args, t_final=T, dt=dt)
        clo, chi = R.reach_cgb(s, *args, t_final=T, dt=dt)
        slo, shi = R.reach_mc(s, *args, t_final=T, dt=dt, m=256, seed=5, precision=64)
        assert np.all(mlo <= slo) and np.all(shi <= mhi)
        assert np.all(clo <= slo) and np.all(shi <= chi)
        x0 = (wl["x_lo"] + wl["x_hi"]) / 2
        t0 = (wl["w_lo"] + wl["w_hi"]) / 2
        plo, phi = R.reach_mm(s, x0, x0, t0, t0, t_final=T, dt=dt)
    traj = O.flow("quad", x0, t0, t_final=T, dt=dt, params=PRM)
    assert_close(plo, traj, TOL64, "point lo")
    assert_close(phi, traj, TOL64, "point hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_full_size_swarm_sampled_agents(method):
    import torch
    K = 10_000_000
    n = 12 * K
    wl = W.quad_swarm(K, seed=0, t_final=0.2)
    dev = torch.device("cuda", 0)
    d = {k: torch.from_numpy(wl[k]).to(dev) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    with R.System("quad", n) as s:
        f = R.reach_mm if method == "mm" else R.reach_cgb
        glo, ghi = f(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    glo, ghi = glo.cpu().numpy(), ghi.cpu().numpy()
    rng = np.random.default_rng(3)
    for k in [0, 1, 127, 128, K - 1] + list(rng.integers(0, K, 20)):
        s12, s3 = slice(12 * k, 12 * k + 12), slice(3 * k, 3 * k + 3)
        olo, ohi = O.reach(method, "quad", wl["x_lo"][s12], wl["x_hi"][s12], wl["w_lo"][s3], wl["w_hi"][s3],
                           t_final=wl["t_final"], dt=wl["dt"], params=W.QUAD_PRM)
        assert_close(glo[s12], olo, TOL64, f"{method} agent {k} lo")
        assert_close(ghi[s12], ohi, TOL64, f"{method} agent {k} hi")


def test_rejected_sizes():
    with pytest.raises(R.ReachError):
        R.System("quad", 13)
    with pytest.raises(R.ReachError):
        R.System("quad", 12, params=(0.0, 9.81, 1.0, 0.05, 0.05, 0.1))
