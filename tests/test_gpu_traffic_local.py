"""Parity of traffic CGB with the box-evaluated contraction matrix (reading
R14) with the FP64 oracle: the on-chip kernel, the streaming kernel (several
steps per launch, ragged tiles, a non-power-of-two v) and sampled cells of the
2^26-cell chain, each recomputed by the oracle on a window wider than its
RK4 domain of dependence."""
import numpy as np
import pytest

import oracle as O
import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

LOCAL = O.TRAFFIC_LOCAL_PRM


@pytest.fixture(autouse=True)
def _reset_options():
    yield
    R.reach_set_option(R.OPT_KERNEL, 0)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 0)


def boxes(n, seed):
    # densities across the free-flow, capacity and congested regimes
    g = np.random.default_rng(seed)
    c = g.uniform(5, 310, n)
    h = g.uniform(0, 6, n)
    return c - h, c + h, np.array([35.0]), np.array([45.0])


def gpu_cgb(n, lo, hi, wlo, whi, T, dt, params):
    with R.System("traffic", n, params=params) as s:
        return R.reach_cgb(s, lo, hi, wlo, whi, t_final=T, dt=dt)


@pytest.mark.parametrize("kernel,n,S", [(0, 16, 1), (0, 200, 1), (2, 3000, 1), (1, 300, 1), (1, 1000, 3),
                                         (1, 4097, 1), (1, 4097, 2)])
def test_local_cgb_matches_oracle(kernel, n, S):
    R.reach_set_option(R.OPT_KERNEL, kernel)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    lo, hi, wlo, whi = boxes(n, seed=n)
    T, dt = 0.37, 0.01
    olo, ohi = O.reach("cgb", "traffic", lo, hi, wlo, whi, t_final=T, dt=dt, params=LOCAL)
    glo, ghi = gpu_cgb(n, lo, hi, wlo, whi, T, dt, LOCAL)
    assert_close(glo, olo, TOL64, "lo")
    assert_close(ghi, ohi, TOL64, "hi")


@pytest.mark.parametrize("v", [0.45, 0.25])
def test_local_cgb_parameters(v):
    prm = (38.0, v, 0.2, 300.0, 1)
    n = 3001
    R.reach_set_option(R.OPT_KERNEL, 1)
    lo, hi, wlo, whi = boxes(n, seed=17)
    o = O.reach("cgb", "traffic", lo, hi, wlo, whi, t_final=0.3, dt=0.01, params=prm)
    g = gpu_cgb(n, lo, hi, wlo, whi, 0.3, 0.01, prm)
    assert_close(g[0], o[0], TOL64, "lo")
    assert_close(g[1], o[1], TOL64, "hi")


def test_local_cgb_is_inside_the_global_box():
    wl = W.traffic_large(1 << 16, seed=3, t_final=1.0)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    loc = gpu_cgb(1 << 16, *args, 1.0, 0.01, LOCAL)
    glob = gpu_cgb(1 << 16, *args, 1.0, 0.01, O.TRAFFIC_PRM)
    assert np.all(loc[0] >= glob[0] - 1e-9) and np.all(loc[1] <= glob[1] + 1e-9)
    assert np.sum(loc[1] - loc[0]) < np.sum(glob[1] - glob[0])


def test_local_cgb_full_size_sampled_cells():
    wl = W.traffic_large(1 << 26, seed=0)
    n, T, dt = 1 << 26, wl["t_final"], wl["dt"]
    N = O.nsteps(T, dt)
    g = gpu_cgb(n, wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], T, dt, LOCAL)
    for i in [0, 1, 5, 4 * N, 12345678, n // 2 + 17, n - 4 * N - 3, n - 2, n - 1]:
        a, b = max(0, i - 4 * N - 2), min(n, i + 4 * N + 3)
        olo, ohi = O.reach("cgb", "traffic", wl["x_lo"][a:b], wl["x_hi"][a:b], wl["w_lo"], wl["w_hi"],
                           t_final=T, dt=dt, params=LOCAL)
        assert_close(g[0][i:i + 1], olo[i - a:i - a + 1], TOL64, f"cell {i} lo")
        assert_close(g[1][i:i + 1], ohi[i - a:i - a + 1], TOL64, f"cell {i} hi")
