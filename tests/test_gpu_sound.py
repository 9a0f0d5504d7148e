"""Outward-rounded traffic MM and CGB (reading R15) on the GPU.

The kernel performs the oracle's operations in the oracle's order, each with
its directed-rounding instruction, so the two boxes agree bit for bit; the
outward box also contains the round-to-nearest box of the same call."""
import numpy as np
import pytest

import oracle as O
import paper_2001_10635_b300 as R
import workloads as W
from reachtest import cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]

SOUND = O.TRAFFIC_SOUND_PRM


@pytest.fixture(autouse=True)
def _reset_options():
    yield
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 0)


def boxes(n, seed):
    g = np.random.default_rng(seed)
    c = g.uniform(5, 310, n)
    h = g.uniform(0, 6, n)
    return c - h, c + h, np.array([35.0]), np.array([45.0])


def run(method, n, args, T, dt, params):
    with R.System("traffic", n, params=params) as s:
        f = R.reach_mm if method == "mm" else R.reach_cgb
        return f(s, *args, t_final=T, dt=dt)


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("n,S", [(1, 1), (2, 1), (16, 1), (300, 2), (4097, 1), (4097, 3)])
def test_sound_matches_oracle_bit_for_bit(method, n, S):
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    args = boxes(n, seed=n + S)
    T, dt = 0.37, 0.01
    o = O.reach(method, "traffic", *args, t_final=T, dt=dt, params=SOUND)
    g = run(method, n, args, T, dt, SOUND)
    np.testing.assert_array_equal(g[0], o[0])
    np.testing.assert_array_equal(g[1], o[1])


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_sound_contains_the_nearest_rounded_box(method):
    wl = W.traffic_large(1 << 20, seed=5, t_final=2.0)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    a = run(method, 1 << 20, args, 2.0, 0.01, None)
    b = run(method, 1 << 20, args, 2.0, 0.01, SOUND)
    assert np.all(b[0] <= a[0]) and np.all(b[1] >= a[1])
    scale = np.abs(a[1]).max()
    assert np.max(a[0] - b[0]) < 1e-11 * scale and np.max(b[1] - a[1]) < 1e-11 * scale


def test_sound_rejections():
    with pytest.raises(R.ReachError):
        R.System("traffic", 8, params=(40.0, 0.5, 1 / 6, 320.0, 1, 1))
    wl = W.traffic_small(16)
    with R.System("traffic", 16, params=SOUND) as s:
        with pytest.raises(R.ReachError):
            R.reach_pipe(s, "mm", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=1.0, dt=0.01, every=10)
