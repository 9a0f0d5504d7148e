"""Parity of the 3-D heat-diffusion path (Sec. 5.4) with the FP64 oracle.

Small cubes run on the on-chip kernel (2n <= 1024) and, forced through
REACH_OPT_KERNEL, on the streaming stage kernels; larger cubes with ragged
tiles (l not a multiple of the 32 x 8 block) run on the stage kernels only.
The l = 1000 cube of the paper (10^9 cells) is checked on sampled cells, each
recomputed by the oracle on a sub-cube that extends 4 N + 1 cells beyond it in
every direction where the grid allows (RK4 applies the 7-point operator four
times a step), so the sub-cube's own faces cannot reach the sampled cell.
"""
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


def random_cube(l, seed):
    """Per-cell random box (no symmetry between the axes to hide a swapped index)."""
    lo, hi = W.random_box(l ** 3, seed=seed, centre=(0.0, 1.0), width=(0.0, 0.1))
    return lo, hi


def run(method, l, lo, hi, T, dt, params):
    with R.System("heat", l ** 3, params=params) as s:
        f = R.reach_mm if method == "mm" else R.reach_cgb
        return f(s, lo, hi, t_final=T, dt=dt)


CASES = [(1, 1), (2, 0), (3, 1), (5, 1), (5, 0), (8, 1)]


@pytest.mark.parametrize("kernel", [0, 1], ids=["auto", "stream"])
@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("l,open_face", CASES, ids=[f"l{l}o{o}" for l, o in CASES])
def test_small_cube_matches_oracle(l, open_face, method, kernel):
    R.reach_set_option(R.OPT_KERNEL, kernel)
    lo, hi = random_cube(l, seed=l)
    prm = (0.05, l, open_face)   # h 6 alpha l^2 stays below 1 at these sizes
    T, dt = 0.4, 0.02
    olo, ohi = O.reach(method, "heat", lo, hi, t_final=T, dt=dt, params=prm)
    glo, ghi = run(method, l, lo, hi, T, dt, prm)
    assert_close(glo, olo, TOL64, f"{method} l={l} lo")
    assert_close(ghi, ohi, TOL64, f"{method} l={l} hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("l", [9, 16, 21, 40, 97])
def test_stage_kernels_match_oracle(l, method):
    # l = 97: thread blocks (32 x 8 cells of a plane) inside the cube as well as
    # on each of its faces
    lo, hi = random_cube(l, seed=100 + l)
    alpha = 0.5 / (6 * 0.02 * l * l)   # h 6 kh = 0.5: strong diffusion per step
    prm = (alpha, l, 1)
    T, dt = 0.5, 0.02
    olo, ohi = O.reach(method, "heat", lo, hi, t_final=T, dt=dt, params=prm)
    glo, ghi = run(method, l, lo, hi, T, dt, prm)
    assert_close(glo, olo, TOL64, f"{method} l={l} lo")
    assert_close(ghi, ohi, TOL64, f"{method} l={l} hi")


def test_default_parameters_and_workload():
    """The paper's workload shape on a 24^3 cube: the default alpha, the open
    face, the heated region; MM and CGB coincide with the exact hull for this
    linear Metzler system, so they agree with each other too."""
    wl = W.heat_cube(24, t_final=1.0)
    olo, ohi = O.reach("mm", "heat", wl["x_lo"], wl["x_hi"], t_final=wl["t_final"], dt=wl["dt"])
    with R.System("heat", 24 ** 3) as s:
        mlo, mhi = R.reach_mm(s, wl["x_lo"], wl["x_hi"], t_final=wl["t_final"], dt=wl["dt"])
        clo, chi = R.reach_cgb(s, wl["x_lo"], wl["x_hi"], t_final=wl["t_final"], dt=wl["dt"])
    assert_close(mlo, olo, TOL64, "mm lo")
    assert_close(mhi, ohi, TOL64, "mm hi")
    assert_close(clo, mlo, 1e-12, "cgb lo vs mm")
    assert_close(chi, mhi, 1e-12, "cgb hi vs mm")


def test_heat_mc_inside_mm():
    l = 4
    lo, hi = random_cube(l, seed=7)
    prm = (0.05, l, 1)
    with R.System("heat", l ** 3, params=prm) as s:
        mlo, mhi = R.reach_mm(s, lo, hi, t_final=0.4, dt=0.02)
        slo, shi = R.reach_mc(s, lo, hi, t_final=0.4, dt=0.02, m=200, seed=3, precision=64)
    olo, ohi = O.reach("mc", "heat", lo, hi, t_final=0.4, dt=0.02, params=prm, m=200, seed=3)
    assert_close(slo, olo, TOL64, "mc lo")
    assert_close(shi, ohi, TOL64, "mc hi")
    # every sample inside the MM box exactly (Sec. 2.1); an escape is reported with its margin
    assert (slo - mlo).min() >= 0.0, ("below", (slo - mlo).min())
    assert (mhi - shi).min() >= 0.0, ("above", (mhi - shi).min())


def _window(c, r, l):
    w = min(l, 2 * r + 1)
    s = min(max(c - r, 0), l - w)
    return s, w


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_full_size_cube_sampled_cells(method):
    import torch
    l, N = 1000, 5
    dt = W.HEAT_DT
    T = N * dt
    dev = torch.device("cuda", 0)
    need = 10 * 8 * l ** 3 + (1 << 30)
    if torch.cuda.mem_get_info(dev)[0] < need:
        pytest.skip("not enough device memory for the 10^9-cell cube")
    xlo, xhi = W.heat_cube_torch(l, dev)
    with R.System("heat", l ** 3) as s:
        f = R.reach_mm if method == "mm" else R.reach_cgb
        glo, ghi = f(s, xlo, xhi, t_final=T, dt=dt)
    del xlo, xhi
    glo = glo.view(l, l, l)
    ghi = ghi.view(l, l, l)
    hot = W.heat_hot_cells(l)
    r = 4 * N + 1
    # (z, y, x): corners, the open face, the heated region's edge and centre
    cells = [(0, 0, 0), (999, 999, 999), (0, 500, 500), (999, 0, 500), (400, 400, 400),
             (399, 500, 600), (599, 599, 599), (500, 500, 500), (10, 987, 3)]
    for (z, y, x) in cells:
        (sz, w), (sy, _), (sx, _) = _window(z, r, l), _window(y, r, l), _window(x, r, l)
        # the initial box of heat_cube restricted to the sub-cube
        m = (hot[sz:sz + w, None, None] & hot[None, sy:sy + w, None] & hot[None, None, sx:sx + w]).ravel()
        sub_lo, sub_hi = np.where(m, 0.9, 0.0), np.where(m, 1.1, 0.01)
        # the sub-cube keeps the full grid's spacing 1/l: alpha / dx^2 unchanged
        alpha_w = W.HEAT_ALPHA * (l / w) ** 2
        olo, ohi = O.reach(method, "heat", sub_lo, sub_hi, t_final=T, dt=dt,
                           params=(alpha_w, w, 1 if sz == 0 else 0))
        k = ((z - sz) * w + (y - sy)) * w + (x - sx)
        g = np.array([glo[z, y, x].item(), ghi[z, y, x].item()])
        o = np.array([olo[k], ohi[k]])
        assert_close(g, o, TOL64, f"{method} cell {(z, y, x)}")
