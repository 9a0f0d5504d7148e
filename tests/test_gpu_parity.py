"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Small and ragged sizes are compared element by element on both kernels (the
on-chip whole-horizon kernel and the streaming stencil kernel, forced through
REACH_OPT_KERNEL), with several steps per launch; the full-size workloads of
the benchmark are compared on sampled cells, each recomputed by the oracle on a
window wider than its RK4 domain of dependence (4 R cells per step and side),
which makes the window's own boundary irrelevant to that cell.
"""
import math

import numpy as np
import pytest

import oracle as O
import paper_2001_10635_b300 as R
import workloads as W
from reachtest import TOL32, TOL64, assert_close, cuda_available

pytestmark = [pytest.mark.gpu,
              pytest.mark.skipif(not cuda_available(), reason="needs a CUDA device")]


@pytest.fixture(autouse=True)
def _reset_options():
    yield
    R.reach_set_option(R.OPT_KERNEL, 0)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 0)
    R.reach_set_option(R.OPT_BLOCK, 0)
    R.reach_set_option(R.OPT_TILE, 0)
    R.reach_set_option(R.OPT_MC_SB, 0)
    R.reach_set_option(R.OPT_MC_LAYOUT, 0)


def gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=None, A=None, **kw):
    with R.System(kind, n, params=params, A=A) as s:
        if method == "mm":
            return R.reach_mm(s, lo, hi, wlo, whi, t_final=T, dt=dt)
        if method == "cgb":
            return R.reach_cgb(s, lo, hi, wlo, whi, t_final=T, dt=dt)
        return R.reach_mc(s, lo, hi, wlo, whi, t_final=T, dt=dt, **kw)


def problem(kind, n, seed=0):
    """(lo, hi, wlo, whi, T, dt, params, A) of a small test problem."""
    g = np.random.default_rng(seed)
    if kind == "traffic":
        c = g.uniform(60, 200, n)
        return c - 4, c + 4, np.array([35.0]), np.array([45.0]), 1.0, 0.01, None, None
    if kind == "ks":
        u = W.ks_profile(n) + g.uniform(-0.01, 0.01, n)
        return u - 1e-3, u + 1e-3, None, None, 0.01, 1e-4, None, None
    if kind == "osc":
        m = n // 2
        q = W.osc_query(m, seed=seed, half_width=1e-3, t_final=1.0)
        return q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], 1.0, 0.005, None, None
    if kind == "heat":
        lo, hi = W.random_box(n, seed=seed, centre=(0.0, 1.0), width=(0.0, 0.1))
        return lo, hi, None, None, 0.2, 0.02, None, None
    if kind == "quad":
        q = W.quad_swarm(n // 12, seed=seed, t_final=0.5)
        return q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], 0.5, q["dt"], None, None
    A = W.linear_general(n, seed=seed, scale=0.5)
    lo, hi = W.random_box(n, seed=seed + 1)
    plo, phi = W.random_box(n, seed=seed + 2, centre=(-0.1, 0.1), width=(0.0, 0.05))
    return lo, hi, plo, phi, 1.0, 0.01, None, A


SMALL = [("traffic", 1), ("traffic", 2), ("traffic", 16), ("traffic", 37), ("ks", 5), ("ks", 64),
         ("ks", 200), ("osc", 2), ("osc", 8), ("osc", 302), ("linear", 1), ("linear", 7), ("linear", 64)]


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("kind,n", SMALL, ids=[f"{k}{n}" for k, n in SMALL])
def test_onchip_matches_oracle(method, kind, n):
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=n)
    olo, ohi = O.reach(method, kind, lo, hi, wlo, whi, t_final=T, dt=dt, params=prm, A=A)
    glo, ghi = gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=prm, A=A)
    assert_close(glo, olo, TOL64, f"{method} {kind} lo")
    assert_close(ghi, ohi, TOL64, f"{method} {kind} hi")


# S = 0: the library's own choice (4 steps per launch for these short traffic
# chains, 2 for these KS grids, 1 for the longer ones)
STREAM = [("traffic", 300, 1), ("traffic", 1000, 3), ("traffic", 4097, 1), ("traffic", 4097, 2),
          ("traffic", 5000, 0), ("traffic", 20011, 0), ("ks", 256, 1), ("ks", 777, 2), ("ks", 3001, 1),
          ("ks", 3001, 0), ("ks", 30001, 0)]


@pytest.mark.parametrize("tile", [2, 8])
@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("kind,n,S", STREAM, ids=[f"{k}{n}S{s}" for k, n, s in STREAM])
def test_streaming_kernel_matches_oracle(method, kind, n, S, tile):
    # both warp-tile widths (64-cell tiles fall back to 256 where the KS halo
    # of three steps per launch would not leave half the tile)
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=n)
    T = 0.37 if kind == "traffic" else 0.005   # 37 / 50 steps: ragged against S
    R.reach_set_option(R.OPT_KERNEL, 1)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    R.reach_set_option(R.OPT_TILE, tile)
    olo, ohi = O.reach(method, kind, lo, hi, wlo, whi, t_final=T, dt=dt, params=prm)
    glo, ghi = gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=prm)
    assert_close(glo, olo, TOL64, f"{method} {kind} lo")
    assert_close(ghi, ohi, TOL64, f"{method} {kind} hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("kind,n", [("traffic", 100003), ("ks", 50001)])
def test_tile_widths_agree_bit_for_bit(method, kind, n):
    # a cell's arithmetic does not depend on the tile that computes it: the
    # 64-cell and 256-cell tiles give the same box, and it is the oracle's
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=5)
    T = 0.2 if kind == "traffic" else 0.003
    R.reach_set_option(R.OPT_KERNEL, 1)
    R.reach_set_option(R.OPT_TILE, 2)
    nlo, nhi = gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=prm)
    R.reach_set_option(R.OPT_TILE, 8)
    wlo_, whi_ = gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=prm)
    assert np.array_equal(nlo, wlo_) and np.array_equal(nhi, whi_)
    olo, ohi = O.reach(method, kind, lo, hi, wlo, whi, t_final=T, dt=dt, params=prm)
    assert_close(nlo, olo, TOL64, f"{method} {kind} lo")
    assert_close(nhi, ohi, TOL64, f"{method} {kind} hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_large_onchip_traffic_matches_oracle(method):
    lo, hi, wlo, whi, T, dt, prm, A = problem("traffic", 4000, seed=3)
    R.reach_set_option(R.OPT_KERNEL, 2)
    olo, ohi = O.reach(method, "traffic", lo, hi, wlo, whi, t_final=0.2, dt=dt)
    glo, ghi = gpu_box(method, "traffic", 4000, lo, hi, wlo, whi, 0.2, dt)
    assert_close(glo, olo, TOL64, "lo")
    assert_close(ghi, ohi, TOL64, "hi")


def test_device_pointers_match_host_pointers():
    import torch
    lo, hi, wlo, whi, T, dt, _, _ = problem("traffic", 5000, seed=9)
    with R.System("traffic", 5000) as s:
        a = R.reach_mm(s, lo, hi, wlo, whi, t_final=0.5, dt=dt)
        d = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in (lo, hi, wlo, whi)]
        b = R.reach_mm(s, *d, t_final=0.5, dt=dt)
        torch.cuda.synchronize()
    assert np.array_equal(a[0], b[0].cpu().numpy()) and np.array_equal(a[1], b[1].cpu().numpy())


# ------------------------------------------------------------------ traffic, n = 16 (the small chain)
def test_traffic16_all_methods():
    wl = W.traffic_small(16)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    kw = dict(t_final=wl["t_final"], dt=wl["dt"])
    boxes = {}
    for method in ("mm", "cgb"):
        o = O.reach(method, "traffic", *args, **kw)
        g = gpu_box(method, "traffic", 16, *args, wl["t_final"], wl["dt"])
        assert_close(g[0], o[0], TOL64, method)
        assert_close(g[1], o[1], TOL64, method)
        boxes[method] = g
    for prec, tol in ((64, TOL64), (32, TOL32)):
        o = O.reach("mc", "traffic", *args, **kw, m=1000, seed=0, prec=prec)
        g = gpu_box("mc", "traffic", 16, *args, wl["t_final"], wl["dt"], m=1000, seed=0, precision=prec)
        assert_close(g[0], o[0], tol, f"mc{prec} lo")
        assert_close(g[1], o[1], tol, f"mc{prec} hi")
        if prec == 64:   # every sample inside the MM and CGB boxes, exactly
            for b in boxes.values():
                assert (g[0] >= b[0]).all() and (g[1] <= b[1]).all()


# ------------------------------------------------------------------ Monte Carlo
MC = [("traffic", 5, 33, 64), ("traffic", 40, 70, 32), ("ks", 64, 70, 64), ("ks", 64, 70, 32),
      ("osc", 8, 100, 64), ("osc", 40, 45, 32), ("linear", 5, 33, 64), ("linear", 12, 1, 32)]


@pytest.mark.parametrize("sb", [0, 8, 32])
@pytest.mark.parametrize("kind,n,m,prec", MC, ids=[f"{k}{n}m{m}p{p}" for k, n, m, p in MC])
def test_mc_onchip_matches_oracle(kind, n, m, prec, sb):
    # sb: samples per block of the on-chip kernel (0: the library's choice, 2
    # for these sample counts)
    R.reach_set_option(R.OPT_MC_SB, sb)
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=7)
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, A=A, m=m, seed=11, prec=prec)
    g = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, A=A, m=m, seed=11, precision=prec)
    tol = TOL64 if prec == 64 else TOL32
    assert_close(g[0], o[0], tol, "lo")
    assert_close(g[1], o[1], tol, "hi")


@pytest.mark.parametrize("prec", [64, 32])
def test_mc_small_chain_same_box_for_every_block_shape(prec):
    # the n = 16 chain over T = 10 with 1000 samples: blocks of 2, 8 and 32
    # samples draw the same samples and give the same box bit for bit, and it
    # is the oracle's
    wl = W.traffic_small(16)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    boxes = []
    for sb in (2, 8, 32):
        R.reach_set_option(R.OPT_MC_SB, sb)
        boxes.append(gpu_box("mc", "traffic", 16, *args, wl["t_final"], wl["dt"], m=1000, seed=0, precision=prec))
    for b in boxes[1:]:
        assert np.array_equal(b[0], boxes[0][0]) and np.array_equal(b[1], boxes[0][1])
    o = O.reach("mc", "traffic", *args, t_final=wl["t_final"], dt=wl["dt"], m=1000, seed=0, prec=prec)
    tol = TOL64 if prec == 64 else TOL32
    assert_close(boxes[0][0], o[0], tol, "lo")
    assert_close(boxes[0][1], o[1], tol, "hi")


MCS = [("traffic", 700, 70, 64), ("traffic", 300, 33, 32), ("ks", 600, 40, 64), ("ks", 513, 65, 32)]


@pytest.mark.parametrize("kind,n,m,prec", MCS, ids=[f"{k}{n}m{m}p{p}" for k, n, m, p in MCS])
def test_mc_streaming_matches_oracle(kind, n, m, prec):
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=5)
    T = 0.13 if kind == "traffic" else 0.003
    R.reach_set_option(R.OPT_KERNEL, 1)
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, m=m, seed=3, prec=prec)
    g = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, m=m, seed=3, precision=prec)
    tol = TOL64 if prec == 64 else TOL32
    assert_close(g[0], o[0], tol, "lo")
    assert_close(g[1], o[1], tol, "hi")


# ------------------------------------------------------------------ edge cases
@pytest.mark.parametrize("method", ["mm", "cgb", "mc"])
def test_zero_horizon_returns_the_box(method):
    lo, hi, wlo, whi, T, dt, _, _ = problem("traffic", 50)
    kw = dict(m=5) if method == "mc" else {}
    g = gpu_box(method, "traffic", 50, lo, hi, wlo, whi, 0.0, dt, **kw)
    if method == "mc":
        assert (g[0] >= lo).all() and (g[1] <= hi).all()
    else:
        assert np.array_equal(g[0], lo) and np.array_equal(g[1], hi)


@pytest.mark.parametrize("kind", ["traffic", "ks", "osc", "linear"])
def test_zero_width_box_is_one_trajectory(kind):
    n = 6 if kind != "ks" else 16
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=1)
    x = 0.5 * (lo + hi)
    w = None if wlo is None else 0.5 * (wlo + whi)
    traj = O.flow(kind, x, w, t_final=T, dt=dt, A=A)
    for method in ("mm", "cgb"):
        g = gpu_box(method, kind, n, x, x, w, w, T, dt, A=A)
        assert_close(g[0], traj, TOL64, method)
        assert_close(g[1], traj, TOL64, method)
    g = gpu_box("mc", kind, n, x, x, w, w, T, dt, A=A, m=40)
    assert_close(g[0], traj, TOL64, "mc")
    assert np.array_equal(g[0], g[1])


def test_invalid_arguments_are_rejected():
    lo, hi, wlo, whi, T, dt, _, _ = problem("traffic", 20)
    with R.System("traffic", 20) as s:
        bad = [dict(t_final=1.0, dt=0.0), dict(t_final=1.0, dt=0.3), dict(t_final=-1.0, dt=0.1),
               dict(t_final=float("nan"), dt=0.1)]
        for kw in bad:
            with pytest.raises(R.ReachError) as e:
                R.reach_mm(s, lo, hi, wlo, whi, **kw)
            assert e.value.code == -1
        with pytest.raises(R.ReachError):
            R.reach_mm(s, hi, lo, wlo, whi, t_final=T, dt=dt)   # lo > hi
        with pytest.raises(R.ReachError):
            R.reach_cgb(s, lo, hi, whi, wlo, t_final=T, dt=dt)  # input lo > hi
        nan = lo.copy()
        nan[3] = np.nan
        with pytest.raises(R.ReachError):
            R.reach_mm(s, nan, hi, wlo, whi, t_final=T, dt=dt)
        for kw in (dict(m=0), dict(m=5, precision=16)):
            with pytest.raises(R.ReachError):
                R.reach_mc(s, lo, hi, wlo, whi, t_final=T, dt=dt, **kw)
    for args in [("osc", 5), ("ks", 3), ("traffic", 0)]:
        with pytest.raises(R.ReachError):
            R.System(*args)


def test_device_side_input_check():
    import torch
    lo, hi, wlo, whi, T, dt, _, _ = problem("traffic", 3000)
    d = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in (hi, lo, wlo, whi)]   # swapped
    with R.System("traffic", 3000) as s:
        for f in (R.reach_mm, R.reach_cgb):
            with pytest.raises(R.ReachError) as e:
                f(s, *d, t_final=T, dt=dt)
            assert e.value.code == -1


def test_nonfinite_result_is_reported():
    n = 16
    lo, hi = np.full(n, -10.0), np.full(n, 10.0)
    with pytest.raises(O.OracleError):
        O.reach("mm", "ks", lo, hi, t_final=2.0, dt=1e-3)
    with R.System("ks", n) as s:
        with pytest.raises(R.ReachError) as e:
            R.reach_mm(s, lo, hi, t_final=2.0, dt=1e-3)
    assert e.value.code == -4


# ------------------------------------------------------------------ full-size workloads, sampled
def _window(i, n, radius_cells):
    a = max(0, i - radius_cells)
    b = min(n, i + radius_cells + 1)
    return a, b


# Cells a 256-cell warp tile owns at one RK4 step per launch: 256 minus a
# halo of 4 R cells per side (traffic R = 1, KS R = 2).  Tile t owns
# [t W, (t + 1) W); the first and last tiles take the chain's boundary path,
# the others the interior path.
TRAFFIC_OWNED = 256 - 2 * 4
KS_OWNED = 256 - 2 * 8


def _tile_edge_cells(n, W):
    """Cells at the offsets 0, 1, W/2 - 1, W - 2, W - 1 of the first and last
    interior tiles and of a middle tile, and the first, second and last cell
    of the last (ragged) tile."""
    ntiles = -(-n // W)
    cells = []
    for t in (1, ntiles // 2, ntiles - 2):
        cells += [t * W + o for o in (0, 1, W // 2 - 1, W - 2, W - 1)]
    last = (ntiles - 1) * W
    cells += [last, last + 1, n - 1]
    return [c for c in cells if 0 <= c < n]


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_traffic_full_size_sampled_cells(method):
    wl = W.traffic_large(1 << 26, seed=0)
    n, T, dt = 1 << 26, wl["t_final"], wl["dt"]
    N = O.nsteps(T, dt)
    g = gpu_box(method, "traffic", n, wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], T, dt)
    assert np.isfinite(g[0]).all() and np.isfinite(g[1]).all() and (g[0] <= g[1]).all()
    cells = [0, 1, 5, 4 * N, 12345678, n // 2 + 17, n - 4 * N - 3, n - 2, n - 1]
    cells += _tile_edge_cells(n, TRAFFIC_OWNED)
    for i in sorted(set(cells)):
        a, b = _window(i, n, 4 * N + 2)
        olo, ohi = O.reach(method, "traffic", wl["x_lo"][a:b], wl["x_hi"][a:b], wl["w_lo"], wl["w_hi"],
                           t_final=T, dt=dt)
        assert_close(g[0][i:i + 1], olo[i - a:i - a + 1], TOL64, f"cell {i} lo")
        assert_close(g[1][i:i + 1], ohi[i - a:i - a + 1], TOL64, f"cell {i} hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_ks_full_size_sampled_cells(method):
    n = 1 << 20
    wl = W.ks_grid(n)
    T, dt = wl["t_final"], wl["dt"]
    N = O.nsteps(T, dt)
    g = gpu_box(method, "ks", n, wl["x_lo"], wl["x_hi"], None, None, T, dt)
    assert np.isfinite(g[0]).all() and (g[0] <= g[1]).all()
    L = 16 * N + 8   # periodic window: the wrap travels 8N cells at most in N steps
    for i in sorted(set([0, 7, n // 3, n - 1] + _tile_edge_cells(n, KS_OWNED))):
        idx = (i - L // 2 + np.arange(L)) % n
        olo, ohi = O.reach(method, "ks", wl["x_lo"][idx], wl["x_hi"][idx], t_final=T, dt=dt,
                           params=wl["params"])
        assert_close(g[0][i:i + 1], olo[L // 2:L // 2 + 1], TOL64, f"cell {i} lo")
        assert_close(g[1][i:i + 1], ohi[L // 2:L // 2 + 1], TOL64, f"cell {i} hi")


def test_ks_full_size_mc32_inside_mm():
    n = 1 << 20
    wl = W.ks_grid(n)
    T, dt = wl["t_final"], wl["dt"]
    mm = gpu_box("mm", "ks", n, wl["x_lo"], wl["x_hi"], None, None, T, dt)
    mc = gpu_box("mc", "ks", n, wl["x_lo"], wl["x_hi"], None, None, T, dt, m=1024, seed=0, precision=32)
    assert np.isfinite(mc[0]).all() and (mc[0] <= mc[1]).all()
    # binary32 trajectories: inside the binary64 MM box up to the binary32
    # parity tolerance (the reading of the mc32 containment test below)
    slack = TOL32 * max(np.abs(mm[0]).max(), np.abs(mm[1]).max())
    assert (mc[0] >= mm[0] - slack).all() and (mc[1] <= mm[1] + slack).all()
    assert (mc[1] - mc[0]).min() > 0


@pytest.mark.parametrize("prec,m,owned", [(32, 24, 32 * 12 - 2 * 24), (64, 8, 32 * 16 - 2 * 8)])
def test_ks_full_size_mc_sampled_rows(prec, m, owned):
    # the configured 2^20-point grid over 500 steps in the launch configuration
    # the bench times (binary32: 12 rows per lane, three steps per launch, W =
    # 336 owned rows per warp tile; binary64: 16 rows per lane, one step per
    # launch, W = 496), fewer samples: at sampled rows, the minimum and maximum
    # over the samples equal the oracle's.  Each sample's initial window is
    # drawn from the oracle's generator with the grid's own component indices,
    # and a window of 16N + 8 rows is wide enough that its periodic ends never
    # reach its centre in N steps.
    n = 1 << 20
    wl = W.ks_grid(n)
    T, dt = wl["t_final"], wl["dt"]
    N = O.nsteps(T, dt)
    seed = 21
    g = gpu_box("mc", "ks", n, wl["x_lo"], wl["x_hi"], None, None, T, dt, m=m, seed=seed, precision=prec)
    assert np.isfinite(g[0]).all() and (g[0] <= g[1]).all()
    L = 16 * N + 8
    rows = [0, n - 1] + _tile_edge_cells(n, owned)[::4]
    for i in sorted(set(rows)):
        idx = (i - L // 2 + np.arange(L)) % n
        lo, hi = wl["x_lo"][idx], wl["x_hi"][idx]
        centre = []
        for j in range(m):
            u = np.array([O.uniform(seed, j, int(k), 0) for k in idx])
            x0 = lo + (hi - lo) * u
            if prec == 32:
                x0 = x0.astype(np.float32).astype(np.float64)
            centre.append(O.flow("ks", x0, t_final=T, dt=dt, params=wl["params"])[L // 2])
        tol = TOL64 if prec == 64 else TOL32
        assert_close(g[0][i:i + 1], np.array([min(centre)]), tol, f"row {i} lo")
        assert_close(g[1][i:i + 1], np.array([max(centre)]), tol, f"row {i} hi")


@pytest.mark.parametrize("v", [0.45, 0.25, 0.5])
@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_streaming_traffic_parameters(method, v):
    # v = 0.5 and 0.25 take the exponent-shift path for v x, 0.45 the multiply
    prm = (38.0, v, 0.2, 300.0)
    n = 3001
    lo, hi, wlo, whi, T, dt, _, _ = problem("traffic", n, seed=17)
    R.reach_set_option(R.OPT_KERNEL, 1)
    o = O.reach(method, "traffic", lo, hi, wlo, whi, t_final=0.3, dt=dt, params=prm)
    g = gpu_box(method, "traffic", n, lo, hi, wlo, whi, 0.3, dt, params=prm)
    assert_close(g[0], o[0], TOL64, "lo")
    assert_close(g[1], o[1], TOL64, "hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
def test_ks_rotation_is_tiling_invariant(method):
    # periodic grid: rotating the input by a shift that is not a multiple of the
    # tile must rotate the output (halo and wrap handling across tiles)
    n, k = 5003, 777
    lo, hi, _, _, _, dt, _, _ = problem("ks", n, seed=31)
    R.reach_set_option(R.OPT_KERNEL, 1)
    a = gpu_box(method, "ks", n, lo, hi, None, None, 0.004, dt)
    b = gpu_box(method, "ks", n, np.roll(lo, k), np.roll(hi, k), None, None, 0.004, dt)
    assert_close(b[0], np.roll(a[0], k), TOL64, "lo")
    assert_close(b[1], np.roll(a[1], k), TOL64, "hi")


PIPE = [("traffic", 16, 1.0, 10), ("traffic", 3000, 0.5, 5), ("ks", 300, 0.004, 8), ("osc", 20, 0.5, 25),
        ("linear", 6, 0.5, 10), ("heat", 4096, 0.2, 2), ("heat", 125, 0.2, 5), ("quad", 60, 0.5, 10)]


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("kind,n,T,every", PIPE, ids=[f"{p[0]}{p[1]}" for p in PIPE])
def test_reach_pipe_matches_oracle(method, kind, n, T, every):
    lo, hi, wlo, whi, _, dt, prm, A = problem(kind, n, seed=41)
    opl, oph = O.reach_pipe(method, kind, lo, hi, wlo, whi, t_final=T, dt=dt, every=every, A=A)
    with R.System(kind, n, A=A) as s:
        gpl, gph = R.reach_pipe(s, method, lo, hi, wlo, whi, t_final=T, dt=dt, every=every)
    assert gpl.shape == opl.shape
    for q in range(opl.shape[0]):
        assert_close(gpl[q], opl[q], TOL64, f"row {q} lo")
        assert_close(gph[q], oph[q], TOL64, f"row {q} hi")


@pytest.mark.parametrize("S", [1, 2, 3])
@pytest.mark.parametrize("kind,prec", [("ks", 32), ("traffic", 32), ("ks", 64)])
def test_mc_streaming_steps_per_launch(kind, prec, S):
    n, m = 1500, 40
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=9)
    T = 0.07 if kind == "traffic" else 0.0007   # 7 steps: ragged against S
    R.reach_set_option(R.OPT_KERNEL, 1)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, m=m, seed=2, prec=prec)
    g = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, m=m, seed=2, precision=prec)
    tol = TOL64 if prec == 64 else TOL32
    assert_close(g[0], o[0], tol, "lo")
    assert_close(g[1], o[1], tol, "hi")


BAD = [("traffic", 16, None), ("traffic", 3000, None), ("traffic", 3000, (40.0, 0.5, 1 / 6, 320.0, 1, 0)),
       ("traffic", 3000, (40.0, 0.5, 1 / 6, 320.0, 0, 1)), ("ks", 64, None), ("ks", 3000, None), ("osc", 40, None),
       ("heat", 27, (0.05, 3, 1)), ("heat", 4096, (1e-4, 16, 1)), ("quad", 120, None)]


@pytest.mark.parametrize("kind,n,prm", BAD, ids=[f"{k}{n}{'p' if p else ''}{i}" for i, (k, n, p) in enumerate(BAD)])
def test_every_kernel_rejects_an_inverted_box(kind, n, prm):
    # one component with lo > hi, in host buffers: with at least one step the
    # kernels check the box on the device and the call returns REACH_EINVAL
    g = np.random.default_rng(n)
    c = g.uniform(1, 2, n)
    lo, hi = c - 0.01, c + 0.01
    lo[n // 2], hi[n // 2] = hi[n // 2], lo[n // 2]
    nw = {"traffic": 1, "ks": 0, "osc": n // 2, "heat": 0, "quad": n // 12 * 3}[kind]
    wlo, whi = (np.full(nw, 35.0), np.full(nw, 45.0)) if nw else (None, None)
    with R.System(kind, n, params=prm) as s:
        methods = [R.reach_mm, R.reach_cgb]
        if prm is None or kind != "traffic":
            methods.append(lambda *a, **k: R.reach_mc(*a, **k, m=40, seed=1, precision=64))
        for f in methods:
            with pytest.raises(R.ReachError) as e:
                f(s, lo, hi, wlo, whi, t_final=0.02, dt=0.01)
            assert e.value.code == -1


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("T,S", [(0.01, 1), (0.05, 1), (0.05, 3), (0.07, 2), (0.16, 1), (0.2, 1), (0.4, 2)])
def test_host_buffer_overlap_path(method, T, S):
    # host buffers in and out take the path that overlaps the copies with the
    # first and last launches; it must give the oracle's box and, bit for bit,
    # the box of the same call on device buffers
    import torch
    n = (1 << 20) + 11   # the overlap path starts at 2^20 cells
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    lo, hi, wlo, whi, _, dt, _, _ = problem("traffic", n, seed=77)
    o = O.reach(method, "traffic", lo, hi, wlo, whi, t_final=T, dt=dt)
    g = gpu_box(method, "traffic", n, lo, hi, wlo, whi, T, dt)
    assert_close(g[0], o[0], TOL64, "lo")
    assert_close(g[1], o[1], TOL64, "hi")
    d = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in (lo, hi, wlo, whi)]
    gd = gpu_box(method, "traffic", n, *d, T, dt)
    np.testing.assert_array_equal(g[0], gd[0].cpu().numpy())
    np.testing.assert_array_equal(g[1], gd[1].cpu().numpy())


# ------------------------------------------------------------------ MC samples inside the boxes
# (kind, n, samples, forced kernel: 0 = the library's choice, 1 = streaming)
CONTAIN = [("traffic", 40, 300, 0), ("traffic", 700, 64, 1), ("ks", 64, 256, 0), ("ks", 600, 64, 1),
           ("osc", 8, 300, 0), ("osc", 40, 256, 0), ("linear", 5, 300, 0), ("linear", 12, 256, 0),
           ("heat", 64, 300, 0), ("heat", 125, 200, 0)]


def _containment_problem(kind, n, kernel):
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=21)
    if kind == "heat":
        l = round(n ** (1 / 3))
        prm = (0.05, l, 1)
    if kernel == 1:
        T = 0.13 if kind == "traffic" else 0.003
    return lo, hi, wlo, whi, T, dt, prm, A


def _escapes(inner, outer):
    """Margins of the inner box inside the outer one (negative: an escape)."""
    return np.asarray(inner[0]) - np.asarray(outer[0]), np.asarray(outer[1]) - np.asarray(inner[1])


@pytest.mark.parametrize("kind,n,m,kernel", CONTAIN, ids=[f"{k}{n}m{m}k{s}" for k, n, m, s in CONTAIN])
def test_mc64_samples_inside_mm_and_cgb_exactly(kind, n, m, kernel):
    # Sec. 2.1: MM and CGB over-approximate the reachable set, so every
    # binary64 sample trajectory ends inside both boxes; checked with no slack
    # (an escape is reported with its margin, never absorbed)
    lo, hi, wlo, whi, T, dt, prm, A = _containment_problem(kind, n, kernel)
    R.reach_set_option(R.OPT_KERNEL, kernel)
    mc = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, params=prm, A=A, m=m, seed=5, precision=64)
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, params=prm, A=A, m=m, seed=5, prec=64)
    assert_close(mc[0], o[0], TOL64, "mc lo")
    assert_close(mc[1], o[1], TOL64, "mc hi")
    for method in ("mm", "cgb"):
        box = gpu_box(method, kind, n, lo, hi, wlo, whi, T, dt, params=prm, A=A)
        dlo, dhi = _escapes(mc, box)
        assert dlo.min() >= 0.0, f"{method}: sample below the box by {-dlo.min()!r} at {int(dlo.argmin())}"
        assert dhi.min() >= 0.0, f"{method}: sample above the box by {-dhi.min()!r} at {int(dhi.argmin())}"


@pytest.mark.parametrize("kind,n,m,kernel", CONTAIN[:6], ids=[f"{k}{n}m{m}k{s}" for k, n, m, s in CONTAIN[:6]])
def test_mc32_samples_inside_mm_within_the_binary32_tolerance(kind, n, m, kernel):
    # binary32 trajectories start from the binary32 rounding of each sample
    # (which may lie outside the binary64 box by half a binary32 unit) and
    # carry binary32 rounding error: they are held to the box widened by the
    # binary32 parity tolerance, TOL32 times the box's magnitude
    lo, hi, wlo, whi, T, dt, prm, A = _containment_problem(kind, n, kernel)
    R.reach_set_option(R.OPT_KERNEL, kernel)
    mc = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, params=prm, A=A, m=m, seed=5, precision=32)
    box = gpu_box("mm", kind, n, lo, hi, wlo, whi, T, dt, params=prm, A=A)
    slack = TOL32 * max(np.abs(box[0]).max(), np.abs(box[1]).max())
    dlo, dhi = _escapes(mc, box)
    assert dlo.min() >= -slack and dhi.min() >= -slack, (dlo.min(), dhi.min(), slack)


@pytest.mark.parametrize("kind,n,m,S", [("ks", 1500, 100, 2), ("traffic", 1500, 77, 2), ("ks", 600, 64, 1),
                                        ("traffic", 3001, 130, 3), ("ks", 150, 33, 2), ("traffic", 70, 1, 1),
                                        ("traffic", 1 << 16, 256, 3), ("ks", 1 << 16, 128, 3)])
def test_mc32_two_samples_per_lane_equal_one_bit_for_bit(kind, n, m, S):
    # the packed binary32 kernels (two samples per lane, in blocks of sample
    # rows or along the rows of a sample pair) perform each sample's operations
    # in the same order as the one-sample kernel: same box, bit for bit, for
    # every layout (grids shorter than one warp tile, where a lane's rows wrap
    # around the periodic grid or run past the chain, and a single sample,
    # whose pair has no second sample, included; and grids of 2^16 points,
    # where each persistent warp of the pair-row kernel takes five to ten items
    # from the device counter and, on the traffic chain, copies each next
    # item's rows ahead); and it is the oracle's within TOL32
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=13)
    T = 0.13 if kind == "traffic" else 0.0013
    R.reach_set_option(R.OPT_KERNEL, 1)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    boxes = {}
    try:
        for layout in (1, 0, 3, 4, 5, 6, 8, 9, 10):
            R.reach_set_option(R.OPT_MC_LAYOUT, layout)
            boxes[layout] = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, m=m, seed=4, precision=32)
    finally:
        R.reach_set_option(R.OPT_MC_LAYOUT, 0)
    for layout, b in boxes.items():
        np.testing.assert_array_equal(b[0], boxes[1][0], err_msg=f"layout {layout} lo")
        np.testing.assert_array_equal(b[1], boxes[1][1], err_msg=f"layout {layout} hi")
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, m=m, seed=4, prec=32)
    assert_close(boxes[0][0], o[0], TOL32, "lo")
    assert_close(boxes[0][1], o[1], TOL32, "hi")


@pytest.mark.parametrize("kind,n,m,S", [("ks", 1500, 37, 1), ("traffic", 1501, 40, 1), ("ks", 2999, 9, 2),
                                        ("traffic", 700, 21, 3), ("ks", 150, 3, 1), ("traffic", 70, 1, 2)])
def test_mc64_layouts_equal_bit_for_bit(kind, n, m, S):
    # binary64 streaming MC in sample-row blocks (8- and 16-warp) and along the
    # rows of one sample (8 / 12 / 16 rows per lane): each sample sees the same
    # operations in the same order, so every layout gives the same box bit for
    # bit, and it is the oracle's within TOL64
    lo, hi, wlo, whi, T, dt, prm, A = problem(kind, n, seed=17)
    T = 0.11 if kind == "traffic" else 0.0011
    R.reach_set_option(R.OPT_KERNEL, 1)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
    boxes = {}
    try:
        for layout in (2, 7, 8, 9, 10):
            R.reach_set_option(R.OPT_MC_LAYOUT, layout)
            boxes[layout] = gpu_box("mc", kind, n, lo, hi, wlo, whi, T, dt, m=m, seed=6, precision=64)
    finally:
        R.reach_set_option(R.OPT_MC_LAYOUT, 0)
    for layout, b in boxes.items():
        np.testing.assert_array_equal(b[0], boxes[2][0], err_msg=f"layout {layout} lo")
        np.testing.assert_array_equal(b[1], boxes[2][1], err_msg=f"layout {layout} hi")
    o = O.reach("mc", kind, lo, hi, wlo, whi, t_final=T, dt=dt, m=m, seed=6, prec=64)
    assert_close(boxes[8][0], o[0], TOL64, "lo")
    assert_close(boxes[8][1], o[1], TOL64, "hi")


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("n,T", [(723, 0.003), (3001, 0.0013), (40001, 0.001)])
def test_ks_all_steps_in_one_launch(method, n, T):
    # the persistent KS kernel (every step in one launch, items started as
    # their neighbouring tiles finish the previous step) gives the box of one
    # launch per step bit for bit, and the oracle's
    lo, hi, _, _, _, dt, _, _ = problem("ks", n, seed=61)
    R.reach_set_option(R.OPT_KERNEL, 1)
    boxes = {}
    try:
        for mode in (1, 2):
            R.reach_set_option(R.OPT_ONE_LAUNCH, mode)
            boxes[mode] = gpu_box(method, "ks", n, lo, hi, None, None, T, dt)
    finally:
        R.reach_set_option(R.OPT_ONE_LAUNCH, 0)
    np.testing.assert_array_equal(boxes[1][0], boxes[2][0])
    np.testing.assert_array_equal(boxes[1][1], boxes[2][1])
    o = O.reach(method, "ks", lo, hi, t_final=T, dt=dt)
    assert_close(boxes[2][0], o[0], TOL64, "lo")
    assert_close(boxes[2][1], o[1], TOL64, "hi")


def test_ks_one_launch_reports_a_bad_box_and_a_nonfinite_result():
    n = 3001
    lo, hi, _, _, _, dt, _, _ = problem("ks", n, seed=62)
    R.reach_set_option(R.OPT_ONE_LAUNCH, 2)
    try:
        with R.System("ks", n) as s:
            with pytest.raises(R.ReachError) as e:
                R.reach_mm(s, hi, lo, t_final=0.001, dt=dt)
            assert e.value.code == -1
            big = np.full(n, 10.0)
            with pytest.raises(R.ReachError) as e:
                R.reach_mm(s, -big, big, t_final=2.0, dt=1e-3)
            assert e.value.code == -4
    finally:
        R.reach_set_option(R.OPT_ONE_LAUNCH, 0)


@pytest.mark.parametrize("method", ["mm", "cgb"])
@pytest.mark.parametrize("n,prm", [(5000, None), (30011, None), (30011, (38.0, 0.45, 0.2, 300.0))])
def test_traffic_all_steps_in_one_launch(method, n, prm):
    # the persistent traffic kernel gives the box of one launch per step bit
    # for bit (both v paths: an exponent shift for v = 0.5, a product for
    # 0.45), and the oracle's; device buffers, as the one-launch path takes
    import torch
    lo, hi, wlo, whi, _, dt, _, _ = problem("traffic", n, seed=63)
    T = 0.37
    d = [torch.tensor(v, dtype=torch.float64, device="cuda") for v in (lo, hi, wlo, whi)]
    boxes = {}
    try:
        for mode in (1, 2):
            R.reach_set_option(R.OPT_ONE_LAUNCH, mode)
            g = gpu_box(method, "traffic", n, *d, T, dt, params=prm)
            boxes[mode] = (g[0].cpu().numpy(), g[1].cpu().numpy())
    finally:
        R.reach_set_option(R.OPT_ONE_LAUNCH, 0)
    np.testing.assert_array_equal(boxes[1][0], boxes[2][0])
    np.testing.assert_array_equal(boxes[1][1], boxes[2][1])
    o = O.reach(method, "traffic", lo, hi, wlo, whi, t_final=T, dt=dt, params=prm)
    assert_close(boxes[2][0], o[0], TOL64, "lo")
    assert_close(boxes[2][1], o[1], TOL64, "hi")
