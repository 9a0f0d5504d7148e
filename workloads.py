"""Seeded synthetic inputs for the interval-reachability workloads.

This module only draws initial boxes, input boxes and query mixes from fixed
seeds; it holds none of the reachability arithmetic.  Both the FP64 oracle
(through the tests) and the CUDA library (through the tests and the benchmark)
take their inputs from here, so both sides see bit-identical data.

Workloads (all synthetic; the paper prints no datasets or reachable boxes):

* traffic chain (Sec. 5.1 of the paper, cell transmission model): n=16 with
  x0 in [100,120]^n, and n=2^26 with box centres 80 + 80 U_i, width 10;
  inflow d in [35, 45], dt = 0.01.
* Kuramoto-Sivashinsky periodic grid: spacing pi/4 (so 128 cells span one
  32*pi period of the initial profile), u0(x) = 0.1 cos(x/16)(1 + sin(x/16))
  +- 1e-3, dt = 1e-4, T = 0.05.
* oscillator-chain queries: m log-uniform in [4, 4096], positions U[-1,1],
  velocities 0, half-width 1e-4, disturbance w in [-0.01, 0.01], dt = 0.005,
  T = 5.
* linear test systems (Metzler, general, nilpotent).
* quadrotor swarm (Sec. 5.2): K agents of 12 states, hover thrust, torque
  inputs, dt = 0.01, T = 2 (see quad_swarm).
* 3-D heat diffusion (Sec. 5.4): unit cube on an l^3 grid, cells meeting
  (0.4, 0.6)^3 in [0.9, 1.1], all others in [0, 0.01]; alpha = 8e-6, face
  z = 0 open, dt = 0.02, T = 20.
* a Poisson arrival trace mixing traffic and KS queries for the serving loop.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.Philox(seed))


# ---------------------------------------------------------------- traffic
TRAFFIC_DT = 0.01
TRAFFIC_D = (35.0, 45.0)


def traffic_small(n: int = 16):
    """Traffic chain, n cells, x0 in [100, 120]^n, d in [35, 45], T = 10."""
    return dict(kind="traffic", x_lo=np.full(n, 100.0), x_hi=np.full(n, 120.0),
                w_lo=np.array([TRAFFIC_D[0]]), w_hi=np.array([TRAFFIC_D[1]]),
                t_final=10.0, dt=TRAFFIC_DT)


def traffic_large(n: int = 1 << 26, seed: int = 0, t_final: float = 2.0, half_width: float = 5.0):
    """Traffic chain with box centres 80 + 80 U_i (U uniform from `seed`), width 10."""
    u = _rng(seed).random(n)
    c = 80.0 + 80.0 * u
    return dict(kind="traffic", x_lo=c - half_width, x_hi=c + half_width,
                w_lo=np.array([TRAFFIC_D[0]]), w_hi=np.array([TRAFFIC_D[1]]),
                t_final=t_final, dt=TRAFFIC_DT)


# ---------------------------------------------------------------- KS
KS_DX = math.pi / 4.0
KS_DT = 1e-4


def ks_profile(n: int, dx: float = KS_DX) -> np.ndarray:
    x = np.arange(n, dtype=np.float64) * dx
    return 0.1 * np.cos(x / 16.0) * (1.0 + np.sin(x / 16.0))


def ks_grid(n: int = 1 << 20, half_width: float = 1e-3, t_final: float = 0.05, dx: float = KS_DX):
    u = ks_profile(n, dx)
    return dict(kind="ks", x_lo=u - half_width, x_hi=u + half_width,
                w_lo=np.zeros(0), w_hi=np.zeros(0), t_final=t_final, dt=KS_DT,
                params=(dx, 1.0, 1.0, 1.0))


# ---------------------------------------------------------------- oscillator chain
OSC_DT = 0.005
OSC_T = 5.0
# The box-evaluated growth bound cannot represent the chain's rotation (its
# off-diagonal bounds are nonnegative), grows like exp(sqrt(3) t) and, driven
# by the disturbance box, overflows between t = 4 and t = 5 for every query of
# the batch; the CGB leg of the batched workload therefore stops at t = 4.
OSC_T_CGB = 4.0
OSC_W = 0.01


def osc_query(m: int, seed: int, half_width: float = 1e-4, t_final: float = OSC_T):
    """One oscillator-chain query: state [x_1..x_m | v_1..v_m]."""
    pos = _rng(seed).uniform(-1.0, 1.0, m)
    c = np.concatenate([pos, np.zeros(m)])
    return dict(kind="osc", x_lo=c - half_width, x_hi=c + half_width,
                w_lo=np.full(m, -OSC_W), w_hi=np.full(m, OSC_W),
                t_final=t_final, dt=OSC_DT)


def osc_sizes(count: int = 4096, seed: int = 0, lo: int = 4, hi: int = 4096) -> np.ndarray:
    """m_q log-uniform in [lo, hi], rounded to integers."""
    u = _rng(seed).random(count)
    return np.rint(np.exp(math.log(lo) + u * (math.log(hi) - math.log(lo)))).astype(np.int64)


def osc_batch(count: int = 4096, seed: int = 0, t_final: float = OSC_T):
    sizes = osc_sizes(count, seed)
    return [osc_query(int(m), seed=1000003 * (seed + 1) + q, t_final=t_final)
            for q, m in enumerate(sizes)]


# ---------------------------------------------------------------- linear test systems
def linear_metzler(n: int, seed: int, diag=(-2.0, -0.5), off=(0.0, 0.4)):
    g = _rng(seed)
    A = g.uniform(*off, (n, n))
    A[np.diag_indices(n)] = g.uniform(*diag, n)
    return A


def linear_general(n: int, seed: int, scale: float = 0.6):
    g = _rng(seed)
    A = g.uniform(-scale, scale, (n, n))
    A[np.diag_indices(n)] = g.uniform(-2.0, -0.5, n)
    return A


def linear_nilpotent(n: int, seed: int):
    """Strictly upper-triangular A (A^n = 0)."""
    g = _rng(seed)
    return np.triu(g.uniform(-1.0, 1.0, (n, n)), k=1)


def random_box(n: int, seed: int, centre=(-1.0, 1.0), width=(0.0, 0.2)):
    g = _rng(seed)
    c = g.uniform(*centre, n)
    h = g.uniform(*width, n)
    return c - h, c + h


# ---------------------------------------------------------------- 3-D heat
HEAT_DT = 0.02
HEAT_T = 20.0
HEAT_ALPHA = 8e-6


def heat_hot_cells(l: int) -> np.ndarray:
    """Boolean mask over one axis: cells [k/l, (k+1)/l] meeting (0.4, 0.6)."""
    k = np.arange(l)
    return (5 * k < 3 * l) & (5 * (k + 1) > 2 * l)


def heat_cube(l: int, t_final: float = HEAT_T, dt: float = HEAT_DT, alpha: float = HEAT_ALPHA,
              open_face: bool = True, hot=(0.9, 1.1), cold=(0.0, 0.01)):
    """Unit cube on an l^3 grid, index i = z l^2 + y l + x: cells meeting the
    heated region (0.4, 0.6)^3 start in `hot`, all others in `cold`."""
    a = heat_hot_cells(l)
    mask = (a[:, None, None] & a[None, :, None] & a[None, None, :]).reshape(-1)
    x_lo = np.where(mask, hot[0], cold[0])
    x_hi = np.where(mask, hot[1], cold[1])
    return {"x_lo": x_lo, "x_hi": x_hi, "t_final": t_final, "dt": dt,
            "params": (alpha, l, 1 if open_face else 0)}


def heat_cube_torch(l: int, device, hot=(0.9, 1.1), cold=(0.0, 0.01)):
    """The box of heat_cube built directly in device memory (for l^3 too large
    to stage from the host)."""
    import torch
    a = torch.from_numpy(heat_hot_cells(l)).to(device)
    lo = torch.full((l, l, l), cold[0], dtype=torch.float64, device=device)
    hi = torch.full((l, l, l), cold[1], dtype=torch.float64, device=device)
    idx = torch.nonzero(a).flatten()
    s0, s1 = int(idx[0]), int(idx[-1]) + 1
    lo[s0:s1, s0:s1, s0:s1] = hot[0]
    hi[s0:s1, s0:s1, s0:s1] = hot[1]
    return lo.reshape(-1), hi.reshape(-1)


# ---------------------------------------------------------------- quadrotor swarm
QUAD_DT = 0.01
QUAD_T = 2.0
QUAD_PRM = (1.4, 9.81, 1.4 * 9.81, 0.054, 0.054, 0.104)   # m, g, F (hover), Jx, Jy, Jz
QUAD_HALF = (0.05,) * 3 + (0.01,) * 3 + (0.01,) * 3 + (0.005,) * 3
QUAD_TAU = (0.005, 0.005, 0.002)


def quad_swarm(K: int, seed: int = 0, t_final: float = QUAD_T, dt: float = QUAD_DT):
    """K independent quadrotors, 12 states each (p_n, p_e, h, velocities,
    phi, theta, psi, angular rates): box centres positions U[-10, 10], velocities
    U[-1, 1], roll / pitch U[-0.2, 0.2], yaw U[-pi, pi], rates U[-0.05, 0.05];
    half-widths QUAD_HALF; torques in [-QUAD_TAU, QUAD_TAU]."""
    g = _rng(seed)
    c = np.empty((K, 12))
    c[:, 0:3] = g.uniform(-10.0, 10.0, (K, 3))
    c[:, 3:6] = g.uniform(-1.0, 1.0, (K, 3))
    c[:, 6:8] = g.uniform(-0.2, 0.2, (K, 2))
    c[:, 8] = g.uniform(-math.pi, math.pi, K)
    c[:, 9:12] = g.uniform(-0.05, 0.05, (K, 3))
    h = np.asarray(QUAD_HALF)
    tau = np.tile(np.asarray(QUAD_TAU), K)
    return {"x_lo": (c - h).reshape(-1), "x_hi": (c + h).reshape(-1), "w_lo": -tau, "w_hi": tau.copy(),
            "t_final": t_final, "dt": dt, "params": QUAD_PRM}


# ---------------------------------------------------------------- serving trace
@dataclass
class Query:
    qid: int
    arrival: float
    kind: str
    method: str
    n: int
    steps: int
    x_lo: np.ndarray = field(repr=False)
    x_hi: np.ndarray = field(repr=False)
    w_lo: np.ndarray = field(repr=False)
    w_hi: np.ndarray = field(repr=False)
    dt: float = 0.0
    params: tuple = ()
    m: int = 0
    prec: int = 64
    seed: int = 0


def _logu(g, lo, hi):
    return math.exp(math.log(lo) + g.random() * (math.log(hi) - math.log(lo)))


def serving_trace(count: int = 4000, rate: float = 2000.0, seed: int = 0,
                  traffic_n=(100, 10_000_000), ks_k=(10, 20), steps=(100, 20000),
                  mc_samples: int = 256, scale_steps: float = 1.0, max_n: int | None = None):
    """Poisson arrivals at `rate` queries/s mixing traffic chains and KS grids.

    Box width ~ logU[1e-4, 1e-1] * scale (100 for traffic, 0.1 for KS); method
    uniform over MM / CGB / MC(256 samples, FP32); horizon logU[100, 20000]
    RK4 steps (times `scale_steps`)."""
    g = _rng(seed)
    t = 0.0
    out = []
    for q in range(count):
        t += g.exponential(1.0 / rate)
        kind = "traffic" if g.random() < 0.5 else "ks"
        method = ("mm", "cgb", "mc")[int(g.integers(0, 3))]
        nsteps = max(1, int(round(_logu(g, *steps) * scale_steps)))
        width = _logu(g, 1e-4, 1e-1)
        if kind == "traffic":
            n = int(round(_logu(g, *traffic_n)))
            if max_n:
                n = min(n, max_n)
            c = 80.0 + 80.0 * g.random(n)
            hw = 0.5 * width * 100.0
            x_lo, x_hi = c - hw, c + hw
            w_lo, w_hi = np.array([TRAFFIC_D[0]]), np.array([TRAFFIC_D[1]])
            dt, params = TRAFFIC_DT, ()
        else:
            n = 1 << int(g.integers(ks_k[0], ks_k[1] + 1))
            if max_n:
                n = min(n, max_n)
            u = ks_profile(n)
            hw = 0.5 * width * 0.1
            x_lo, x_hi = u - hw, u + hw
            w_lo = w_hi = np.zeros(0)
            dt, params = KS_DT, (KS_DX, 1.0, 1.0, 1.0)
        out.append(Query(qid=q, arrival=t, kind=kind, method=method, n=n, steps=nsteps,
                         x_lo=x_lo, x_hi=x_hi, w_lo=w_lo, w_hi=w_hi, dt=dt, params=params,
                         m=mc_samples if method == "mc" else 0,
                         prec=32 if method == "mc" else 64, seed=q))
    return out
