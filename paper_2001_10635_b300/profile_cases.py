"""Run one named workload once (after one warm-up call), for profiler captures.

    python -m paper_2001_10635_b300.profile_cases CASE [--n N] [--m M] [--t T]

Cases:
  ks_mm, ks_cgb        KS grid, n points (default 2^20), T (default 0.05)
  ks_mc32, ks_mc64     KS grid, m samples (default 256 / 32)
  traffic_mm           traffic chain, n cells (default 2^24), T (default 0.02)
  traffic16_mm         traffic chain n = 16, T = 10 (on-chip kernel)
  traffic_cgbl         traffic CGB with the box-evaluated C, n cells (default 2^24), T (default 0.02)
  traffic_sound_mm     outward-rounded traffic MM, n cells (default 2^24), T (default 0.02)
  osc_batch            the 4096-query oscillator batch (MM T=5, CGB T=4)
  heat_mm, heat_cgb    heat cube of side l = --n (default 256), --t (default 0.1)
  quad_mm, quad_cgb, quad_mc32   quadrotor swarm of --n agents (default 10^6), --t (default 0.1)
"""
from __future__ import annotations

import argparse
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def main(argv=None):
    import torch

    import paper_2001_10635_b300 as R
    import workloads as W

    ap = argparse.ArgumentParser()
    ap.add_argument("case")
    ap.add_argument("--n", type=int, default=0)
    ap.add_argument("--m", type=int, default=0)
    ap.add_argument("--t", type=float, default=0.0)
    a = ap.parse_args(argv)
    dev = torch.device("cuda", 0)
    to = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)

    if a.case.startswith("ks_"):
        n = a.n or (1 << 20)
        wl = W.ks_grid(n, t_final=a.t or 0.05)
        x0, x1 = to(wl["x_lo"]), to(wl["x_hi"])
        with R.System("ks", n) as s:
            kw = dict(t_final=wl["t_final"], dt=wl["dt"])
            if a.case == "ks_mm":
                f = lambda: R.reach_mm(s, x0, x1, **kw)
            elif a.case == "ks_cgb":
                f = lambda: R.reach_cgb(s, x0, x1, **kw)
            else:
                prec = 32 if a.case == "ks_mc32" else 64
                m = a.m or (256 if prec == 32 else 32)
                f = lambda: R.reach_mc(s, x0, x1, **kw, m=m, seed=0, precision=prec)
            f()
            f()
    elif a.case == "traffic_mm":
        n = a.n or (1 << 24)
        wl = W.traffic_large(n, t_final=a.t or 0.02)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        with R.System("traffic", n) as s:
            for _ in range(2):
                R.reach_mm(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.case in ("traffic_cgbl", "traffic_sound_mm"):
        n = a.n or (1 << 24)
        wl = W.traffic_large(n, t_final=a.t or 0.02)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        prm = (40.0, 0.5, 1 / 6, 320.0, 1, 0) if a.case == "traffic_cgbl" else (40.0, 0.5, 1 / 6, 320.0, 0, 1)
        f = R.reach_cgb if a.case == "traffic_cgbl" else R.reach_mm
        with R.System("traffic", n, params=prm) as s:
            for _ in range(2):
                f(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.case == "traffic16_mm":
        wl = W.traffic_small(16)
        with R.System("traffic", 16) as s:
            for _ in range(2):
                R.reach_mm(s, wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.case in ("heat_mm", "heat_cgb"):
        l = a.n or 256
        lo, hi = W.heat_cube_torch(l, dev)
        with R.System("heat", l ** 3) as s:
            f = R.reach_mm if a.case == "heat_mm" else R.reach_cgb
            for _ in range(2):
                f(s, lo, hi, t_final=a.t or 0.1, dt=W.HEAT_DT)
    elif a.case.startswith("quad_"):
        K = a.n or 1_000_000
        wl = W.quad_swarm(K, seed=0, t_final=a.t or 0.1)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        args = (d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"])
        kw = dict(t_final=wl["t_final"], dt=wl["dt"])
        with R.System("quad", 12 * K) as s:
            for _ in range(2):
                if a.case == "quad_mm":
                    R.reach_mm(s, *args, **kw)
                elif a.case == "quad_cgb":
                    R.reach_cgb(s, *args, **kw)
                else:
                    R.reach_mc(s, *args, **kw, m=a.m or 32, seed=0, precision=32)
    elif a.case == "osc_batch":
        sizes = W.osc_sizes(4096, seed=0)
        systems, qs = {}, []
        for k, m in enumerate(sizes):
            q = W.osc_query(int(m), seed=1000003 + k)
            s = systems.setdefault(int(m), R.System("osc", 2 * int(m)))
            d = {kk: to(q[kk]) for kk in ("x_lo", "x_hi", "w_lo", "w_hi")}
            for method, T in (("mm", W.OSC_T), ("cgb", W.OSC_T_CGB)):
                qs.append(dict(sys=s, method=method, x0_lo=d["x_lo"], x0_hi=d["x_hi"], w_lo=d["w_lo"],
                               w_hi=d["w_hi"], t_final=T, dt=W.OSC_DT))
        with R.Batch(qs) as b:
            b.run()
            b.run()
    else:
        raise SystemExit(f"unknown case {a.case}")
    torch.cuda.synchronize()
    print("done", a.case, R.reach_kernel_launches(), "launches")


if __name__ == "__main__":
    main()
