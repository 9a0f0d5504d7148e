"""Benchmark: RK4 interval reachability on the 2^26-cell traffic chain.

One step = one pass of the hot path over the workload: the mixed-monotonicity
box (Algorithm 3) and the contraction/growth-bound box (Algorithm 2) of the
traffic cell-transmission chain with n = 2^26 cells, x0 box centres
80 + 80 U_i (seed 0) of width 10, inflow d in [35, 45], dt = 0.01, T = 2
(200 RK4 steps each).  Metric: state-component RK4 updates per second
(MM and CGB integrate 2n components each).

  value  inputs resident in HBM (device tensors), CUDA events on the stream
  e2e    the same through the public API with host buffers (page-locked,
         passed as numpy arrays): the library's host->device copies and the
         result readback are inside the timed region
  roofline  the dominant kernel (stencil_traffic_flow<MM>, all 200 steps of a
         call in one launch): FP64-pipe operations per launch / its launch
         time, against the FP64 issue rate of 148 SMs x 2 ops/clk x 2.032 GHz
  cpu_baseline / --impl reference  the FP64 oracle on one host core, on the
         first 2^20 cells of the same workload (full horizon)

Multi-GPU: the path is run as independent replicas, one per rank (weak
scaling); ranks meet only in a barrier and the max-over-ranks timing.
"""
from __future__ import annotations

import argparse
import json
import os
import platform
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import workloads as W  # noqa: E402

N_CELLS = 1 << 26
T_FINAL, DT = 2.0, 0.01
NSTEPS = 200
# FP64 pipe operations per component-step of the fused kernel (add, mul and
# fma each count one).  Per cell and stage the traffic flux costs w (xbar - x')
# (v x with v = 0.5 is an exponent shift on the integer pipe), then the flux
# difference, the stage input and the accumulator: 4 per stage, minus the first
# accumulator and the last stage input, plus the final update = 15.  The CGB
# center costs the same; its radius (linear, constant C) takes RK4 in nested
# form, two fused multiply-adds per stage = 8, so a CGB component-step
# averages (15 + 8) / 2.
FP64_OPS = {"mm": 15.0, "cgb": 11.5}
SM_COUNT, FP64_PER_SM_CLK, SM_MAX_MHZ = 148, 2, 2032.0
FP64_PEAK_OPS = SM_COUNT * FP64_PER_SM_CLK * SM_MAX_MHZ * 1e6
CPU_SAMPLE_CELLS = 1 << 20
# DRAM bytes (read + write) per cell and RK4 step of stencil_traffic_flow<MM>,
# from the ncu capture of one launch on 2^24 cells over 10 steps; the traffic
# is proportional to cells x steps, so it is scaled to the run's n and steps
NCU_DRAM_BYTES_PER_CELL_STEP = (2.825961e9 + 2.646587e9) / ((1 << 24) * 10)


def max_over_ranks(x: float, dist, device) -> float:
    """The largest value of x over all ranks (timings: the job takes as long as
    its slowest replica).  One process per GPU; dist may be None (one rank)."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_rate(units_per_rank: float, world: int, seconds: float) -> float:
    """Whole-job throughput of weak-scaled replicas: all ranks' units over the
    slowest rank's time."""
    return units_per_rank * world / seconds


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:
        return {}


class Clocks:
    """nvidia-smi sampling during the timed region."""

    Q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.rows = []
        self.proc = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            parts = [p.strip() for p in line.split(",")]
            if len(parts) == 7:
                self.rows.append(parts)

    def stop(self):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
        if not self.rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm = [float(r[0]) for r in self.rows if r[0].replace(".", "").isdigit()]
        mx = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[k] for r in self.rows for k in range(4) if r[3 + k].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(self.rows)}


def host_cpu():
    """The host the oracle runs on: logical CPUs (nproc) and the CPU model."""
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.startswith("model name"):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return {"nproc": os.cpu_count(), "cpu_model": model or platform.processor() or "unknown"}


def cpu_oracle_rate(cells: int = CPU_SAMPLE_CELLS):
    """The FP64 oracle (single thread) on the first `cells` cells, both methods."""
    import oracle as O
    wl = W.traffic_large(N_CELLS, seed=0) if cells == N_CELLS else None
    if wl is None:
        full = W.traffic_large(N_CELLS, seed=0)
        wl = dict(full, x_lo=full["x_lo"][:cells].copy(), x_hi=full["x_hi"][:cells].copy())
    t0 = time.perf_counter()
    for method in ("mm", "cgb"):
        O.reach(method, "traffic", wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=T_FINAL, dt=DT)
    sec = time.perf_counter() - t0
    comp_steps = 2 * 2 * cells * NSTEPS
    return comp_steps / sec, sec, comp_steps


def oracle_rates():
    """The oracle (one host core) on bounded samples of the extra sections'
    workloads, in each section's unit; each sample is a few seconds of CPU."""
    import oracle as O
    out = {}

    def timed(label, comps, fn, sample):
        t0 = time.perf_counter()
        fn()
        sec = time.perf_counter() - t0
        out[label] = {"value": comps / sec, "unit": "comp-steps/s", "cores": 1, **host_cpu(), "kind": "oracle",
                      "sample": sample, "s": sec}

    ks = W.ks_grid(1 << 14, t_final=0.005)
    timed("ks_mm", 2 * (1 << 14) * 50,
          lambda: O.reach("mm", "ks", ks["x_lo"], ks["x_hi"], t_final=0.005, dt=1e-4),
          "KS grid n=2^14, MM, 50 steps")
    hc = W.heat_cube(64, t_final=0.2)
    timed("heat3d_mm", 2 * 64 ** 3 * 10,
          lambda: O.reach("mm", "heat", hc["x_lo"], hc["x_hi"], t_final=0.2, dt=W.HEAT_DT),
          "heat cube l=64 (the paper's alpha and region), MM, 10 steps")
    qs = W.quad_swarm(2000, seed=0)
    timed("quad_mm", 2 * 12 * 2000 * 200,
          lambda: O.reach("mm", "quad", qs["x_lo"], qs["x_hi"], qs["w_lo"], qs["w_hi"], t_final=qs["t_final"],
                          dt=qs["dt"]),
          "quadrotor swarm K=2000, MM, 200 steps")
    for label, prm, cells in (("traffic_cgb_local", O.TRAFFIC_LOCAL_PRM, 1 << 16),
                              ("traffic_sound_mm", O.TRAFFIC_SOUND_PRM, 1 << 12)):
        method = "cgb" if "cgb" in label else "mm"
        tr = W.traffic_large(cells, seed=0)
        timed(label, 2 * cells * 200,
              lambda prm=prm, method=method, tr=tr: O.reach(method, "traffic", tr["x_lo"], tr["x_hi"], tr["w_lo"],
                                                            tr["w_hi"], t_final=2.0, dt=0.01, params=prm),
              f"traffic chain n={cells}, {method.upper()}, 200 steps")
    sizes = W.osc_sizes(4096, seed=0)[:64]
    def osc_subset():
        for k, m in enumerate(sizes):
            q = W.osc_query(int(m), seed=1000003 + k, t_final=W.OSC_T)
            O.reach("mm", "osc", q["x_lo"], q["x_hi"], q["w_lo"], q["w_hi"], t_final=W.OSC_T, dt=W.OSC_DT)
    timed("batched_mm", sum(2 * 2 * int(m) * 1000 for m in sizes), osc_subset,
          "the first 64 queries of the oscillator batch, MM, 1000 steps")
    return out


def _pct(v, q):
    return float(np.percentile(np.asarray(v), q)) if len(v) else None


def bench_batched(R, torch, dev, runs=3, solo_stride=1):
    """4096 oscillator-chain queries x (MM to T=5, CGB to T=4), one graph launch of
    the batched persistent kernels, against the same queries launched one by one
    (all of them by default; every `solo_stride`-th one otherwise).  CGB runs to
    T=4: its box-supremum growth bound overflows between t=4 and t=5 for every
    query (oracle and GPU agree)."""
    sizes = W.osc_sizes(4096, seed=0)
    systems, qs = {}, []
    for k, m in enumerate(sizes):
        q = W.osc_query(int(m), seed=1000003 + k, t_final=W.OSC_T)
        s = systems.setdefault(int(m), R.System("osc", 2 * int(m)))
        d = {kk: torch.tensor(q[kk], dtype=torch.float64, device=dev) for kk in ("x_lo", "x_hi", "w_lo", "w_hi")}
        for method, T in (("mm", W.OSC_T), ("cgb", W.OSC_T_CGB)):
            qs.append(dict(sys=s, method=method, x0_lo=d["x_lo"], x0_hi=d["x_hi"], w_lo=d["w_lo"],
                           w_hi=d["w_hi"], t_final=T, dt=W.OSC_DT))
    comp = [2 * q["sys"].n * int(round(q["t_final"] / q["dt"])) for q in qs]
    t0 = time.perf_counter()
    b = R.Batch(qs)
    create_s = time.perf_counter() - t0
    b.run()   # warm
    times, fin = [], None
    launches0 = R.reach_kernel_launches()
    for _ in range(runs):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        st, fin = b.run()
        times.append(time.perf_counter() - t0)
    batch_launches = (R.reach_kernel_launches() - launches0) / runs
    tb = statistics.median(times)
    sub = list(range(0, len(qs), solo_stride))
    lat = []
    launches0 = R.reach_kernel_launches()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for i in sub:
        q = qs[i]
        fn = R.reach_mm if q["method"] == "mm" else R.reach_cgb
        t1 = time.perf_counter()
        fn(q["sys"], q["x0_lo"], q["x0_hi"], q["w_lo"], q["w_hi"], t_final=q["t_final"], dt=q["dt"])
        lat.append(time.perf_counter() - t1)
    ts = time.perf_counter() - t0
    solo_launches = R.reach_kernel_launches() - launches0
    solo_rate = sum(comp[i] for i in sub) / ts
    info = b.info()
    layout = b.layout()
    b.close()
    for s in systems.values():
        s.close()
    return {"workload": "4096 oscillator-chain queries, m log-uniform in [4, 4096] (seed 0), MM T=5 + CGB T=4, "
                        "dt=0.005, box half-width 1e-4, w in [-0.01, 0.01]",
            "cgb_horizon_note": "CGB runs to T=4: the box-supremum growth bound of the chain overflows between "
                                "t=4 and t=5 for every query (oracle and GPU agree)",
            "queries": len(qs), "comp_steps": int(sum(comp)),
            "value": sum(comp) / tb, "unit": "comp-steps/s", "run_s": tb, "create_s": create_s,
            "create_s_in_library": layout["create_s"],
            "value_with_create": sum(comp) / (tb + create_s),
            "create_note": "create = planning + layout tuning on 24-step horizons + graph capture, once per batch",
            "latency_p50_ms": _pct(fin, 50) * 1e3, "latency_p99_ms": _pct(fin, 99) * 1e3,
            "latency_note": "completion time of each query from the start of the batch (all submitted at once)",
            "tuned": {"cpt": layout["cpt"], "cluster_from": layout["cluster_from"]},
            "tune_ms": layout["tune_ms"], "kernels_per_run": info["kernels"],
            "gpu_launches_per_run": batch_launches,
            "solo": {"queries": len(sub), "sample": "every query" if solo_stride == 1 else f"every {solo_stride}th query",
                     "s": ts, "value": solo_rate,
                     "service_p50_ms": _pct(lat, 50) * 1e3, "service_p99_ms": _pct(lat, 99) * 1e3,
                     "gpu_launches": solo_launches},
            "speedup_vs_solo": (sum(comp) / tb) / solo_rate,
            "speedup_vs_solo_with_create": (sum(comp) / (tb + create_s)) / solo_rate}


def bench_ks(R, torch, dev):
    """Kuramoto-Sivashinsky grid n = 2^20 (dt 1e-4, T 0.05): MM, CGB, and MC
    with 1024 samples in FP32 and in FP64, the configured workload in full."""
    n = 1 << 20
    wl = W.ks_grid(n)
    d = {k: torch.tensor(wl[k], dtype=torch.float64, device=dev) for k in ("x_lo", "x_hi")}
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    N = int(round(wl["t_final"] / wl["dt"]))
    out = {"workload": "KS periodic grid n=2^20, dx=pi/4, dt=1e-4, T=0.05 (500 RK4 steps), u0 +- 1e-3"}
    with R.System("ks", n) as s:
        for name, fn, kw, comps in (("mm", R.reach_mm, {}, 2 * n), ("cgb", R.reach_cgb, {}, 2 * n),
                                    ("mc32_m1024", R.reach_mc, dict(m=1024, precision=32), 1024 * n),
                                    ("mc64_m1024", R.reach_mc, dict(m=1024, precision=64), 1024 * n)):
            # warm: two steps load the kernels and grow the memory pool
            fn(s, d["x_lo"], d["x_hi"], t_final=2 * wl["dt"], dt=wl["dt"], lo=lo, hi=hi, **kw)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            fn(s, d["x_lo"], d["x_hi"], t_final=wl["t_final"], dt=wl["dt"], lo=lo, hi=hi, **kw)
            sec = time.perf_counter() - t0
            out[name] = {"s": sec, "value": comps * N / sec, "unit": "comp-steps/s"}
            if name in KS_FP64_OPS:
                out[name]["fp64_frac"] = KS_FP64_OPS[name] * comps * N / sec / FP64_PEAK_OPS
            if name == "mc32_m1024":
                # binary32: FP32 FMA-pipe fraction, and HBM at the default
                # three steps per launch (8 B per sample-component-step / S)
                S = R.reach_get_option(R.OPT_STEPS_PER_LAUNCH) or 3
                out[name]["fp32_frac"] = KS_FP32_OPS * comps * N / sec / FP32_PEAK_OPS
                out[name]["steps_per_launch"] = S
                out[name]["hbm_frac_at_S"] = 8.0 / S * comps * N / sec / (load_peaks().get("hbm_gbs", 6400.0) * 1e9)
    out["fp64_ops_per_comp_step"] = KS_FP64_OPS
    out["fp32_ops_per_comp_step"] = KS_FP32_OPS
    return out


# FP64 pipe operations per component-step of the KS stencil kernels: per stage
# and component MM takes 7 (two pair sums, one difference shared by two, four
# fused operations per half) plus the stage input and accumulator, CGB 9
# (center 4, radius 5) plus those two; over four stages, minus the first
# accumulator and the last stage input, plus the final update
KS_FP64_OPS = {"mm": 35.0, "cgb": 43.0, "mc64_m1024": 35.0}
# FP32 operations per sample-component-step of the binary32 KS sample
# trajectory (the same 35-operation RK4 step, each a lane of a packed
# instruction), and the FP32 FMA pipe's rate: 128 lanes per SM per clock
KS_FP32_OPS = 35.0
FP32_PEAK_OPS = 148 * 128 * 2032e6


# FP64 pipe operations per component-step of the heat stage kernels (RK4 in
# nested form for the linear system): per stage five neighbour additions, the
# fma with the neighbour count and the stage fma = 7, four stages = 28
HEAT_FP64_OPS = 28.0


def bench_heat(R, torch, dev, l=1000, steps=10):
    """3-D heat diffusion on the paper's l = 1000 cube (10^9 cells, Sec. 5.4),
    MM and CGB over `steps` RK4 steps, timed with CUDA events; the rate gives
    the time of the paper's 1000-step run."""
    n = l ** 3
    need = 10 * 8 * n + (2 << 30)
    if torch.cuda.mem_get_info(dev)[0] < need:
        return {"skipped": f"needs {need / 2**30:.0f} GiB of device memory"}
    dt = W.HEAT_DT
    T = steps * dt
    xlo, xhi = W.heat_cube_torch(l, dev)
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    stream = torch.cuda.current_stream(dev)
    out = {"workload": f"heat cube l={l} (n=1e9), alpha=8e-6, open face z=0, (0.4,0.6)^3 in [0.9,1.1], "
                       f"else [0,0.01], dt=0.02, {steps} RK4 steps per call",
           "unit": "comp-steps/s"}
    with R.System("heat", n) as s:
        for name, fn in (("mm", R.reach_mm), ("cgb", R.reach_cgb)):
            fn(s, xlo, xhi, t_final=T, dt=dt, lo=lo, hi=hi, stream=stream)   # warm
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(s, xlo, xhi, t_final=T, dt=dt, lo=lo, hi=hi, stream=stream)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            rate = 2 * n * steps / sec
            ops = HEAT_FP64_OPS * 2 * n * steps / sec
            out[name] = {"s": sec, "value": rate, "ms_per_rk4_step": sec / steps * 1e3,
                         "fp64_frac": ops / FP64_PEAK_OPS,
                         "minutes_for_1000_steps": sec / steps * 1000 / 60}
    out["paper_minutes_for_1000_steps"] = 350.2
    out["fp64_ops_per_comp_step"] = HEAT_FP64_OPS
    del xlo, xhi, lo, hi
    torch.cuda.empty_cache()
    return out


def bench_quad(R, torch, dev, K=10_000_000):
    """Quadrotor swarm (Sec. 5.2) at the largest size the paper reports on a
    GPU: n = 1.2e8 states (10^7 agents), hover thrust, torque inputs, dt = 0.01,
    T = 2 (200 RK4 steps); MM, CGB and MC with 32 FP32 samples."""
    n = 12 * K
    wl = W.quad_swarm(K, seed=0)
    d = {k: torch.from_numpy(wl[k]).to(dev) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    stream = torch.cuda.current_stream(dev)
    N = int(round(wl["t_final"] / wl["dt"]))
    out = {"workload": f"quadrotor swarm K={K} (n={n}), hover thrust, torques +-(5e-3, 5e-3, 2e-3), "
                       f"dt=0.01, T=2 ({N} RK4 steps), one launch per call",
           "unit": "comp-steps/s"}
    args = (d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"])
    with R.System("quad", n) as s:
        for name, fn, kw, comps in (("mm", R.reach_mm, {}, 2 * n), ("cgb", R.reach_cgb, {}, 2 * n),
                                    ("mc32_m32", R.reach_mc, dict(m=32, seed=0, precision=32), 32 * n)):
            fn(s, *args, t_final=wl["t_final"], dt=wl["dt"], lo=lo, hi=hi, stream=stream, **kw)   # warm
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(s, *args, t_final=wl["t_final"], dt=wl["dt"], lo=lo, hi=hi, stream=stream, **kw)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            out[name] = {"s": sec, "value": comps * N / sec}
    out["paper_gpu_seconds_for_this_n"] = 46.0
    out["paper_note"] = "p3.2xlarge (V100), CGB, n = 1.2e8; the paper does not state its horizon"
    del d, lo, hi
    torch.cuda.empty_cache()
    return out


def bench_traffic_local(R, torch, dev, d, n):
    """Traffic CGB with the contraction matrix taken over the current box
    (reading R14) on the headline workload: time and the summed width of the
    final box against the global bound's."""
    stream = torch.cuda.current_stream(dev)
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    out = {"workload": f"traffic chain n={n}, CGB with box-evaluated C, dt=0.01, T=2 (200 RK4 steps)",
           "unit": "comp-steps/s"}
    widths = {}
    for name, prm in (("local", (40.0, 0.5, 1.0 / 6.0, 320.0, 1)), ("global", None)):
        with R.System("traffic", n, params=prm) as s:
            args = (d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"])
            R.reach_cgb(s, *args, t_final=T_FINAL, dt=DT, lo=lo, hi=hi, stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            R.reach_cgb(s, *args, t_final=T_FINAL, dt=DT, lo=lo, hi=hi, stream=stream)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            widths[name] = float((hi - lo).sum())
            if name == "local":
                out["value"] = 2 * n * NSTEPS / sec
                out["s"] = sec
    out["width_sum_local_over_global"] = widths["local"] / widths["global"]
    return out


def bench_traffic_sound(R, torch, dev, d, n):
    """Outward-rounded traffic MM and CGB (reading R15) on the headline
    workload: time, and how far the outward box reaches beyond the
    round-to-nearest one."""
    stream = torch.cuda.current_stream(dev)
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    rlo = torch.empty_like(lo)
    rhi = torch.empty_like(lo)
    args = (d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"])
    out = {"workload": f"traffic chain n={n}, outward-rounded MM and CGB, dt=0.01, T=2 (200 RK4 steps)",
           "unit": "comp-steps/s"}
    with R.System("traffic", n, params=(40.0, 0.5, 1.0 / 6.0, 320.0, 0, 1)) as s, R.System("traffic", n) as sr:
        for name, fn in (("mm", R.reach_mm), ("cgb", R.reach_cgb)):
            fn(s, *args, t_final=T_FINAL, dt=DT, lo=lo, hi=hi, stream=stream)
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(s, *args, t_final=T_FINAL, dt=DT, lo=lo, hi=hi, stream=stream)
            e1.record(stream)
            e1.synchronize()
            sec = e0.elapsed_time(e1) * 1e-3
            fn(sr, *args, t_final=T_FINAL, dt=DT, lo=rlo, hi=rhi, stream=stream)
            torch.cuda.synchronize()
            scale = float(rhi.abs().max())
            out[name] = {"s": sec, "value": 2 * n * NSTEPS / sec,
                         "max_outward_excess_rel": max(float((rlo - lo).max()), float((hi - rhi).max())) / scale,
                         "contains_nearest": bool((lo <= rlo).all() and (hi >= rhi).all())}
    return out


def bench_temporal_blocking(R, torch, dev):
    """RK4 steps per launch S (halo 4 R S recomputed) on traffic MM (FP64,
    n = 2^24) and on KS MC32 (n = 2^20, 256 samples): the FP64 kernels are bound
    by the FP64 pipe, so recomputation costs more than the HBM traffic it saves."""
    out = {}
    n = 1 << 24
    wl = W.traffic_large(n, seed=0, t_final=0.24)
    d = {k: torch.tensor(wl[k], dtype=torch.float64, device=dev) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    ks = W.ks_grid(1 << 20, t_final=0.012)
    kd = {k: torch.tensor(ks[k], dtype=torch.float64, device=dev) for k in ("x_lo", "x_hi")}
    with R.System("traffic", n) as s, R.System("ks", 1 << 20) as sk:
        for S in (1, 2, 4):
            R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, S)
            R.reach_mm(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=0.24, dt=0.01)
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            R.reach_mm(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=0.24, dt=0.01)
            sec = time.perf_counter() - t0
            out[f"traffic_mm_S{S}"] = 2 * n * 24 / sec
            if S <= 2:
                kw = dict(t_final=0.012, dt=1e-4, m=256, seed=0, precision=32)
                R.reach_mc(sk, kd["x_lo"], kd["x_hi"], **kw)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                R.reach_mc(sk, kd["x_lo"], kd["x_hi"], **kw)
                sec = time.perf_counter() - t0
                out[f"ks_mc32_S{S}"] = 256 * (1 << 20) * 120 / sec
                # algorithmic HBM bytes: one binary32 read and write per sample-component and launch
                gbs = out[f"ks_mc32_S{S}"] * 8.0 / S / 1e9
                out[f"ks_mc32_S{S}_hbm_gbs"] = gbs
                out[f"ks_mc32_S{S}_hbm_frac"] = gbs / load_peaks().get("hbm_gbs", 6400.0)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 0)
    out["unit"] = "comp-steps/s"
    return out


def bench_traffic16(R):
    """Traffic chain n = 16, T = 10 (1000 steps): latency of one call."""
    wl = W.traffic_small(16)
    args = (wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"])
    out = {"workload": "traffic chain n=16, x0 in [100,120]^16, d in [35,45], dt=0.01, T=10"}
    with R.System("traffic", 16) as s:
        for name, fn, kw in (("mm", R.reach_mm, {}), ("cgb", R.reach_cgb, {}),
                             ("mc64_m1000", R.reach_mc, dict(m=1000, precision=64)),
                             ("mc32_m1000", R.reach_mc, dict(m=1000, precision=32))):
            fn(s, *args, t_final=wl["t_final"], dt=wl["dt"], **kw)
            t0 = time.perf_counter()
            reps = 5
            for _ in range(reps):
                fn(s, *args, t_final=wl["t_final"], dt=wl["dt"], **kw)
            out[name + "_ms"] = (time.perf_counter() - t0) / reps * 1e3
    return out


def _comp_steps(q):
    n = q.n
    return (q.m * n if q.method == "mc" else 2 * n) * q.steps


def _failed(bad):
    """Failed queries by status name (both arms fail the same ones: KS boxes
    that overflow over the longest horizons give REACH_ENONFINITE)."""
    import paper_2001_10635_b300 as R
    return {R.strerror(k): v for k, v in sorted(bad.items())}


def _serve_run(R, trace, systems, rate_scale, slots, budget):
    """Arrivals at trace times / rate_scale through the server; returns latencies."""
    import threading as th
    srv = R.Server(slots=slots, hbm_budget_bytes=budget)
    tickets = [None] * len(trace)
    t0 = time.perf_counter()

    def feed():
        for i, q in enumerate(trace):
            at = (q.arrival - trace[0].arrival) / rate_scale
            delay = at - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
            tickets[i] = (time.perf_counter(), srv.submit(systems[(q.kind, q.n)], q.method, q.x_lo, q.x_hi, *w,
                                                          t_final=q.steps * q.dt, dt=q.dt, m=q.m, seed=q.seed,
                                                          precision=q.prec))

    feeder = th.Thread(target=feed)
    feeder.start()
    lat, bad = [], {}
    last = t0
    for i in range(len(trace)):
        while tickets[i] is None:
            time.sleep(0.0005)
        sub_t, (tk, _) = tickets[i]
        st, qs, rs = srv.wait(tk, timeout_s=600)
        done_t = sub_t + qs + rs
        if st != 0:
            bad[st] = bad.get(st, 0) + 1
        lat.append(done_t - sub_t)
        last = max(last, done_t)
    feeder.join()
    peak = srv.stats()["bytes_peak"]
    queued = srv.queued()
    srv.close()
    return lat, last - t0, bad, peak, queued


def _fifo_run(R, trace, systems, rate_scale):
    """Plain per-query launches: one at a time in arrival order on one stream."""
    lat, bad = [], {}
    t0 = time.perf_counter()
    for q in trace:
        at = (q.arrival - trace[0].arrival) / rate_scale
        now = time.perf_counter() - t0
        if at > now:
            time.sleep(at - now)
        s = systems[(q.kind, q.n)]
        kw = dict(t_final=q.steps * q.dt, dt=q.dt)
        w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
        try:
            if q.method == "mm":
                R.reach_mm(s, q.x_lo, q.x_hi, *w, **kw)
            elif q.method == "cgb":
                R.reach_cgb(s, q.x_lo, q.x_hi, *w, **kw)
            else:
                R.reach_mc(s, q.x_lo, q.x_hi, *w, **kw, m=q.m, seed=q.seed, precision=q.prec)
        except R.ReachError as e:
            bad[e.code] = bad.get(e.code, 0) + 1
        lat.append(time.perf_counter() - t0 - at)
    return lat, time.perf_counter() - t0, bad


def bench_serving(R, count=60, sweep_count=30, slots=8, budget=160 << 30, loads=(0.5, 0.7, 0.9)):
    """The seeded 2000 q/s Poisson trace at its stated sizes (traffic n in
    [1e2, 1e7], KS n = 2^10..2^20, MM / CGB / MC-256-FP32, 100..20000 RK4
    steps): its first `count` arrivals at the offered rate, and its first
    `sweep_count` at 50 / 70 / 90% of the measured serving capacity, served
    and as plain per-query launches in arrival order (FIFO)."""
    # the trace is drawn sequentially, so its first `count` arrivals are those of the full trace
    trace = W.serving_trace(count=count, rate=2000.0, seed=0)
    systems = {}
    for q in trace:
        if (q.kind, q.n) not in systems:
            systems[(q.kind, q.n)] = R.System(q.kind, q.n)
    work = sum(_comp_steps(q) for q in trace)
    # warm every kernel kind once
    for q in trace[:12]:
        w = (q.w_lo, q.w_hi) if q.kind == "traffic" else (None, None)
        kw = dict(t_final=q.dt * 2, dt=q.dt)
        s = systems[(q.kind, q.n)]
        (R.reach_mm if q.method == "mm" else R.reach_cgb)(s, q.x_lo, q.x_hi, *w, **kw)
    lat, span, bad, peak, queued = _serve_run(R, trace, systems, 1.0, slots, budget)
    flat, fspan, fbad = _fifo_run(R, trace, systems, 1.0)
    capacity = len(trace) / span
    # latency against offered load: the first sweep_count arrivals at 50%, 70%
    # and 90% of the measured serving capacity, through the server and one at
    # a time (where a small query waits behind every large one ahead of it)
    sus = trace[:sweep_count]
    sweep = []
    for frac in loads:
        scale = frac * capacity / 2000.0
        slat, sspan, sbad, _, _ = _serve_run(R, sus, systems, scale, slots, budget)
        sflat, sfspan, sfbad = _fifo_run(R, sus, systems, scale)
        sweep.append({"load": frac, "rate_qps": 2000.0 * scale, "queries": len(sus),
                      "p50_ms": _pct(slat, 50) * 1e3, "p99_ms": _pct(slat, 99) * 1e3, "failed": _failed(sbad),
                      "makespan_s": sspan,
                      "fifo_p50_ms": _pct(sflat, 50) * 1e3, "fifo_p99_ms": _pct(sflat, 99) * 1e3,
                      "fifo_makespan_s": sfspan, "fifo_failed": _failed(sfbad)})
    for s in systems.values():
        s.close()
    return {"workload": f"seeded Poisson trace, 2000 q/s offered, at its stated sizes: traffic n logU[1e2, 1e7], "
                        f"KS n = 2^10..2^20, box widths logU[1e-4, 1e-1] x scale, MM / CGB / MC-256-FP32, "
                        f"horizons logU[100, 20000] RK4 steps; the first {count} of its 4000 arrivals at the "
                        f"offered rate, the first {sweep_count} in the load sweep",
            "queries": len(trace), "comp_steps": int(work), "slots": slots, "hbm_budget_bytes": budget,
            "queue_blocks": R.reach_get_option(R.OPT_SERVE_QUEUE_BLOCKS),
            "queue_n": R.reach_get_option(R.OPT_SERVE_QUEUE_N),
            "max_wide": R.reach_get_option(R.OPT_SERVE_MAX_WIDE),
            "peak_admitted_bytes": peak,
            "served": {"value": work / span, "unit": "comp-steps/s", "makespan_s": span,
                       "queries_per_s": len(trace) / span, "p50_ms": _pct(lat, 50) * 1e3,
                       "p99_ms": _pct(lat, 99) * 1e3, "failed": _failed(bad), "on_device_queue": queued},
            "per_query_fifo": {"value": work / fspan, "unit": "comp-steps/s", "makespan_s": fspan,
                               "p50_ms": _pct(flat, 50) * 1e3, "p99_ms": _pct(flat, 99) * 1e3, "failed": _failed(fbad)},
            "speedup_vs_fifo": fspan / span,
            "sustainable": sweep[len(sweep) // 2] if sweep else None, "load_sweep": sweep}


def headline_config(n, world):
    return {"workload": f"traffic chain n={n}, MM + CGB, dt=0.01, T=2 (200 RK4 steps each)",
            "n": n, "rk4_steps": NSTEPS, "methods": ["mm", "cgb"],
            "l2": "inputs larger than L2 (2 x 512 MiB state per call)",
            "parallelism": f"replicas x{world}"}


def run_reference(args):
    """--impl reference: the oracle as it stands, timed on the host cores on a
    bounded sample of the same workload (rank 0 only)."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus)))
    if rank != 0:
        return 0
    for _ in range(max(args.warmup, 0)):
        cpu_oracle_rate()
    rates = []
    for _ in range(args.steps):
        r, sec, cs = cpu_oracle_rate()
        rates.append(r)
    value = statistics.median(rates)
    sample = f"first {CPU_SAMPLE_CELLS} cells of the 2^26-cell chain, MM + CGB, 200 RK4 steps, per step"
    line = {"metric": "state-component RK4 updates/s", "value": value, "unit": "comp-steps/s",
            "impl": "reference", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "higher_is_better": True, "dtype": "f64", "data": "synthetic",
            "config": headline_config(N_CELLS, world),
            "cpu_baseline": {"value": value, "unit": "comp-steps/s", "cores": 1, **host_cpu(), "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": "comp-steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "vs_baseline": None}
    print(json.dumps(line))
    return 0


def run_profile_case(a):
    """--profile-case CASE: run one named workload twice (a warm-up call, then
    the call a profiler captures) and exit; no timing, no JSON line.

    Cases (sizes from --case-n / --case-m / --case-t, else the defaults):
      ks_mm, ks_cgb        KS grid, n points (default 2^20), T (default 0.05)
      ks_mc32, ks_mc64     KS grid, m samples (default 256 / 32)
      traffic_mm           traffic chain, n cells (default 2^24), T (default 0.02)
      traffic_mc32         traffic chain, n cells (default 2^20), m samples (default 256), T (default 0.09)
      traffic16_mm         traffic chain n = 16, T = 10 (on-chip kernel)
      traffic_cgbl         traffic CGB with the box-evaluated C, n cells (default 2^24), T (default 0.02)
      traffic_sound_mm     outward-rounded traffic MM, n cells (default 2^24), T (default 0.02)
      osc_batch            the 4096-query oscillator batch (MM T=5, CGB T=4)
      heat_mm, heat_cgb    heat cube of side l = n (default 256), T (default 0.1)
      quad_mm, quad_cgb, quad_mc32   quadrotor swarm of n agents (default 10^6), T (default 0.1)
    """
    import torch

    import paper_2001_10635_b300 as R

    dev = torch.device("cuda", 0)
    to = lambda v: torch.tensor(v, dtype=torch.float64, device=dev)
    for kv in a.case_opt:
        key, val = kv.split("=")
        R.reach_set_option(int(key), int(val))

    if a.profile_case.startswith("ks_"):
        n = a.case_n or (1 << 20)
        wl = W.ks_grid(n, t_final=a.case_t or 0.05)
        x0, x1 = to(wl["x_lo"]), to(wl["x_hi"])
        with R.System("ks", n) as s:
            kw = dict(t_final=wl["t_final"], dt=wl["dt"])
            if a.profile_case == "ks_mm":
                f = lambda: R.reach_mm(s, x0, x1, **kw)
            elif a.profile_case == "ks_cgb":
                f = lambda: R.reach_cgb(s, x0, x1, **kw)
            else:
                prec = 32 if a.profile_case == "ks_mc32" else 64
                m = a.case_m or (256 if prec == 32 else 32)
                f = lambda: R.reach_mc(s, x0, x1, **kw, m=m, seed=0, precision=prec)
            f()
            f()
    elif a.profile_case == "traffic_mc32":
        n = a.case_n or (1 << 20)
        wl = W.traffic_large(n, t_final=a.case_t or 0.09)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        with R.System("traffic", n) as s:
            for _ in range(2):
                R.reach_mc(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"],
                           m=a.case_m or 256, seed=0, precision=32)
    elif a.profile_case == "traffic_mm":
        n = a.case_n or (1 << 24)
        wl = W.traffic_large(n, t_final=a.case_t or 0.02)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        with R.System("traffic", n) as s:
            for _ in range(2):
                R.reach_mm(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.profile_case in ("traffic_cgbl", "traffic_sound_mm"):
        n = a.case_n or (1 << 24)
        wl = W.traffic_large(n, t_final=a.case_t or 0.02)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        prm = (40.0, 0.5, 1 / 6, 320.0, 1, 0) if a.profile_case == "traffic_cgbl" else (40.0, 0.5, 1 / 6, 320.0, 0, 1)
        f = R.reach_cgb if a.profile_case == "traffic_cgbl" else R.reach_mm
        with R.System("traffic", n, params=prm) as s:
            for _ in range(2):
                f(s, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.profile_case == "traffic16_mm":
        wl = W.traffic_small(16)
        with R.System("traffic", 16) as s:
            for _ in range(2):
                R.reach_mm(s, wl["x_lo"], wl["x_hi"], wl["w_lo"], wl["w_hi"], t_final=wl["t_final"], dt=wl["dt"])
    elif a.profile_case in ("heat_mm", "heat_cgb"):
        l = a.case_n or 256
        lo, hi = W.heat_cube_torch(l, dev)
        with R.System("heat", l ** 3) as s:
            f = R.reach_mm if a.profile_case == "heat_mm" else R.reach_cgb
            for _ in range(2):
                f(s, lo, hi, t_final=a.case_t or 0.1, dt=W.HEAT_DT)
    elif a.profile_case.startswith("quad_"):
        K = a.case_n or 1_000_000
        wl = W.quad_swarm(K, seed=0, t_final=a.case_t or 0.1)
        d = {k: to(wl[k]) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
        args = (d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"])
        kw = dict(t_final=wl["t_final"], dt=wl["dt"])
        with R.System("quad", 12 * K) as s:
            for _ in range(2):
                if a.profile_case == "quad_mm":
                    R.reach_mm(s, *args, **kw)
                elif a.profile_case == "quad_cgb":
                    R.reach_cgb(s, *args, **kw)
                else:
                    R.reach_mc(s, *args, **kw, m=a.case_m or 32, seed=0, precision=32)
    elif a.profile_case == "osc_batch":
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
        raise SystemExit(f"unknown case {a.profile_case}")
    torch.cuda.synchronize()
    print("done", a.profile_case, R.reach_kernel_launches(), "launches")
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--no-e2e", action="store_true", help="skip the end-to-end host-buffer leg")
    ap.add_argument("--no-extra", action="store_true", help="skip the batched, KS and small-config sections")
    ap.add_argument("--cells", type=int, default=N_CELLS,
                    help="chain length (default 2^26; smaller values are for profiler captures only)")
    ap.add_argument("--profile-case", default="", help="run one named workload for a profiler capture and exit")
    ap.add_argument("--serving-run", default="",
                    help="COUNT:SWEEP:LOADS, e.g. 400:100:0.9: only the serving comparison, with COUNT arrivals at the "
                         "offered rate and SWEEP at each comma-free list of loads (0.5/0.7/0.9), printed as JSON")
    ap.add_argument("--case-n", type=int, default=0)
    ap.add_argument("--case-m", type=int, default=0)
    ap.add_argument("--case-t", type=float, default=0.0)
    ap.add_argument("--case-opt", action="append", default=[],
                    help="KEY=VALUE: a library option (reach_set_option) for the profile case, e.g. 12=1 for one "
                         "launch per RK4 step")
    args = ap.parse_args()
    if args.profile_case:
        return run_profile_case(args)
    if args.serving_run:
        import paper_2001_10635_b300 as R
        cnt, sweep, loads = args.serving_run.split(":")
        res = bench_serving(R, count=int(cnt), sweep_count=int(sweep),
                            loads=tuple(float(v) for v in loads.split("/")))
        print(json.dumps({"serving": res}))
        return 0
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_2001_10635_b300 as R

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.cells
    wl = W.traffic_large(n, seed=0)
    dev = torch.device("cuda", local)
    def pinned(a):
        # page-locked host buffer seen by the library as a plain host pointer
        t = torch.empty(a.size, dtype=torch.float64, pin_memory=True)
        v = t.numpy()
        v[:] = a
        return v

    host = {k: pinned(np.ascontiguousarray(wl[k])) for k in ("x_lo", "x_hi", "w_lo", "w_hi")}
    d = {k: torch.from_numpy(v).to(dev) for k, v in host.items()}
    lo = torch.empty(n, dtype=torch.float64, device=dev)
    hi = torch.empty_like(lo)
    stream = torch.cuda.current_stream(dev)
    sysm = R.System("traffic", n)
    R.reach_set_option(R.OPT_KERNEL, 0)
    R.reach_set_option(R.OPT_STEPS_PER_LAUNCH, 0)

    method_ms = {"mm": [], "cgb": []}

    def step(record=False):
        for method, fn in (("mm", R.reach_mm), ("cgb", R.reach_cgb)):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn(sysm, d["x_lo"], d["x_hi"], d["w_lo"], d["w_hi"], t_final=T_FINAL, dt=DT, lo=lo, hi=hi,
               stream=stream)
            e1.record(stream)
            if record:
                e1.synchronize()
                method_ms[method].append(e0.elapsed_time(e1))

    for _ in range(args.warmup):
        step()
    clocks = Clocks(local)
    barrier()
    clocks.start()
    launches0 = R.reach_kernel_launches()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        step(record=True)
    t1.record(stream)
    barrier()
    clk = clocks.stop()
    launches = R.reach_kernel_launches() - launches0
    ms = max_over_ranks(t0.elapsed_time(t1), dist, dev)
    value = job_rate(2 * 2 * n * NSTEPS * args.steps, world, ms * 1e-3)

    # end to end through the public API with host buffers
    hlo = pinned(np.zeros(n))
    hhi = pinned(np.zeros(n))
    e2e_steps = 0 if args.no_e2e else max(1, min(args.steps, 2))
    if e2e_steps:
        R.reach_mm(sysm, host["x_lo"], host["x_hi"], host["w_lo"], host["w_hi"], t_final=T_FINAL, dt=DT,
                   lo=hlo, hi=hhi)
    barrier()
    te = time.perf_counter()
    for _ in range(e2e_steps):
        R.reach_mm(sysm, host["x_lo"], host["x_hi"], host["w_lo"], host["w_hi"], t_final=T_FINAL, dt=DT,
                   lo=hlo, hi=hhi)
        R.reach_cgb(sysm, host["x_lo"], host["x_hi"], host["w_lo"], host["w_hi"], t_final=T_FINAL, dt=DT,
                    lo=hlo, hi=hhi)
    barrier()
    e2e_sec = max_over_ranks(time.perf_counter() - te, dist, dev)
    e2e_value = job_rate(2 * 2 * n * NSTEPS * e2e_steps, world, e2e_sec) if e2e_steps else None
    h2d = 2 * (2 * n + 2) * 8
    d2h = 2 * 2 * n * 8

    # dominant kernel: the traffic kernel that runs a call's 200 steps in one
    # launch (the MM call is that launch; CGB adds the box conversion)
    per_launch_ms = {m: statistics.median(v) for m, v in method_ms.items()}
    ops = {m: FP64_OPS[m] * 2 * n * NSTEPS for m in method_ms}   # per launch
    achieved = {m: ops[m] / (per_launch_ms[m] * 1e-3) for m in method_ms}
    mm_achieved = achieved["mm"]
    peaks = load_peaks()
    hbm = peaks.get("hbm_gbs", 6400.0)
    eff_gbs = 16.0 * value / world / 1e9
    line = {
        "metric": "state-component RK4 updates/s", "value": value, "unit": "comp-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": headline_config(n, world),
        "e2e": {"value": e2e_value, "unit": "comp-steps/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "roofline": {"bound": "alu", "achieved": mm_achieved / 1e9, "peak": FP64_PEAK_OPS / 1e9,
                     "unit": "Gop/s (FP64 pipe)", "frac": mm_achieved / FP64_PEAK_OPS,
                     "traffic": NCU_DRAM_BYTES_PER_CELL_STEP * n * NSTEPS,
                     "traffic_note": "ncu dram__bytes_read+write of one MM launch on 2^24 cells over 10 steps, "
                                     "scaled to n cells and 200 steps (algorithmic: 16 B x 2n per step)",
                     "kernel": "stencil_traffic_flow<MM>",
                     "per_launch_ms": per_launch_ms, "fp64_ops_per_comp_step": FP64_OPS,
                     "cgb_frac": achieved["cgb"] / FP64_PEAK_OPS,
                     "peak_source": "148 SMs x 2 FP64 ops/clk x 2032 MHz (recipe nominal FP64 1.25 TFLOP/s)",
                     "hbm_effective_gbs": eff_gbs, "hbm_frac_of_measured": eff_gbs / hbm},
        "clocks": clk,
        "gpu_launches": int(launches),
    }
    # the extra sections describe single-GPU workloads: they run in the N = 1
    # run only, so the scaling runs time the headline step and nothing else
    if not args.no_extra and n == N_CELLS and world == 1:
        line["batched"] = bench_batched(R, torch, dev)
        line["ks"] = bench_ks(R, torch, dev)
        line["traffic16"] = bench_traffic16(R)
        line["temporal_blocking"] = bench_temporal_blocking(R, torch, dev)
        line["serving"] = bench_serving(R)
        line["heat3d"] = bench_heat(R, torch, dev)
        line["quad"] = bench_quad(R, torch, dev)
        line["traffic_cgb_local"] = bench_traffic_local(R, torch, dev, d, n)
        line["traffic_sound"] = bench_traffic_sound(R, torch, dev, d, n)
    if rank == 0 and world == 1 and not args.no_cpu and n == N_CELLS:
        if "batched" in line:
            line["cpu_oracle_sections"] = oracle_rates()
        r, sec, cs = cpu_oracle_rate()
        line["cpu_baseline"] = {"value": r, "unit": "comp-steps/s", "cores": 1, **host_cpu(), "kind": "oracle",
                                "sample": f"first {CPU_SAMPLE_CELLS} cells, MM + CGB, 200 steps ({sec:.1f} s)"}
    sysm.close()
    if rank == 0:
        print(json.dumps(line))
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
