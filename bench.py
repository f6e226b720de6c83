#!/usr/bin/env python3
"""Benchmark: phi/c_s/c_l cell-updates per second of the fused explicit step.

Workload (one step = one forward-Euler step of the whole hot path over the
grid): 3D 256^3 FP32, spherical solid seed of radius 20 cells with seeded
surface noise, k_e = 0.1, undercooling 0.5 of the freezing range, D_s/D_l =
1e-4, dx = W/2, 19-point Laplacian, no-flux box.  The device state (phi, c,
d = c_s - c_l and the compensation word of c: 4 x 64 MiB, read and written
every step) is larger than the 129 MB L2, so no flush is needed between steps.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Under torchrun (N > 1) the one 256^3 grid is cut into N z-slabs, one per rank,
with the two ghost planes per cut exchanged over NCCL before every step
(strong scaling); --mode replicas runs one independent grid per rank instead
(weak scaling, no collective on the data path).  Rank 0 prints one JSON line.
`--impl reference` times the FP64 CPU oracle (the method as plainly written)
on this host's cores instead.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_2303_09671_gb300 import workloads as wl  # noqa: E402

METRIC = "phi/c_s/c_l cell-updates/s (3D 256^3 FP32)"
UNIT = "cell-updates/s"
PARAMS = dict(A=1.0, b=1.0)         # trapping parameter and normal-mobility shape


def workload(n):
    return wl.sphere_seed_3d(n=n, radius_cells=20.0, **PARAMS)


def config(n, steps_note):
    return {"workload": f"3D sphere seed {n}^3 FP32 (k_e=0.1, u=0.5, D_s/D_l=1e-4, dx=W/2, "
                        f"19-pt, no-flux, A={PARAMS['A']}, b={PARAMS['b']})",
            "grid": [n, n, n], "dtype": "f32",
            "cache": (f"state {16 * n ** 3 / 1e6:.0f} MB (phi, c, d, c_lo) "
                      + ("> L2 (129 MB), no flush" if 16 * n ** 3 > 129e6 else "fits in L2 (129 MB)")),
            "scaling_unit": "one independent grid per rank", **steps_note}


# Algorithmic FP32 operations of one 3D cell-update (19-point Laplacian), counted
# from the formulas of the step with every add, multiply, reciprocal and log as
# one operation and a fused multiply-add as two: pointwise values 24, phase-field
# rate 117, three faces 3 x 116, update 20 = 509.  Twelve of them are
# reciprocals and logarithms (2 logs per cell, 4 reciprocals in the rate, 2 per
# face), which run on the multi-function unit, not the FMA pipe: 497 FMA-pipe
# operations and 12 MUFU operations per cell-update.
OPS_PER_CELL_UPDATE = 509
MUFU_PER_CELL_UPDATE = 12
FMA_OPS_PER_CELL_UPDATE = OPS_PER_CELL_UPDATE - MUFU_PER_CELL_UPDATE
BYTES_PER_CELL_UPDATE = 24          # FP32 read + write of phi, c_s, c_l (algorithmic)
FP32_LANES, MUFU_LANES = 128, 16    # per SM and clock: FP32 FMA lanes, MUFU results

# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one step3d_kernel
# launch from an ncu capture, per cell-update, and the SHA-256 of the sources
# of the kernel's device code the capture ran.  The figure is reported as null
# as soon as those sources differ from the ones captured.
TRAFFIC_CAPTURE = {
    "bytes_per_cell_update": (280.978176e6 + 231.392768e6) / 256 ** 3,
    "captured_grid": 256,
    "sources": ("pf_step3d.cu", "pf_lanes.cuh", "pf_internal.cuh", "pf_tma.cuh"),
    "sha256": ("cc3e6915fa7a0823646513dba91b988aa60f547d9888bd650733450d5b1313cf",
               "1f20de031e00e90a502b3a819635ef32b8ffbda74d768230f9bfa3e8ef2f8e27",
               "47c14bc813e01ef31966d105fe81a4bca92110885cc77bf8470a1be24dce418c",
               "d0e4d28dc69ba3f9ab24c2a28e424d3fb6e1dc64da959f226126a9eb197caa19"),
}


def step3d_traffic(cells):
    """DRAM bytes per launch at `cells` scaled from the capture, or None if stale."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_2303_09671_gb300", "csrc")
    for name, want in zip(TRAFFIC_CAPTURE["sources"], TRAFFIC_CAPTURE["sha256"]):
        try:
            with open(os.path.join(csrc, name), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != want:
                    return None
        except OSError:
            return None
    return TRAFFIC_CAPTURE["bytes_per_cell_update"] * cells


def max_over_ranks(values, dist=None, device="cpu"):
    """Element-wise maximum of per-rank timings (the slowest rank sets the
    job's time); the identity without a process group."""
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t]


def weak_scaling_rate(cells_per_rank, steps, world, seconds):
    """Whole-job cell-updates per second: every rank advances its own grid."""
    return cells_per_rank * steps * world / seconds


def load_peaks():
    """(HBM GB/s, SM max MHz, source) from MEASURED_PEAKS.json, else the fallback."""
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), float(pk.get("sm_max_mhz", 2070.0)), "measured"
    except Exception:
        return 6800.0, 2070.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *exc):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"], "samples": 0}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(n, max_seconds=25.0):
    """Time the FP64 oracle on a bounded sample of the workload on the host cores."""
    import oracle
    pr, phi, cs, cl = workload(n)
    st = oracle.State(pr, phi.astype(np.float32).astype(np.float64),
                      cs.astype(np.float32).astype(np.float64), cl.astype(np.float32).astype(np.float64))
    st.step(1)                               # warm-up (page-in, thread start)
    cells = int(np.prod(pr["n"]))
    steps, t0 = 0, time.perf_counter()
    while True:
        st.step(1)
        steps += 1
        el = time.perf_counter() - t0
        if el > max_seconds or steps >= 3:
            break
    out = {"value": cells * steps / el, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"{steps} FP64 oracle steps of the full {n}^3 grid after 1 warm-up step",
           "seconds": el}
    # one host thread on a 64^3 grid of the same recipe (seed radius scaled to the box)
    all_threads = oracle.num_threads()
    try:
        oracle.set_threads(1)
        pr1, phi1, cs1, cl1 = wl.sphere_seed_3d(n=64, radius_cells=5.0, **PARAMS)
        st1 = oracle.State(pr1, phi1, cs1, cl1)
        st1.step(1)
        s1, t1 = 0, time.perf_counter()
        while True:
            st1.step(1)
            s1 += 1
            el1 = time.perf_counter() - t1
            if el1 > 2.0 or s1 >= 5:
                break
        out["single_thread_64"] = {"value": 64 ** 3 * s1 / el1, "unit": UNIT, "cores": 1,
                                   "sample": f"{s1} FP64 oracle steps of a 64^3 sphere seed, one thread"}
    finally:
        oracle.set_threads(all_threads)
    return out


def sm_count(device=0):
    import torch
    return int(torch.cuda.get_device_properties(device).multi_processor_count)


def kv_brief(steps=500):
    """Bounded k(V) figures for the default line.  (1) The 256-instance sweep of
    kv_sweep_inputs for a fixed budget of `steps` steps: one batched run
    (persistent launches in a CUDA graph) against a per-instance loop of the
    single-handle step, launched step by step and, a stronger baseline, with
    each instance's steps captured in a CUDA graph and replayed.  (2) Four
    steep-gradient pulled fronts (G = 0.2 per W, D_s/D_l = 0.1, A = b = 1, V in
    0.2..2) run to steady state by the batch's own convergence test
    (|dk/dt| < 1e-8 per unit time after 200 W of pulling), with the steady state
    checked by mass balance: the solid 5-20 W behind the front carries c_inf."""
    import torch
    from paper_2303_09671_gb300 import pf
    lengths, vs, prs, dts, phi, cs, cl = kv_sweep_inputs()
    f32 = [a.astype(np.float32) for a in (phi, cs, cl)]
    K = int(steps)
    pf.run_batch(prs[0], lengths, vs, *f32, dt=dts, max_steps=K, steps_per_launch=K,
                 launches_per_graph=1, tol=-1.0)                      # warm-up (autotune)
    res = pf.run_batch(prs[0], lengths, vs, *f32, dt=dts, max_steps=K, steps_per_launch=K,
                       launches_per_graph=1, tol=-1.0)
    batch_s = res["gpu_ms"] * 1e-3
    stream = torch.cuda.Stream()
    loop_s = graph_s = 0.0
    o = 0
    with torch.cuda.stream(stream):
        for pr, n, dt in zip(prs, lengths, dts):
            n = int(n)
            src = [a[o:o + n] for a in f32]
            o += n
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            with pf.Sim(dict(pr, dt=dt), "fp32", stream=stream.cuda_stream) as s:
                s.set_fields(*src)
                e0.record(stream)
                s.step(K)
                e1.record(stream)
                e1.synchronize()
                loop_s += e0.elapsed_time(e1) * 1e-3
                s.set_fields(*src)
                s.set_clock(0, 0)
                g = torch.cuda.CUDAGraph()
                with torch.cuda.graph(g, stream=stream):
                    s.step(K)
                e0.record(stream)
                g.replay()
                e1.record(stream)
                e1.synchronize()
                graph_s += e0.elapsed_time(e1) * 1e-3
                del g
    out = {"workload": "256 pulled fronts of kv_sweep_inputs, fixed budget", "steps": K,
           "batch_gpu_s": batch_s, "loop_gpu_s": loop_s, "loop_graph_gpu_s": graph_s,
           "speedup_vs_loop": loop_s / batch_s, "speedup_vs_graph_loop": graph_s / batch_s,
           "cells_per_thread": int(res["cells_per_thread"])}
    # steady state of steep-gradient fronts
    k_e, vs4, n = 0.1, np.array([0.2, 0.5, 1.0, 2.0]), 2048
    prs4, fl = [], [[], [], []]
    for v in vs4:
        pr, a, b, c = wl.pulled_front_1d(N=n, dx=0.5, V=float(v), k_e=k_e, D_s=0.1, A=1.0, b=1.0,
                                         G_theta=0.2, front_cell=64)
        prs4.append(pr)
        for lst, x in zip(fl, (a, b, c)):
            lst.append(x)
    dts4 = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs4, vs4)]
    packed = [np.concatenate(x).astype(np.float32) for x in fl]
    t0 = time.perf_counter()
    r = pf.run_batch(prs4[0], [n] * 4, vs4, *packed, dt=dts4, max_steps=200000, steps_per_launch=1000,
                     launches_per_graph=4, check_every=1000, window=20.0, tol=1e-8, min_travel=200.0,
                     want_fields=True)
    wall = time.perf_counter() - t0
    mb = []
    for i in range(4):
        f = r["phi"][i * n:(i + 1) * n].astype(np.float64)
        j = np.where((f[:-1] >= 0.5) & (f[1:] < 0.5))[0]
        if len(j) != 1 or j[0] < 20:      # no front in the window (a fully trapping front falls back
            mb.append(None)               # past the cold end), or too little solid behind it
            continue
        p = f ** 3 * (6 * f * f - 15 * f + 10)
        c = p * r["cs"][i * n:(i + 1) * n] + (1 - p) * r["cl"][i * n:(i + 1) * n]
        mb.append(float(np.abs(c[max(0, j[0] - 40):j[0] - 10] - 1.0).max()))
    out["steady"] = {"workload": "4 pulled fronts x 2048 cells, G=0.2/W, D_s/D_l=0.1, k_e=0.1, A=b=1, FP32",
                     "V": vs4.tolist(), "converged": r["converged"].astype(int).tolist(),
                     "steps": r["steps"].tolist(), "t": r["t"].tolist(), "k_v": r["k_v"].tolist(),
                     "solid_behind_front_minus_cinf": mb, "gpu_s": r["gpu_ms"] * 1e-3, "wall_s": wall,
                     "criterion": "|dk/dt| < 1e-8 per unit time over 20 time units, after 200 W of pulling"}
    return out


def adjoint_brief(steps=5000):
    """Bounded derivative figures for the default line: d k_i / d(M_phi, A, b)
    of the 16 pulled fronts of adjoint_inputs over `steps` FP32 steps, by the
    tangent-linear run and by the reverse sweep, each against the forward run."""
    from paper_2303_09671_gb300 import pf
    lengths, vs, prs, dts, phi, cs, cl, kt = adjoint_inputs()
    K = int(steps)
    f32 = [a.astype(np.float32) for a in (phi, cs, cl)]
    spl = max(1, K // 4)
    fw = dict(dt=dts, max_steps=K, steps_per_launch=spl, launches_per_graph=4, check_every=K, tol=-1.0)
    pf.run_batch(prs[0], lengths, vs, *f32, **dict(fw, max_steps=spl, launches_per_graph=1))     # warm-up
    fwd = pf.run_batch(prs[0], lengths, vs, *f32, **fw)
    out = {"workload": "16 pulled fronts x 2048 cells, V 0.05..5, A=1.1, b=1, FP32", "steps": K,
           "forward_gpu_s": fwd["gpu_ms"] * 1e-3}
    ref = None
    for mode in ("tangent", "reverse"):
        kw = dict(k_target=kt, dt=dts, mode=mode)
        if mode == "tangent":
            kw["steps_per_launch"] = spl
        pf.adjoint(prs[0], lengths, vs, *f32, spl, **kw)                                          # warm-up
        a = pf.adjoint(prs[0], lengths, vs, *f32, K, **kw)
        out[mode] = {"gpu_s": a["gpu_ms"] * 1e-3, "cost_ratio": a["gpu_ms"] / fwd["gpu_ms"]}
        if ref is None:
            ref = a["dk"]
        else:
            out[mode]["dk_vs_tangent_max_rel"] = float(np.abs(a["dk"] - ref).max() / np.abs(ref).max())
    return out


def run_slabs(args, torch, dist, world, rank, local):
    """N > 1: the one 256^3 grid cut into `world` z-slabs, one per rank; before
    every step each rank sends its two boundary planes per cut to its
    neighbours and imports theirs (NCCL point-to-point, 2 x 2 x 256^2 x 16 B =
    4.2 MB per rank and step) while the z-chunks of its step that read no
    ghost plane already run (pf_step_begin), then steps the chunks next to the
    cuts (pf_step_end).  Strong scaling: the work is fixed, `value` counts the
    whole grid's cells."""
    from paper_2303_09671_gb300.slabs import SlabRun
    n = args.size
    pr, phi, cs, cl = workload(n)
    cells = int(np.prod(pr["n"]))
    run = SlabRun(pr, "fp32", rank, world, dist)
    z0, nzl = run.z0, run.nzl
    own = [np.ascontiguousarray(a[z0:z0 + nzl], dtype=np.float32) for a in (phi, cs, cl)]
    del phi, cs, cl
    run.set_fields(*own)
    S0 = run.solute_total()
    for _ in range(args.warmup):
        run.step(1)
    dist.barrier()
    torch.cuda.synchronize()
    stream = torch.cuda.current_stream()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        ev0.record(stream)
        for _ in range(args.steps):
            run.step(1)
        ev1.record(stream)
        ev1.synchronize()
    dist.barrier()
    ms = ev0.elapsed_time(ev1)
    drift = abs(run.solute_total() - S0) / abs(S0)
    # end to end: each rank uploads its slab from pinned host memory, exchanges,
    # steps, and reads its slab back
    pinned = [torch.from_numpy(a).pin_memory().numpy() for a in own]
    back = [torch.empty(a.shape, dtype=torch.float32).pin_memory().numpy() for a in own]
    ke = max(1, args.e2e_steps)
    dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ke):
        run.set_fields(*pinned)
        run.step(1)
        run.sim.get_fields(out_host=back)
    torch.cuda.synchronize()
    e2e_s = time.perf_counter() - t0
    ms_max, e2e_max = max_over_ranks([ms, e2e_s], dist, device="cuda")
    if rank == 0:
        value = cells * args.steps / (ms_max * 1e-3)
        hbm_peak, sm_mhz, how = load_peaks()
        sms = sm_count(local)
        own_cells = int(np.prod(own[0].shape))
        step_s = ms / args.steps * 1e-3
        achieved = FMA_OPS_PER_CELL_UPDATE * own_cells / step_s / 1e12
        alu_peak = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config(n, {"parallelism": f"z-slabs x{world}: NCCL send/recv of 2 ghost planes per cut "
                                                "and step (pf_get_halo / pf_set_halo), overlapped with the "
                                                "step's interior chunks (pf_step_begin / pf_step_end)",
                                 "scaling_unit": "one grid over all ranks"}),
            "roofline": {"bound": "alu", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                         "frac": achieved / alu_peak, "traffic": None,
                         "traffic_note": "rank 0's slab; the step time includes the halo exchange",
                         "kernel": "step3d_kernel<float,32,16,19-point>",
                         "ops_per_cell_update": FMA_OPS_PER_CELL_UPDATE},
            "e2e": {"value": cells * ke / e2e_max, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * cells,
                    "d2h_bytes_per_step": 3 * 4 * cells, "steps": ke},
            "gpu_launches": args.steps, "solute_drift": drift, "clocks": clk.summary(),
        }
        print(json.dumps(out), flush=True)
    run.close()
    dist.destroy_process_group()
    return 0


def run_calibrate_steady(args):
    """Calibration of the trapping parameter A and the mobility shape b so
    that steady pulled fronts follow the target k(V) = (k_e + V/V_D)/(1 + V/V_D),
    V_D = 1 (the tuning of Sec. "Tailoring the partition coefficient: Selection
    of A"): 8 fronts with V log-spaced in 0.1..0.5, 2048 cells, the steep frozen
    gradient (0.2 per W, D_s/D_l = 0.1, k_e = 0.1) on which they reach steady
    state within the 10^5 steps of a run, FP32 value + tangent-linear
    derivative per iteration (pf_adjoint), Adam on (log A, log b) with A kept in
    [0.9, 2] and b in [0.05, 1] (where the model stays finite), from A = 1.1,
    b = 1."""
    from paper_2303_09671_gb300 import pf
    n, k_e = 2048, 0.1
    vs = np.logspace(np.log10(0.1), np.log10(0.5), 8)
    nsteps = args.steps if args.steps != 2000 else 100000
    iters = args.calibrate if args.calibrate > 0 else 40
    made = [wl.pulled_front_1d(N=n, dx=0.5, V=float(v), k_e=k_e, D_s=0.1, A=1.1, b=1.0, G_theta=0.2,
                               front_cell=64) for v in vs]
    prs = [m[0] for m in made]
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    f32 = [np.concatenate([m[i] for m in made]).astype(np.float32) for i in (1, 2, 3)]
    kt = (k_e + vs) / (1 + vs)
    hist = []
    t0 = time.perf_counter()
    theta, losses = pf.calibrate(prs[0], [n] * len(vs), vs, *f32, nsteps, kt, iters=iters, lr=0.05,
                                 wrt=("A", "b"), dt=dts, bounds={"A": (0.9, 2.0), "b": (0.05, 1.0)},
                                 callback=lambda it, cur, r: hist.append(r["k"].tolist()))
    wall = time.perf_counter() - t0
    out = {"metric": "k(V) calibration loss sum (k - k_target)^2 (8 steady pulled fronts)", "value": losses[-1],
           "unit": "loss", "n_gpus": 1, "steps": nsteps, "higher_is_better": False, "dtype": "f32",
           "data": "synthetic",
           "config": {"workload": "8 pulled fronts x 2048 cells, V log-spaced 0.1..0.5, G=0.2/W, D_s/D_l=0.1, "
                                  "k_e=0.1, target (k_e+V)/(1+V)", "iters": iters, "lr": 0.05,
                      "start": {"A": 1.1, "b": 1.0}, "bounds": {"A": [0.9, 2.0], "b": [0.05, 1.0]}},
           "loss_first": losses[0], "loss_last": losses[-1], "params": theta, "wall_s": wall,
           "V": vs.tolist(), "k_target": kt.tolist(), "k_first": hist[0], "k_last": hist[-1]}
    print(json.dumps(out), flush=True)
    return 0


def run_banding(args):
    """The band-forming workload of Sec. "Oscillations and solute bands": Si-As
    pulled fronts at G = 1.4e6 K/m and D_s/D_l = 1e-3 (banding_front), pulled
    at 32 speeds from 0.05 to 0.5 m/s, 8192 cells each (4096 W), FP32, through the
    batched kernel for `--steps` steps (default 2x10^5 = 2x10^4 time units),
    at the two trapping settings that stay finite from this start (A = 1, b = 1
    and A = 1.5, b = 0.1; the paper's own A = 2, b = 1e-3 diverges).  Reports
    cell-updates/s and, per front, the final k_v and the front's offset from
    the pulled reference position; oscillating fronts would show up as
    unsettled offsets and k_v between partitioning and trapping."""
    from paper_2303_09671_gb300 import pf
    K = args.steps if args.steps != 2000 else 200000
    vps = list(np.round(np.linspace(0.05, 0.5, 32), 6))
    n = 8192
    out = {"metric": "phi/c_s/c_l cell-updates/s (banding: Si-As pulled fronts, batched)", "unit": "cell-updates/s",
           "n_gpus": 1, "steps": K, "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "Si-As, G=1.4e6 K/m, D_s/D_l=1e-3, v_p 0.05..0.5 m/s (32), W=d0, 8192 cells, "
                                  "start at the liquidus of c_inf"}, "runs": []}
    total_cells, total_s = 0, 0.0
    for A, b in ((1.0, 1.0), (1.5, 0.1)):
        made = [wl.banding_front(v, A=A, b=b, N=n) for v in vps]
        prs = [m[0] for m in made]
        vs = [pr["v_pull"] for pr in prs]
        dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
        f32 = [np.concatenate([m[i] for m in made]).astype(np.float32) for i in (1, 2, 3)]
        spl = 5000
        m = len(vs)
        pf.run_batch(prs[0], [n] * m, vs, *f32, dt=dts, max_steps=spl, steps_per_launch=spl,
                     launches_per_graph=1, tol=-1.0)                                   # warm-up
        res = pf.run_batch(prs[0], [n] * m, vs, *f32, dt=dts, max_steps=K, steps_per_launch=spl,
                           launches_per_graph=4, check_every=K, tol=-1.0, want_fields=True)
        total_cells += m * n * K
        total_s += res["gpu_ms"] * 1e-3
        for i, (pr, v, dt) in enumerate(zip(prs, vs, dts)):
            f = res["phi"][i * n:(i + 1) * n].astype(np.float64)
            j = np.where((f[:-1] >= 0.5) & (f[1:] < 0.5))[0]
            t = float(res["t"][i])
            shifts = int(np.floor(v * t / pr["dx"]))
            if len(j):
                a_, b_ = f[j[-1]], f[j[-1] + 1]
                xw = (j[-1] + 0.5 + (a_ - 0.5) / (a_ - b_)) * pr["dx"]
                offset = xw + shifts * pr["dx"] - pr["x0"] - v * t
            else:
                offset = None
            out["runs"].append({"A": A, "b": b, "v_p_m_s": vps[i], "V": v, "t": t, "k_v": float(res["k_v"][i]),
                                "front_minus_pulled_W": offset, "crossings": int(len(j))})
    out["value"] = total_cells / total_s
    out["gpu_s"] = total_s
    print(json.dumps(out), flush=True)
    return 0


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    import oracle
    n = args.size
    pr, phi, cs, cl = workload(n)
    st = oracle.State(pr, phi.astype(np.float32).astype(np.float64),
                      cs.astype(np.float32).astype(np.float64), cl.astype(np.float32).astype(np.float64))
    cells = int(np.prod(pr["n"]))
    for _ in range(args.warmup):
        st.step(1)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        st.step(1)
    el = time.perf_counter() - t0
    v = cells * args.steps / el
    out = {"impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
           "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
           "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
           "data": "synthetic", "config": config(n, {"arm": "FP64 CPU oracle, full grid per step"}),
           "cpu_baseline": {"value": v, "unit": UNIT, "cores": oracle.num_threads(), "kind": "oracle",
                            "sample": f"full {n}^3 grid, {args.steps} timed steps"},
           "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)
    return 0


def kv_sweep_inputs(n_inst=256, seed=4):
    """256 1D pulled fronts: lengths uniform in 512..8192 cells (seeded), pulling
    velocities log-spaced in 1e-3..10 (scaled), frozen gradient 5.25e-3 per W."""
    rng = np.random.default_rng(seed)
    lengths = rng.integers(512, 8193, size=n_inst)
    vs = np.logspace(-3, 1, n_inst)
    prs, phis, css, cls = [], [], [], []
    for n, v in zip(lengths, vs):
        pr, phi, cs, cl = wl.pulled_front_1d(N=int(n), dx=0.5, V=float(v), G_theta=5.25e-3,
                                             front_cell=128, A=1.0, b=1.0)
        prs.append(pr)
        phis.append(phi)
        css.append(cs)
        cls.append(cl)
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    return lengths, vs, prs, dts, np.concatenate(phis), np.concatenate(css), np.concatenate(cls)


def run_kv_to_steady(args):
    """The k(V) sweep as its configuration states it: all 256 fronts of
    kv_sweep_inputs run until |dk_v/dt| < 1e-8 per unit time (over 20 time
    units, after 200 W of pulling) or 2x10^6 steps, FP32, one batched run;
    reports the time, how many converged, and per front k_v, the steps taken
    and the mass balance of the solid 5-20 W behind the front (|c - c_inf|,
    which vanishes at a true steady state; None when the front left the
    window or sits too close to its cold end)."""
    from paper_2303_09671_gb300 import pf
    lengths, vs, prs, dts, phi, cs, cl = kv_sweep_inputs()
    f32 = [a.astype(np.float32) for a in (phi, cs, cl)]
    t0 = time.perf_counter()
    r = pf.run_batch(prs[0], lengths, vs, *f32, dt=dts, max_steps=2000000, steps_per_launch=5000,
                     launches_per_graph=4, check_every=5000, window=20.0, tol=1e-8, min_travel=200.0,
                     want_fields=True)
    wall = time.perf_counter() - t0
    fronts, o = [], 0
    for i, n in enumerate(lengths):
        n = int(n)
        f = r["phi"][o:o + n].astype(np.float64)
        j = np.where((f[:-1] >= 0.5) & (f[1:] < 0.5))[0]
        p = f ** 3 * (6 * f * f - 15 * f + 10)
        c = p * r["cs"][o:o + n] + (1 - p) * r["cl"][o:o + n]
        mb = float(np.abs(c[max(0, j[0] - 40):j[0] - 10] - 1.0).max()) if len(j) == 1 and j[0] >= 20 else None
        fronts.append({"V": float(vs[i]), "n": n, "k_v": float(r["k_v"][i]), "steps": int(r["steps"][i]),
                       "converged": bool(r["converged"][i]), "solid_minus_cinf": mb})
        o += n
    conv = r["converged"].astype(bool)
    steady = [fr for fr in fronts if fr["converged"] and fr["solid_minus_cinf"] is not None
              and fr["solid_minus_cinf"] < 1e-3]
    out = {"metric": "time to steady k(V), 256 pulled fronts (batched)", "value": r["gpu_ms"] * 1e-3, "unit": "s",
           "n_gpus": 1, "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "kv-sweep: 256 1D pulled fronts, lengths U{512..8192} (seed 4), V log-spaced "
                                  "1e-3..10, G=5.25e-3, A=1, b=1, to |dk/dt| < 1e-8 or 2e6 steps"},
           "wall_s": wall, "converged": int(conv.sum()), "steady_by_mass_balance": len(steady),
           "steps_converged_max": int(r["steps"][conv].max()) if conv.any() else None,
           "cell_updates_per_s": float(np.sum(np.asarray(lengths) * r["steps"]) / (r["gpu_ms"] * 1e-3)),
           "fronts": fronts}
    print(json.dumps(out), flush=True)
    return 0


def instance_shares(lengths, parts):
    """Contiguous shares [(first, count)] of the instances for `parts` ranks,
    cut where the running cell count crosses r / parts of the total, so that
    every rank steps about the same number of cells; every share holds at
    least one instance while there are enough."""
    lengths = np.asarray(lengths, dtype=np.int64)
    n, parts = len(lengths), int(parts)
    if parts < 1 or parts > n:
        raise ValueError("need 1 <= parts <= instances")
    cum = np.cumsum(lengths)
    cuts = [0]
    for r in range(1, parts):
        c = int(np.searchsorted(cum, cum[-1] * r / parts, side="left")) + 1
        cuts.append(min(max(c, cuts[-1] + 1), n - (parts - r)))
    cuts.append(n)
    return [(cuts[r], cuts[r + 1] - cuts[r]) for r in range(parts)]


def run_kv_sweep_ranks(args, world, rank, local):
    """N > 1: the 256 fronts split across ranks by instance_shares, each rank
    one batched run of its share, no exchange between them (NCCL for the
    barriers and the max over ranks only)."""
    import datetime
    import torch
    import torch.distributed as dist
    from paper_2303_09671_gb300 import pf
    torch.cuda.set_device(local)
    dist.init_process_group("nccl", init_method="env://", timeout=datetime.timedelta(seconds=300))
    out = kv_sweep_shard(args, dist, world, rank, pf.run_batch, device="cuda")
    if out is not None:
        print(json.dumps(out), flush=True)
    dist.barrier()
    dist.destroy_process_group()
    return 0


def kv_sweep_shard(args, dist, world, rank, run_batch, device):
    """Rank `rank`'s share of the sweep through run_batch (pf.run_batch's
    signature), timed by its device milliseconds; rank 0 returns the line
    (others None).  Strong scaling: the sweep is fixed, `value` counts every
    rank's instance-steps over the slowest rank's device time."""
    lengths, vs, prs, dts, phi, cs, cl = kv_sweep_inputs()
    first, count = instance_shares(lengths, world)[rank]
    off = np.concatenate([[0], np.cumsum(lengths)])
    lo, hi = int(off[first]), int(off[first + count])
    mine = slice(first, first + count)
    f32 = [np.ascontiguousarray(a[lo:hi], dtype=np.float32) for a in (phi, cs, cl)]
    K = args.steps
    spl = max(1, K // 4)
    kw = dict(dt=dts[mine], steps_per_launch=spl, tol=-1.0)
    run_batch(prs[0], lengths[mine], vs[mine], *f32, max_steps=spl, launches_per_graph=1, **kw)   # warm-up
    dist.barrier()
    res = run_batch(prs[0], lengths[mine], vs[mine], *f32, max_steps=K, launches_per_graph=4, **kw)
    (batch_s,) = max_over_ranks([res["gpu_ms"] * 1e-3], dist, device=device)
    if rank != 0:
        return None
    cells = int(np.sum(lengths))
    return {"metric": "1D pulled-front instance-steps/s (256 instances, 512..8192 cells)",
            "value": len(lengths) * K / batch_s, "unit": "instance-steps/s", "n_gpus": world, "steps": K,
            "higher_is_better": True, "scaling": "strong", "dtype": "f32", "data": "synthetic",
            "config": {"workload": "kv-sweep: 256 1D pulled fronts, lengths U{512..8192} (seed 4), "
                                   "V log-spaced 1e-3..10, G=5.25e-3, A=1, b=1, fixed step budget",
                       "parallelism": f"instances split across {world} ranks by cells, no exchange",
                       "cells_total": cells},
            "batch_gpu_s": batch_s, "cell_updates_per_s": cells * K / batch_s}


def run_kv_sweep(args):
    """Batched k(V) sweep (one persistent launch per chunk, CUDA graph) against a
    per-instance loop of the single-handle path, same steps, same GPU."""
    import torch
    from paper_2303_09671_gb300 import pf
    if args.to_steady:
        return run_kv_to_steady(args)
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if world > 1:
        return run_kv_sweep_ranks(args, world, int(os.environ.get("RANK", "0")),
                                  int(os.environ.get("LOCAL_RANK", "0")))
    lengths, vs, prs, dts, phi, cs, cl = kv_sweep_inputs()
    K = args.steps
    f32 = [a.astype(np.float32) for a in (phi, cs, cl)]
    spl = max(1, K // 4)
    pf.run_batch(prs[0], lengths, vs, *f32, dt=dts, max_steps=spl, steps_per_launch=spl,
                 launches_per_graph=1, tol=-1.0)                     # warm-up (autotune, module load)
    t0 = time.perf_counter()
    res = pf.run_batch(prs[0], lengths, vs, *f32, dt=dts, max_steps=K, steps_per_launch=spl,
                       launches_per_graph=4, tol=-1.0)
    batch_wall = time.perf_counter() - t0
    batch_s = res["gpu_ms"] * 1e-3
    # per-instance loop of the single-handle kernel
    stream = torch.cuda.Stream()
    loop_s, o = 0.0, 0
    with torch.cuda.stream(stream):
        for pr, n, dt in zip(prs, lengths, dts):
            n = int(n)
            with pf.Sim(dict(pr, dt=dt), "fp32", stream=stream.cuda_stream) as s:
                s.set_fields(f32[0][o:o + n], f32[1][o:o + n], f32[2][o:o + n])
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.step(K)
                e1.record(stream)
                e1.synchronize()
                loop_s += e0.elapsed_time(e1) * 1e-3
            o += n
    cells = int(np.sum(lengths))
    out = {"metric": "1D pulled-front instance-steps/s (256 instances, 512..8192 cells)",
           "value": len(lengths) * K / batch_s, "unit": "instance-steps/s", "n_gpus": 1, "steps": K,
           "higher_is_better": True, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "kv-sweep: 256 1D pulled fronts, lengths U{512..8192} (seed 4), "
                                  "V log-spaced 1e-3..10, G=5.25e-3, A=1, b=1, fixed step budget",
                      "cells_total": cells, "cells_per_thread": res["cells_per_thread"]},
           "batch_gpu_s": batch_s, "batch_wall_s": batch_wall, "batch_launches": res["launches"],
           "loop_gpu_s": loop_s, "loop_launches": len(lengths) * K,
           "speedup_vs_loop": loop_s / batch_s,
           "cell_updates_per_s": cells * K / batch_s}
    print(json.dumps(out), flush=True)
    return 0


def adjoint_inputs(n_inst=16, n=2048, A=1.1, b=1.0):
    """16 pulled fronts of 2048 cells, V log-spaced in 0.05..5 (scaled), the
    frozen gradient of the k(V) sweep; target k(V) = (k_e + V/V_D)/(1 + V/V_D),
    V_D = 1 (the velocity-dependent partition law the calibration fits)."""
    vs = np.logspace(np.log10(0.05), np.log10(5.0), n_inst)
    prs, phis, css, cls = [], [], [], []
    for v in vs:
        pr, phi, cs, cl = wl.pulled_front_1d(N=n, dx=0.5, V=float(v), G_theta=5.25e-3, front_cell=256,
                                             A=A, b=b)
        prs.append(pr)
        phis.append(phi)
        css.append(cs)
        cls.append(cl)
    dts = [min(0.9 * wl.stable_dt(pr), 0.5 * pr["dx"] / v) for pr, v in zip(prs, vs)]
    k_e = prs[0]["k_e"]
    k_target = (k_e + vs) / (1.0 + vs)
    return [n] * n_inst, vs, prs, dts, np.concatenate(phis), np.concatenate(css), np.concatenate(cls), k_target


def run_adjoint(args):
    """Cost of the parameter derivatives d k_i / d(M_phi, A, b) (pf_adjoint, FP32
    value + derivative) against the forward run alone (pf_run_batch, same steps)."""
    from paper_2303_09671_gb300 import pf
    lengths, vs, prs, dts, phi, cs, cl, kt = adjoint_inputs()
    K = args.steps
    f32 = [a.astype(np.float32) for a in (phi, cs, cl)]
    spl = max(1, K // 4)
    fw = dict(dt=dts, max_steps=K, steps_per_launch=spl, launches_per_graph=4, check_every=K, tol=-1.0)
    pf.run_batch(prs[0], lengths, vs, *f32, **dict(fw, max_steps=spl, launches_per_graph=1))   # warm-up
    t0 = time.perf_counter()
    fwd = pf.run_batch(prs[0], lengths, vs, *f32, **fw)
    fwd_wall = time.perf_counter() - t0
    pf.adjoint(prs[0], lengths, vs, *f32, spl, k_target=kt, dt=dts, steps_per_launch=spl)       # warm-up
    t0 = time.perf_counter()
    adj = pf.adjoint(prs[0], lengths, vs, *f32, K, k_target=kt, dt=dts, steps_per_launch=spl)
    adj_wall = time.perf_counter() - t0
    ratio = adj["gpu_ms"] / fwd["gpu_ms"]
    # the same derivatives by the reverse sweep (checkpoints every ~sqrt(K) steps)
    pf.adjoint(prs[0], lengths, vs, *f32, spl, k_target=kt, dt=dts, mode="reverse")             # warm-up
    t0 = time.perf_counter()
    rev = pf.adjoint(prs[0], lengths, vs, *f32, K, k_target=kt, dt=dts, mode="reverse")
    rev_wall = time.perf_counter() - t0
    out = {"metric": "adjoint/forward cost ratio (d k_i / d(M_phi, A, b), 16 pulled fronts x 2048 cells)",
           "value": ratio, "unit": "ratio of device times", "n_gpus": 1, "steps": K,
           "higher_is_better": False, "dtype": "f32", "data": "synthetic",
           "config": {"workload": "16 1D pulled fronts x 2048 cells, V log-spaced 0.05..5, G=5.25e-3, "
                                  "A=1.1, b=1, k_target=(k_e+V)/(1+V)",
                      "parameters": list(pf.ADJ_PARAMS)},
           "forward_gpu_s": fwd["gpu_ms"] * 1e-3, "forward_wall_s": fwd_wall,
           "adjoint_gpu_s": adj["gpu_ms"] * 1e-3, "adjoint_wall_s": adj_wall,
           "wall_ratio": adj_wall / fwd_wall,
           "k_forward_vs_adjoint_max_abs": float(np.abs(fwd["k_v"] - adj["k"]).max()),
           "loss": adj["loss"], "grad": [float(g) for g in adj["grad"]],
           "reverse": {"gpu_s": rev["gpu_ms"] * 1e-3, "wall_s": rev_wall,
                       "cost_ratio": rev["gpu_ms"] / fwd["gpu_ms"],
                       "dk_vs_tangent_max_rel": float(np.abs(rev["dk"] - adj["dk"]).max()
                                                      / np.abs(adj["dk"]).max()),
                       "path": "reverse sweep of the fused step, checkpoints every ceil(sqrt(K)) steps"}}
    if args.calibrate > 0:
        # Adam on log(M_phi, A, b) towards the target curve, one pf_adjoint per iteration
        t0 = time.perf_counter()
        hist, err = [], None
        try:
            theta, hist = pf.calibrate(prs[0], lengths, vs, *f32, K, kt, iters=args.calibrate, lr=0.02,
                                       precision="fp32", dt=dts)
        except pf.PFError as e:   # a parameter set on which the run does not stay finite
            theta, err = None, str(e)
        out["calibration"] = {"iters": args.calibrate, "lr": 0.02, "wall_s": time.perf_counter() - t0,
                              "loss_first": hist[0] if hist else None, "loss_last": hist[-1] if hist else None,
                              "loss_min": min(hist) if hist else None, "params": theta, "error": err,
                              "start": {k: prs[0][k] for k in pf.ADJ_PARAMS}}
    print(json.dumps(out), flush=True)
    return 0


def run_secondary(args):
    """The other workload shapes of the paper on the same step (not the headline):
    planar1d = 1D planar front, N = 1024, FP64, dx = W/4, the free energy F_h
    read back every step (Sec. "Numerical technique"; latency-bound by design);
    perturbed2d = 2D perturbed front 1024^2 FP32, 9-point Laplacian, periodic
    along the front, no-flux across (state 16.8 MB: L2-resident)."""
    print(json.dumps(measure_secondary(args.workload, args.steps, max(args.warmup, 3))), flush=True)
    return 0


def secondary_brief(workload, steps):
    """The 1D and 2D configurations at their full step counts for the default
    line: cell-updates/s and ms per step on the device (CUDA events), F_h
    monotonicity for the 1D front."""
    o = measure_secondary(workload, steps, 3, full=False)
    keep = ("value", "unit", "ms_per_step", "steps", "dtype", "wall_s", "energy_non_increasing", "steps_per_s")
    brief = {k: o[k] for k in keep if k in o}
    brief["workload"] = o["config"]["workload"]
    brief["grid"] = o["config"]["grid"]
    if "path" in o["config"]:
        brief["path"] = o["config"]["path"]
    return brief


def measure_secondary(workload, K, W, full=True):
    import torch
    from paper_2303_09671_gb300.pf import Sim
    stream = torch.cuda.Stream()
    if workload == "planar1d":
        pr, phi, cs, cl = wl.planar_1d(A=1.0, b=1.0)
        prec, per_step_energy = "fp64", True
        desc = "1D planar front N=1024 FP64 (k_e=0.1, u=0.3, D_s/D_l=1e-4, dx=W/4), F_h every step"
    else:
        pr, phi, cs, cl = wl.perturbed_front_2d(A=1.0, b=1.0)
        prec, per_step_energy = "fp32", False
        desc = ("2D perturbed front 1024^2 FP32 (k_e=0.15, u=0.3, D_s/D_l=1e-3, dx=W/2, 9-pt, "
                "periodic along the front, no-flux across, 8 seeded modes, amplitude 2 cells)")
    cells = int(np.prod(pr["n"]))
    with torch.cuda.stream(stream):
        sim = Sim(pr, prec, stream=stream.cuda_stream)
        sim.set_fields(phi, cs, cl)
        for _ in range(W):
            sim.step(1)
            if per_step_energy:
                sim.energy()
        stream.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        per_call = None
        if per_step_energy and full:
            # F_h after every step recorded on the device (pf_step_energies), read back once
            t0 = time.perf_counter()
            ev0.record(stream)
            F = sim.step_energies(K)
            ev1.record(stream)
            ev1.synchronize()
            wall = time.perf_counter() - t0
            ms = ev0.elapsed_time(ev1)
            # the same with a host read-back of F_h after every step (pf_step + pf_energy)
            t0 = time.perf_counter()
            ev0.record(stream)
            for _ in range(K):
                sim.step(1)
                sim.energy()
            ev1.record(stream)
            ev1.synchronize()
            per_call = {"ms_per_step": ev0.elapsed_time(ev1) / K, "wall_s": time.perf_counter() - t0,
                        "path": "pf_step + pf_energy per step (F_h read back every step)"}
        elif per_step_energy:
            t0 = time.perf_counter()
            ev0.record(stream)
            F = sim.step_energies(K)
            ev1.record(stream)
            ev1.synchronize()
            wall = time.perf_counter() - t0
            ms = ev0.elapsed_time(ev1)
        else:
            t0 = time.perf_counter()
            ev0.record(stream)
            for _ in range(K):
                sim.step(1)
            ev1.record(stream)
            ev1.synchronize()
            wall = time.perf_counter() - t0
            ms = ev0.elapsed_time(ev1)
        sim.close()
    out = {"metric": f"phi/c_s/c_l cell-updates/s ({workload})", "value": cells * K / (ms * 1e-3),
           "unit": "cell-updates/s", "n_gpus": 1, "steps": K, "warmup": W, "ms_per_step": ms / K,
           "higher_is_better": True, "dtype": "f64" if prec == "fp64" else "f32", "data": "synthetic",
           "config": {"workload": desc, "grid": list(pr["n"]), "per_step_energy": per_step_energy},
           "wall_s": wall, "gpu_launches": K * (3 if per_step_energy else 1)}
    if per_step_energy:
        out["energy_non_increasing"] = bool(np.all(np.diff(F) <= 1e-12 * abs(F[0])))
        out["steps_per_s"] = K / wall
        out["config"]["path"] = "pf_step_energies: a step and the F_h reduction per step on the device, read back once"
    if per_step_energy and full:
        # the same run as one persistent launch that records F_h on the device
        from paper_2303_09671_gb300 import pf
        n = int(pr["n"][0])
        spl = max(1, K // 4)
        pf.run_batch(pr, [n], [0.0], phi, cs, cl, precision=prec, dt=[pr["dt"]], max_steps=spl,
                     steps_per_launch=spl, launches_per_graph=1, check_every=spl, tol=-1.0,
                     energy_every=1)                                     # warm-up
        t0 = time.perf_counter()
        res = pf.run_batch(pr, [n], [0.0], phi, cs, cl, precision=prec, dt=[pr["dt"]], max_steps=K,
                           steps_per_launch=spl, launches_per_graph=4, check_every=K, tol=-1.0,
                           energy_every=1)
        pwall = time.perf_counter() - t0
        E = res["energy"][0]
        # one SM's FP64 units bound the single CTA (GB300's FP64 rate is a small
        # fraction of its FP32 rate), so the per-call path over many SMs stays the value
        out["persistent"] = {"cell_updates_per_s": cells * K / (res["gpu_ms"] * 1e-3),
                             "ms_per_step": res["gpu_ms"] / K, "wall_s": pwall,
                             "launches": int(res["launches"]),
                             "energy_non_increasing": bool(np.all(np.diff(E) <= 1e-12 * abs(E[0]))),
                             "path": "one persistent shared-memory CTA recording F_h on the device "
                                     "every step (pf_run_batch, energy_every = 1)"}
        out["per_call"] = per_call
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--size", type=int, default=256)
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--calibrate", type=int, default=0,
                    help="adjoint workload: Adam iterations of the k(V) calibration after the timing")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="leave out the bounded kv_sweep, adjoint, planar1d and perturbed2d keys of the default line")
    ap.add_argument("--workload", default="sphere3d",
                    choices=["sphere3d", "kv-sweep", "adjoint", "planar1d", "perturbed2d", "banding",
                             "calibrate-steady"])
    ap.add_argument("--to-steady", action="store_true",
                    help="kv-sweep workload: run every front to steady state (or 2e6 steps) instead of a fixed budget")
    ap.add_argument("--mode", default="slabs", choices=["slabs", "replicas"],
                    help="N > 1: one grid cut into z-slabs with a halo exchange every step (strong "
                         "scaling), or one independent grid per rank (weak scaling)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.workload == "kv-sweep":
        return run_kv_sweep(args)
    if args.workload == "adjoint":
        return run_adjoint(args)
    if args.workload in ("planar1d", "perturbed2d"):
        return run_secondary(args)
    if args.workload == "banding":
        return run_banding(args)
    if args.workload == "calibrate-steady":
        return run_calibrate_steady(args)
    if args.impl == "reference":
        return run_reference(args)

    import torch
    from paper_2303_09671_gb300.pf import Sim

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import datetime
        import torch.distributed as dist
        # a bounded timeout: a rank that stops answering ends the run with an
        # error instead of holding every GPU
        dist.init_process_group("nccl", init_method="env://", timeout=datetime.timedelta(seconds=300))
        if args.mode == "slabs":
            return run_slabs(args, torch, dist, world, rank, local)

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    n = args.size
    pr, phi, cs, cl = workload(n)
    cells = int(np.prod(pr["n"]))
    f32 = [np.ascontiguousarray(a, dtype=np.float32) for a in (phi, cs, cl)]
    stream = torch.cuda.Stream()
    with torch.cuda.stream(stream):
        sim = Sim(pr, "fp32", stream=stream.cuda_stream)
        sim.set_fields(*f32)
        S0 = sim.solute_total()
        for _ in range(args.warmup):
            sim.step(1)
        barrier()
        stream.synchronize()
        ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        with ClockSampler(local) as clk:
            ev0.record(stream)
            for _ in range(args.steps):
                sim.step(1)
            ev1.record(stream)
            ev1.synchronize()
        barrier()
        ms = ev0.elapsed_time(ev1)
        S1 = sim.solute_total()
        drift = abs(S1 - S0) / abs(S0)

        # end to end through the public API with host buffers: every step uploads
        # the state (phi, c_s, c_l) from pinned host memory, steps, and reads the
        # stepped fields back into pinned host memory
        pinned = [torch.from_numpy(a).pin_memory() for a in f32]
        host_views = [p.numpy() for p in pinned]
        # two sets of page-locked result arrays, used in turn: each step's
        # read-back is queued without a wait and overlaps the next upload
        back = [[torch.empty(a.shape, dtype=torch.float32).pin_memory().numpy() for a in f32] for _ in range(2)]
        ke = max(1, args.e2e_steps)
        barrier()
        t0 = time.perf_counter()
        for i in range(ke):
            # upload overlapped with the step; the inputs stay unchanged, so the
            # call need not wait for its copies (the next one is queued at once)
            sim.set_fields_step(*host_views, n=1, wait=False)
            sim.get_fields_async(out_host=back[i % 2])     # the stepped fields, to the host
        sim.sync()
        e2e_s = time.perf_counter() - t0
        if not all(np.isfinite(b).all() for bb in back for b in bb):
            raise RuntimeError("non-finite field in the end-to-end leg")
        # the same with only the solute total read back (8 bytes a step), each
        # result queued into page-locked memory so that the next upload is
        # queued without a host stall
        results = torch.zeros(ke, dtype=torch.float64).pin_memory().numpy()
        barrier()
        t0 = time.perf_counter()
        for i in range(ke):
            sim.set_fields_step(*host_views, n=1)
            sim.solute_total_async(results, i)
        stream.synchronize()
        e2e_solute_s = time.perf_counter() - t0
        if not np.isfinite(results).all():
            raise RuntimeError("non-finite solute total in the end-to-end leg")
        sim.close()

    ms_max, e2e_max, e2e_sol_max = max_over_ranks([ms, e2e_s, e2e_solute_s], dist, device="cuda")
    value = weak_scaling_rate(cells, args.steps, world, ms_max * 1e-3)
    e2e_value = weak_scaling_rate(cells, ke, world, e2e_max)
    e2e_sol_value = weak_scaling_rate(cells, ke, world, e2e_sol_max)

    if rank == 0:
        hbm_peak, sm_mhz, how = load_peaks()
        sms = sm_count(local)
        launch_s = ms / args.steps * 1e-3
        achieved_gbs = BYTES_PER_CELL_UPDATE * cells / launch_s / 1e9
        # FP32 FMA-pipe peak: every lane issuing one FMA (2 operations) per clock;
        # the reciprocals and logarithms run beside it on the MUFU
        alu_peak = sms * FP32_LANES * 2 * sm_mhz * 1e6 / 1e12
        achieved_tops = FMA_OPS_PER_CELL_UPDATE * cells / launch_s / 1e12
        mufu_peak = sms * MUFU_LANES * sm_mhz * 1e6 / 1e12
        mufu_achieved = MUFU_PER_CELL_UPDATE * cells / launch_s / 1e12
        traffic = step3d_traffic(cells)
        cap = TRAFFIC_CAPTURE["captured_grid"]
        traffic_note = ("kernel sources changed since the capture" if traffic is None else
                        f"ncu DRAM bytes of one launch at {cap}^3" +
                        ("" if cap == n else f", scaled by cells to {n}^3"))
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": config(n, {"parallelism": f"independent grid per GPU x{world}"}),
            "roofline": {"bound": "alu", "achieved": achieved_tops, "peak": alu_peak,
                         "unit": "TFLOP/s", "frac": achieved_tops / alu_peak, "traffic": traffic,
                         "traffic_note": traffic_note,
                         "peak_source": f"derived: {sms} SMs x {FP32_LANES} FP32 lanes x 2 x {sm_mhz:.0f} MHz",
                         "kernel": "step3d_kernel<float,32,16,19-point>",
                         "ops_per_cell_update": FMA_OPS_PER_CELL_UPDATE,
                         "ops_note": (f"{OPS_PER_CELL_UPDATE} algorithmic FP32 operations per cell-update, "
                                      f"of which {MUFU_PER_CELL_UPDATE} reciprocals/logarithms run on the MUFU "
                                      "(see mufu) and the rest on the FMA pipe"),
                         "mufu": {"ops_per_cell_update": MUFU_PER_CELL_UPDATE, "achieved": mufu_achieved,
                                  "peak": mufu_peak, "frac": mufu_achieved / mufu_peak, "unit": "Top/s",
                                  "peak_source": f"derived: {sms} SMs x {MUFU_LANES} MUFU results x {sm_mhz:.0f} MHz"}},
            "roofline_hbm": {"bound": "hbm", "achieved": achieved_gbs, "peak": hbm_peak, "unit": "GB/s",
                             "frac": achieved_gbs / hbm_peak, "peak_source": how,
                             "bytes_per_cell_update": BYTES_PER_CELL_UPDATE},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * cells,
                    "d2h_bytes_per_step": 3 * 4 * cells, "steps": ke,
                    "path": "pf_set_fields_step (copy-engine upload overlapped with the step) + pf_get_fields_async "
                            "to pinned host memory (copy-engine read-back overlapped with the next upload)"},
            "e2e_solute_only": {"value": e2e_sol_value, "unit": UNIT, "h2d_bytes_per_step": 3 * 4 * cells,
                                "d2h_bytes_per_step": 8, "steps": ke,
                                "path": "pf_set_fields_step + pf_solute_total_async (8-byte result per step)"},
            "gpu_launches": args.steps,
            "solute_drift": drift,
            "clocks": clk.summary(),
        }
        if world == 1 and not args.no_secondary:
            out["kv_sweep"] = kv_brief()
            out["adjoint"] = adjoint_brief()
            out["planar1d"] = secondary_brief("planar1d", 20000)        # the 1D configuration, as stated
            out["perturbed2d"] = secondary_brief("perturbed2d", 10000)  # the 2D configuration, as stated
        if world == 1 and not args.no_cpu_baseline:
            out["cpu_baseline"] = cpu_baseline(n)
        print(json.dumps(out), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
