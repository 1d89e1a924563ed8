"""Benchmark: triangle-stage updates/s of the compact two-layer GKS on GB300.

Workload (one GPU): precision/balance configuration at full size -- a jittered
1024 x 1024-square mesh of the unit square (2,097,152 triangles, walls), a
Gaussian bump b = 0.5 exp(-50 r^2), flat interface (h1 + b = 0.8) and flat
upper layer (h2 = 0.2), zero velocity, chi = 0.98, CFL 0.5. One benchmark step
is one S2O4 time step (two stages) over the whole mesh, i.e. every part of the
hot path: CFL step, reconstruction, interface levels, edge solution, sources,
update and gradients.

`value` is the FP32 form (FP64 for the balance terms and sums) with the
learned troubled-cell gate, trained first on this GPU from the solver's own
seeded runs; the plain FP32 form and the plain FP64 GPU form of the same
workload are reported beside it, with the L1 differences to the FP64 form
after the timed runs and on the smooth periodic case.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun (N > 1) every rank runs its own replica of the workload (the
mesh is not partitioned: replicas only); value = all ranks' triangle-stages /
max time over ranks.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2306_04467_gb300 import replicas  # noqa: E402  (host helpers only; no GPU work at import)
from paper_2306_04467_gb300.replicas import dist_env  # noqa: E402

METRIC = "triangle-stage updates/s vs plain FP64 GPU at stated L1 error; % roofline"
UNIT = "triangle-stage updates/s"
N_SQ = 1024

# Per-unit work of each kernel: (FP32 flops, FP64 flops, algorithmic DRAM
# bytes). Flops are the hardware counts (sm__sass_thread_inst_executed_op_
# {f,d}{add,mul,fma}[2] with FMA = 2 flops) of the launches of one step of the
# benchmark workload at 512 x 512 squares (524,288 cells, 787,456 edges), per
# unit; the FP32-form reconstruction count is the gated one on this workload
# (every tile smooth). Bytes are the minimum one launch must move with the
# structure-of-arrays layout, each cell or edge record read or written once
# (reconstruction: operators 9x17 + 7 + stencil 9 + gathers + two 36-value
# side records out, without the P1 and smoothness rows for gated tiles; gate:
# 3 neighbour ids and transforms, eta1/h2 values and gradients, scales;
# interface: edge geometry, both cells' side records, two levels out; edge:
# the same plus plane rows and blend weights, 24 interface values out;
# edge_fused (the gated runs' interface levels and edge solution in one
# kernel): the edge kernel's bytes without the plane rows, which the gate
# makes unnecessary on this workload, plus the two levels out and the depth
# fluxes in FP64 in place of R;
# update: three edges' fluxes and interface values, state in/out with the
# S2O4 snapshot, mirrors out). Units: cells for recon, gate and update, edges for iface, edge and
# edge_fused.
WORK_PER_UNIT = {
    "fp32": {"recon": (2196, 0, 1069), "gate": (257, 0, 51), "iface": (836, 0, 265), "edge": (5405, 0, 374),
             "edge_fused": (5719, 0, 366), "update": (317, 45, 564)},
    "fp64": {"recon": (69, 4593, 2209), "gate": (280, 0, 63), "iface": (15, 1349, 473), "edge": (107, 9162, 696),
             "update": (0, 343, 850)},
}
# Measured FMA-chain peaks of this GB300 pool (TFLOP/s, 2 flops per FMA).
PEAK_TFLOPS = {"fp32": 76.5, "fp64": 1.254}
# DRAM bytes per unit (dram__bytes_read.sum + dram__bytes_write.sum of the
# same launches, per unit; inputs larger than L2, traffic grows with units).
TRAFFIC_PER_UNIT = {"fp32": {"recon": 1027.0, "gate": 51.0, "iface": 259.0, "edge": 327.0, "edge_fused": 359.0,
                             "update": 445.0}}


KERNEL_NAME = {"edge_fused": "k_edgef", "edge_deferred": "k_edge_deferred"}


def roofline(form, kernel, units, ms, hbm_gbs):
    """Binding limit of one kernel launch: the slowest of its FP32 work at the
    FP32 peak, its FP64 work at the FP64 peak and its algorithmic bytes at the
    measured HBM bandwidth; achieved is that resource's rate in this launch."""
    f32, f64, by = WORK_PER_UNIT[form][kernel]
    t = ms * 1e-3
    limits = {"fp32": f32 * units / (PEAK_TFLOPS["fp32"] * 1e12),
              "fp64": f64 * units / (PEAK_TFLOPS["fp64"] * 1e12),
              "hbm": by * units / (hbm_gbs * 1e9)}
    bind = max(limits, key=limits.get)
    if bind == "hbm":
        return {"bound": "hbm", "kernel": KERNEL_NAME.get(kernel, "k_" + kernel), "achieved": by * units / t / 1e9, "peak": hbm_gbs,
                "unit": "GB/s", "frac": limits[bind] / t, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    work = f32 if bind == "fp32" else f64
    return {"bound": "alu", "pipe": bind, "kernel": KERNEL_NAME.get(kernel, "k_" + kernel), "achieved": work * units / t / 1e12,
            "peak": PEAK_TFLOPS[bind], "unit": "TFLOP/s", "frac": limits[bind] / t,
            "peak_source": "measured %s FMA-chain peak (gks2l_alu_peaks, same run)" % bind.upper()}


def read_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except OSError:
        return {}


class ClockSampler:
    """nvidia-smi clock/throttle samples every 50 ms while a region runs."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index=0):
        self.index = index
        self.samples = []
        self._p = None

    def __enter__(self):
        try:
            self._p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + self.Q,
                                        "--format=csv,noheader,nounits", "-lms", "50"],
                                       stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)   # let the first sample land before the timed region
        except OSError:
            self._p = None
        return self

    def __exit__(self, *a):
        if self._p is None:
            return
        time.sleep(0.1)
        self._p.terminate()
        try:
            out, _ = self._p.communicate(timeout=5)
        except subprocess.TimeoutExpired:
            self._p.kill()
            out, _ = self._p.communicate()
        self.samples = [[x.strip() for x in line.split(",")] for line in out.splitlines() if line.strip()]

    def summary(self):
        rows = [r for r in self.samples if len(r) >= 9]
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no nvidia-smi samples"], "samples": 0}

        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [v for v in (num(r[1]) for r in rows) if v is not None]
        mx = [v for v in (num(r[2]) for r in rows) if v is not None]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].strip().lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def oracle_rate(seconds_budget=15.0, n=48, stages_per_step=2, max_steps=None):
    """The FP64 CPU oracle on a bounded sample of the same workload: the same
    problem on an n x n-square mesh; returns (triangle-stages/s, description)."""
    from oracle.oracle import Oracle
    from paper_2306_04467_gb300 import inputs
    prob = inputs.lake_at_rest(n, chi=0.98)
    o = Oracle.from_problem(prob)
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.advance(stages_per_step)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget or (max_steps and steps >= max_steps):
            break
    rate = prob.mesh.n_tri * stages_per_step * steps / el
    desc = "oracle (serial FP64 C, 1 thread) on the same workload at %dx%d squares (%d triangles), %d steps, %.1f s" % (
        n, n, prob.mesh.n_tri, steps, el)
    return rate, desc, steps, el


def run_reference(args):
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.oracle import Oracle
    from paper_2306_04467_gb300 import inputs
    n = 48
    prob = inputs.lake_at_rest(n, chi=0.98)
    o = Oracle.from_problem(prob)
    for _ in range(args.warmup):
        o.advance(2)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        o.advance(2)
    el = time.perf_counter() - t0
    rate = prob.mesh.n_tri * 2 * args.steps / el
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * el / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic (seeded jittered mesh, analytic initial data)",
        "config": {"workload": "lake at rest over a Gaussian bump, jittered %dx%d-square mesh of the unit "
                               "square (%d triangles; bounded sample of the 1024x1024 workload), walls, chi=0.98"
                               % (n, n, prob.mesh.n_tri), "l2": "working set below L2 (CPU run)"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d steps of 2 stages on %d triangles" % (args.steps, prob.mesh.n_tri)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_profile_case(args):
    from paper_2306_04467_gb300 import gks2l as g
    from paper_2306_04467_gb300 import inputs
    prob = inputs.lake_at_rest(args.profile_case, chi=0.98)
    prec = g.GKS2L_FP64 if args.form == "fp64" else g.GKS2L_FP32
    kw = {}
    if args.form == "fp32_learned":
        from paper_2306_04467_gb300 import gate
        P, _ = gate.default_gate()
        kw = dict(indicator=g.GKS2L_INDICATOR_MLP, indicator_threshold=gate.THRESHOLD)
    par = g.default_params(g=prob.g, chi=prob.chi, cfl=prob.cfl, precision=prec, **kw)
    s = g.Solver(prob.mesh, par, prob.b_vert)
    s.set_state(prob.avg, prob.grad)
    if kw:
        s.set_mlp(P)
        s.advance(2)   # the first stage after set_mlp is the plain method
    import torch
    torch.cuda.synchronize()
    torch.cuda.profiler.start()   # a profiler started with capture off records from here
    ms = s.profile_kernels(1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_case": args.profile_case, "form": args.form, "n_tri": prob.mesh.n_tri,
                      "kernel_ms": ms}))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=30)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_SQ, help="squares per side of the mesh")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="profiling mode: one step of the workload at this many squares per side, kernels "
                         "launched one by one (for ncu captures of a small case)")
    ap.add_argument("--form", default="fp32", choices=["fp32", "fp32_learned", "fp64"])
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.profile_case:
        return run_profile_case(args)

    import torch
    ws, rank, local = dist_env()
    if ws > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    from paper_2306_04467_gb300 import gks2l as g
    from paper_2306_04467_gb300 import inputs

    def barrier():
        if ws > 1:
            torch.distributed.barrier()

    def max_over_ranks(x):
        return x if ws == 1 else replicas.max_over_ranks(x, dev)

    # CPU baseline first (host cores, before any GPU work): rank 0 only
    cpu = None
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        rate, desc, _, _ = oracle_rate()
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    prob = inputs.lake_at_rest(args.n, chi=0.98)
    nt = prob.mesh.n_tri
    n_edges = (3 * nt + 2 * (prob.mesh.nx + prob.mesh.ny)) // 2
    stream = torch.cuda.Stream(device=dev)

    # the learned gate: harvested from the solver's own seeded runs and trained
    # on this GPU by the library's kernels (outside the timed region)
    from paper_2306_04467_gb300 import gate
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        gate_params, gate_q = gate.default_gate()
        torch.cuda.synchronize(dev)
        gate_train_s = time.perf_counter() - t0

    def solver(p, prec, learned):
        kw = dict(indicator=g.GKS2L_INDICATOR_MLP, indicator_threshold=gate.THRESHOLD) if learned else {}
        par = g.default_params(g=p.g, chi=p.chi, cfl=p.cfl, precision=prec, **kw)
        s = g.Solver(p.mesh, par, p.b_vert, device=dev, stream=stream)
        s.set_state(p.avg, p.grad)
        if learned:
            s.set_mlp(gate_params)
        return s

    forms = (("fp32_learned", g.GKS2L_FP32, True), ("fp32", g.GKS2L_FP32, False), ("fp64", g.GKS2L_FP64, False))
    results = {}
    live_peaks = None
    for form, prec, learned in forms:
        with torch.cuda.stream(stream):
            s = solver(prob, prec, learned)
            shapes = s.autotune(1)
            steps = args.steps if prec == g.GKS2L_FP32 else max(2, args.steps // 4)
            s.advance(2 * args.warmup)
            torch.cuda.synchronize(dev)
            barrier()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            sampler = ClockSampler(local)
            with sampler:
                torch.cuda.synchronize(dev)
                if form == "fp32_learned":
                    torch.cuda.profiler.start()   # a profiler started with capture off records the timed region
                e0.record(stream)
                s.advance(2 * steps, sync=False)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                if form == "fp32_learned":
                    torch.cuda.profiler.stop()
            barrier()
            ms = e0.elapsed_time(e1) / steps
            ms = max_over_ranks(ms)
            st = s.stats()
            if st["status"] != 0:
                raise RuntimeError("device status %d after the timed run" % st["status"])
            a, _ = s.get_state()
            kern = s.profile_kernels(2)
            if form == "fp32_learned":
                live_peaks = s.alu_peaks()
            results[form] = {"ms_per_step": ms, "steps": steps, "clocks": sampler.summary(), "kernels": kern,
                             "state": a, "workspace": s.workspace_bytes, "shapes": shapes,
                             "smooth_fraction": st["smooth_fraction"]}
            # end to end through the C ABI with host (pinned) buffers
            if form == "fp32_learned":
                ha = torch.empty(6 * nt, dtype=torch.float64).pin_memory()
                hg = torch.empty(12 * nt, dtype=torch.float64).pin_memory()
                ha.copy_(torch.from_numpy(np.ascontiguousarray(prob.avg).ravel()))
                hg.copy_(torch.from_numpy(np.ascontiguousarray(prob.grad).ravel()))
                n_e2e = max(2, steps // 2)
                torch.cuda.synchronize(dev)
                t0 = time.perf_counter()
                for _ in range(n_e2e):
                    s.set_state_host_ptr(ha.data_ptr(), hg.data_ptr())
                    s.advance(2, sync=False)
                    s.get_state_host_ptr(ha.data_ptr(), hg.data_ptr())
                torch.cuda.synchronize(dev)
                el = max_over_ranks(time.perf_counter() - t0)
                results[form]["e2e"] = {"value": ws * nt * 2 * n_e2e / el, "unit": UNIT,
                                        "h2d_bytes_per_step": 18 * 8 * nt, "d2h_bytes_per_step": 18 * 8 * nt}
            del s
            torch.cuda.empty_cache()

    def l1_rel(p, a, b):
        P = p.mesh.xy[p.mesh.tri]
        area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                            (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
        return max(float(np.sum(area * np.abs(a[v] - b[v])) / np.sum(area * np.abs(b[v]))) for v in (0, 3))

    l1 = {f: l1_rel(prob, results[f]["state"], results["fp64"]["state"]) for f in ("fp32_learned", "fp32")}
    # the stated error on a case that moves: the smooth periodic case (512
    # triangles, 100 stages), each FP32 form against the plain FP64 GPU form
    smooth = inputs.smooth_periodic(16)
    with torch.cuda.stream(stream):
        ref = solver(smooth, g.GKS2L_FP64, False)
        ref.advance(100)
        a64, _ = ref.get_state()
        l1_smooth = {}
        for form, prec, learned in forms[:2]:
            s = solver(smooth, prec, learned)
            s.advance(100)
            l1_smooth[form] = l1_rel(smooth, s.get_state()[0], a64)
            if learned:
                l1_smooth["smooth_fraction"] = s.stats()["smooth_fraction"]

    rh = results["fp32_learned"]
    value = replicas.job_rate(nt * 2, rh["ms_per_step"], ws)
    rates = {f: replicas.job_rate(nt * 2, results[f]["ms_per_step"], ws) for f in results}
    # roofline of the dominant kernel of the headline form
    # with the gate the interface levels and the edge solution run as one fused
    # kernel (the library reports it in the edge slot) followed by a pass over
    # the edges whose solution needs the plane gradients (the interface slot)
    k = rh["kernels"]
    kern = {"recon": k["recon"], "edge_fused": k["edge"], "edge_deferred": k["iface"], "update": k["update"],
            "step_begin": k["step_begin"], "gate": k["gate"]}
    names = ("recon", "edge_fused", "update")
    top = max(names, key=lambda x: kern[x])
    units = nt if top in ("recon", "update") else n_edges
    hbm = read_peaks().get("hbm_gbs", 6800.0)
    if live_peaks:
        PEAK_TFLOPS.update(live_peaks)
    roof = roofline("fp32", top, units, kern[top], hbm)
    tpu = TRAFFIC_PER_UNIT.get("fp32", {}).get(top)
    roof["traffic"] = tpu * units if tpu else None
    roof["per_kernel"] = {x: round(roofline("fp32", x, nt if x in ("recon", "gate", "update") else n_edges, kern[x],
                                             hbm)["frac"], 4) for x in names + ("gate",)}
    timed = names + ("edge_deferred", "gate")
    ksum = sum(kern[x] for x in timed)
    share = {x: kern[x] / ksum for x in timed}
    launches_per_step = 1 + 2 * 5   # step start + (reconstruction, gate, fused edge, deferred edges, update) per stage
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": rh["steps"],
        "warmup": args.warmup, "ms_per_step": rh["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64+bf16",
        "data": "synthetic (seeded jittered mesh, analytic initial data)",
        "config": {"workload": "precision/balance case: lake at rest over a Gaussian bump "
                               "b=0.5exp(-50r^2), h1+b=0.8, h2=0.2, u=0, chi=0.98, walls, jittered "
                               "%dx%d-square mesh (%d triangles), S2O4 step = 2 stages" % (args.n, args.n, nt),
                   "form": "FP32 moments/reconstruction with FP64 balance terms and sums, learned BF16 gate",
                   "l2": "inputs larger than L2 (operators and state %.1f GB)" % (rh["workspace"] / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "launch_shapes": rh["shapes"]},
        "forms": {f: {"value": rates[f], "ms_per_step": results[f]["ms_per_step"],
                      "l1_rel_vs_fp64_gpu": l1.get(f, 0.0)} for f in results},
        "speedup_over_fp64_gpu": value / rates["fp64"],
        "l1_rel_smooth_case_vs_fp64_gpu": l1_smooth,
        "gate": {"train_s": gate_train_s, "train_quality": gate_q, "smooth_fraction": rh["smooth_fraction"],
                 "threshold": gate.THRESHOLD},
        "kernel_ms": {k: round(v, 4) for k, v in kern.items()},
        "kernel_share": {k: round(v, 4) for k, v in share.items()},
        "roofline": roof,
        "alu_peaks_tflops": live_peaks,
        "clocks": rh["clocks"],
        "e2e": rh["e2e"],
        "gpu_launches": launches_per_step * rh["steps"],
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
