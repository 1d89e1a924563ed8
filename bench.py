"""Benchmark: triangle-stage updates/s of the compact two-layer GKS on GB300.

Headline workload (one GPU): the large configuration -- an internal wave over
a ridge on a jittered 5656 x 707-square mesh of [0, 8] x [0, 1] (7,997,584
triangles, walls), b = 0.3 exp(-20 (x - 4)^2), interface 0.7 - 0.1 exp(-20
(x - 1)^2), free surface 1, zero velocity, chi = 0.97, CFL 0.5, a run of 2000
stages of which a window from its start is timed. One benchmark step is one
S2O4 time step (two stages) over the whole mesh: every part of the hot path
(CFL step, reconstruction, interface levels, edge solution, sources, update
and gradients).

`value` is the FP32 form (FP64 for the balance terms and sums) with the
learned troubled-cell gate, trained first on this GPU from the solver's own
seeded runs; the plain FP32 form and the plain FP64 GPU form of the same
workload are reported beside it, each with its L1 difference to the FP64 form
after the same number of stages from the same initial state. The learned
indicator's workload (interface dam break, 1,602,050 triangles) and the
precision workload (lake at rest, 2,097,152 triangles) follow as secondary
lines with the same three forms.

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

# The workloads: (generator, full-size arguments, description).
WORKLOADS = {
    "large": ("internal_wave_ridge", dict(nx=5656, ny=707),
              "large configuration: internal wave over a ridge, b=0.3exp(-20(x-4)^2), interface "
              "0.7-0.1exp(-20(x-1)^2), free surface 1, u=0, chi=0.97, walls, jittered %dx%d-square mesh of "
              "[0,8]x[0,1] (%d triangles), CFL 0.5, 2000-stage run timed over a window from its start"),
    "dambreak": ("interface_dambreak", dict(n=895),
                 "learned-indicator configuration: interface dam break (h1,h2)=(0.6,0.4)|(0.4,0.6), flat bottom, "
                 "u=0, chi=0.98, walls, jittered %dx%d-square mesh of [-1,1]^2 (%d triangles)"),
    "lake": ("lake_at_rest", dict(n=1024),
             "precision/balance configuration: lake at rest over a Gaussian bump b=0.5exp(-50r^2), h1+b=0.8, "
             "h2=0.2, u=0, chi=0.98, walls, jittered %dx%d-square mesh (%d triangles)"),
}


def make_workload(name, scale=1.0):
    """The workload's problem at full size (scale 1) or with the squares per
    side scaled down (a bounded sample of the same workload)."""
    from paper_2306_04467_gb300 import inputs
    gen, kw, _ = WORKLOADS[name]
    kw = {k: max(4, int(round(v * scale))) for k, v in kw.items()}
    if name == "lake":
        return getattr(inputs, gen)(kw["n"], chi=0.98)
    return getattr(inputs, gen)(**kw)


def describe(name, prob):
    return WORKLOADS[name][2] % (prob.mesh.nx, prob.mesh.ny, prob.mesh.n_tri)


# Algorithmic work per unit of each kernel: (FP32 flops, FP64 flops,
# algorithmic DRAM bytes) in the FP32 form; the FP64 form does the same flops
# in FP64. Flops follow the method's per-step operation counts (multiply-add
# = 2 flops; divisions, square roots and transcendentals are counted apart):
#   reconstruction, per cell: the P3 fit 918 MAC (6 variables x 9 x 17), the
#     three P1 fits 180 MAC, smoothness indicators and WENO weights 600 MAC;
#     a cell the gate calls smooth needs the P3 fit only;
#   edge solution, per edge: 2 Gauss points x 2 layers x 700 flops for the
#     gas-kinetic solution (half-space moments, slopes, force, A-bar, the five
#     moment sets, time integrals and fit) plus evaluating both cells'
#     polynomials (value and gradient, 6 variables) at the two points,
#     4 x 6 x 27 MAC;
#   interface levels, per edge: both sides' levels and discharges at two
#     points (4 x 3 x 10 MAC) and the blend, per layer;
#   update, per cell: 400 flops (three edges' residuals, sources, S2O4,
#     Gauss-theorem gradients);
#   gate, per cell: the feature construction (the network's 1.8k MAC run on
#     the BF16 tensor cores and are not counted here).
# Bytes are the minimum one launch moves with the structure-of-arrays layout,
# each cell or edge record read or written once (reconstruction: operators
# 9x17 + 7 + stencil 9 + gathers + two 36-value side records out, without the
# P1 and smoothness rows for gated tiles; gate: 3 neighbour ids and
# transforms, eta1/h2 values and gradients, scales; interface: edge geometry,
# both cells' side records, two levels out; edge: the same plus plane rows
# and blend weights, fluxes and time derivatives out, own levels out;
# edge_fused: the edge kernel's bytes without the plane rows plus the two
# levels out; update: three edges' fluxes, time derivatives, own levels and
# interface values, state in/out with the S2O4 snapshot, mirrors out). Units:
# cells for recon, gate and update, edges for iface, edge and edge_fused.
RECON_P3, RECON_REST = 2 * 918, 2 * (180 + 600)
EDGE_FLOPS = 4 * 700 + 2 * 4 * 6 * 27
IFACE_FLOPS = 2 * (2 * 4 * 3 * 10 + 20)
WORK_PER_UNIT = {
    "recon": (RECON_P3 + RECON_REST, 1069),
    "gate": (260, 51),
    "iface": (IFACE_FLOPS, 265),
    "edge": (EDGE_FLOPS, 374),
    "edge_fused": (EDGE_FLOPS, 366),
    "update": (400, 570),
}
# FP32 flops per unit that the hardware executes (ncu sm__sass_thread_inst_
# executed_op_f{add,mul,fma} with FMA = 2): reported beside the algorithmic
# counts as the overhead ratio. recon, gate, edge_fused, update: one step of
# the large configuration at 1416 x 177 squares (501,264 triangles), the
# current kernels; iface and edge (the plain form's): the lake at 512 x 512
# squares, captured before the edge kernels' last instruction cuts.
EXECUTED_FP32_PER_UNIT = {"recon": 2214, "gate": 258, "iface": 836, "edge": 5405, "edge_fused": 5500,
                          "update": 319}
# Measured FMA-chain peaks of this GB300 pool (TFLOP/s, 2 flops per FMA); the
# bench replaces them with the same run's own measurement.
PEAK_TFLOPS = {"fp32": 76.5, "fp64": 1.254}
# DRAM bytes per unit (dram__bytes_read.sum + dram__bytes_write.sum of the
# same launches, per unit, mean of the two stages) from an ncu capture of the
# current kernels on the large configuration at 1416 x 177 squares (inputs
# larger than L2); the bench scales them to its launch by the units. A kernel
# is listed only while it is unchanged since that capture.
TRAFFIC_PER_UNIT = {"recon": 1040.0, "gate": 59.1, "edge_fused": 362.5, "update": 461.3}


KERNEL_NAME = {"edge_fused": "k_edgef", "edge_deferred": "k_edge_deferred"}


def recon_flops(smooth_fraction):
    """Reconstruction flops per cell when a fraction of the cells take the
    linear weights (the gate's smooth cells skip the P1 fits and weights)."""
    return RECON_P3 + (1.0 - smooth_fraction) * RECON_REST


# the P1 candidate rows (30) and smoothness forms (45) of a cell, which only
# a cell with the nonlinear weights reads
RECON_LATE_BYTES = 4 * (30 + 45)


def recon_bytes(smooth_fraction):
    """Reconstruction bytes per cell when a fraction of the cells take the
    linear weights and so need neither their P1 rows nor smoothness forms."""
    return WORK_PER_UNIT["recon"][1] + (1.0 - smooth_fraction) * RECON_LATE_BYTES


def roofline(form, kernel, units, ms, hbm_gbs, smooth_fraction=0.0):
    """Binding limit of one kernel launch: the slower of its algorithmic
    flops at the form's pipe peak (FP32 or FP64 FMA chains) and its
    algorithmic bytes at the measured HBM bandwidth; achieved is that
    resource's rate in this launch."""
    fl, by = WORK_PER_UNIT[kernel]
    if kernel == "recon":
        fl, by = recon_flops(smooth_fraction), recon_bytes(smooth_fraction)
    pipe = "fp64" if form == "fp64" else "fp32"
    if form == "fp64":
        by = 2 * by   # every R-typed record is a double
    t = ms * 1e-3
    limits = {pipe: fl * units / (PEAK_TFLOPS[pipe] * 1e12), "hbm": by * units / (hbm_gbs * 1e9)}
    bind = max(limits, key=limits.get)
    name = KERNEL_NAME.get(kernel, "k_" + kernel)
    if bind == "hbm":
        return {"bound": "hbm", "kernel": name, "achieved": by * units / t / 1e9, "peak": hbm_gbs,
                "unit": "GB/s", "frac": limits[bind] / t, "peak_source": "measured (MEASURED_PEAKS.json hbm_gbs)"}
    return {"bound": "alu", "pipe": pipe, "kernel": name, "achieved": fl * units / t / 1e12,
            "peak": PEAK_TFLOPS[pipe], "unit": "TFLOP/s", "frac": limits[bind] / t,
            "peak_source": "measured %s FMA-chain peak (gks2l_alu_peaks, same run)" % pipe.upper()}


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


SAMPLE_SCALE = {"large": 16 / 707, "dambreak": 48 / 895, "lake": 48 / 1024}


def oracle_rate(workload="large", seconds_budget=15.0, stages_per_step=2):
    """The FP64 CPU oracle, as it stands, on a bounded sample of the workload
    (the same problem on a mesh with fewer squares per side); returns
    (triangle-stages/s, description)."""
    from oracle.oracle import Oracle
    prob = make_workload(workload, SAMPLE_SCALE[workload])
    o = Oracle.from_problem(prob)
    t0 = time.perf_counter()
    steps = 0
    while True:
        o.advance(stages_per_step)
        steps += 1
        el = time.perf_counter() - t0
        if el >= seconds_budget:
            break
    rate = prob.mesh.n_tri * stages_per_step * steps / el
    desc = ("oracle (serial FP64 C, 1 thread) on a bounded sample of the same workload: %dx%d squares "
            "(%d triangles), %d steps of 2 stages, %.1f s" % (prob.mesh.nx, prob.mesh.ny, prob.mesh.n_tri, steps, el))
    return rate, desc


def run_reference(args):
    """The reference arm: the FP64 CPU oracle as it stands, timed on the host
    cores on a bounded sample of the headline workload (rank 0 only)."""
    ws, rank, _ = dist_env()
    if rank != 0:
        return
    from oracle.oracle import Oracle
    prob = make_workload(args.workload, SAMPLE_SCALE[args.workload])
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
        "config": {"workload": describe(args.workload, prob) + " (bounded sample of the full-size workload)",
                   "l2": "working set below L2 (CPU run)"},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": "%d steps of 2 stages on %d triangles" % (args.steps, prob.mesh.n_tri)},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def run_profile_case(args):
    """One step of the workload at a reduced size (the squares across the
    workload's short side), the kernels launched one by one between
    cudaProfilerStart/Stop: the small case for ncu captures."""
    from paper_2306_04467_gb300 import gks2l as g
    full = WORKLOADS[args.workload][1]
    prob = make_workload(args.workload, args.profile_case / min(full.values()))
    prec = g.GKS2L_FP64 if args.form == "fp64" else g.GKS2L_FP32
    kw = {}
    if args.form == "fp32_learned":
        from paper_2306_04467_gb300 import gate
        P, _ = gate.default_gate()
        kw = dict(indicator=g.GKS2L_INDICATOR_MLP, indicator_threshold=gate.THRESHOLD)
    par = g.default_params(g=prob.g, chi=prob.chi, cfl=prob.cfl, precision=prec, **kw)
    s = g.Solver(prob.mesh, par, prob.b_vert)
    s.set_state(prob.avg, prob.grad)
    s.set_launch_shapes([1, 1, 1, args.gate_variant])
    if kw:
        s.set_mlp(P)
        s.advance(2)   # the first stage after set_mlp is the plain method
    import torch
    torch.cuda.synchronize()
    torch.cuda.profiler.start()   # a profiler started with capture off records from here
    ms = s.profile_kernels(1)
    torch.cuda.synchronize()
    torch.cuda.profiler.stop()
    print(json.dumps({"profile_case": args.profile_case, "workload": args.workload, "form": args.form,
                      "gate_variant": args.gate_variant,
                      "n_tri": prob.mesh.n_tri, "n_edges": n_edges(prob), "kernel_ms": ms}))


def n_edges(prob):
    """Edges of a walled or periodic N_x x N_y-square mesh."""
    m = prob.mesh
    if m.period[0] > 0:
        return 3 * m.n_tri // 2
    return (3 * m.n_tri + 2 * (m.nx + m.ny)) // 2


def l1_rel(p, a, b):
    """Reading R12's relative L1 difference, the larger over the two depths."""
    P = p.mesh.xy[p.mesh.tri]
    area = 0.5 * np.abs((P[:, 1, 0] - P[:, 0, 0]) * (P[:, 2, 1] - P[:, 0, 1]) -
                        (P[:, 1, 1] - P[:, 0, 1]) * (P[:, 2, 0] - P[:, 0, 0]))
    return max(float(np.sum(area * np.abs(a[v] - b[v])) / np.sum(area * np.abs(b[v]))) for v in (0, 3))


FORMS = (("fp32_learned", True), ("fp32", False), ("fp64", False))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="large", choices=sorted(WORKLOADS))
    ap.add_argument("--secondary", default="dambreak,lake,ensemble",
                    help="comma-separated workloads measured after the headline one ('' for none)")
    ap.add_argument("--repeats", type=int, default=3,
                    help="extra timed blocks of K steps of the headline form (reported beside the value)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--profile-case", type=int, default=0,
                    help="profiling mode: one step of the workload with this many squares across its short "
                         "side, kernels launched one by one (for ncu captures of a small case)")
    ap.add_argument("--form", default="fp32_learned", choices=["fp32", "fp32_learned", "fp64"])
    ap.add_argument("--gate-variant", type=int, default=0, choices=list(range(16)),
                    help="profiling mode: the gate kernel (variant %% 4; 0: mma.sync warp tiles, 1: tcgen05 "
                         "CTA tiles, 2 and 3: tcgen05 with two and four times the blocks per SM), its placement "
                         "(variant / 4 %% 2; beside the edge kernels or the reconstruction) and the gated run's "
                         "edge path (variant / 8; the fused pass or the plain interface and edge kernels)")
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
        rate, desc = oracle_rate(args.workload)
        cpu = {"value": rate, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc}

    stream = torch.cuda.Stream(device=dev)

    # the learned gate: harvested from the solver's own seeded runs and trained
    # on this GPU by the library's kernels (outside the timed region)
    from paper_2306_04467_gb300 import gate
    with torch.cuda.stream(stream):
        t0 = time.perf_counter()
        gate_params, gate_q = gate.default_gate()
        torch.cuda.synchronize(dev)
        gate_train_s = time.perf_counter() - t0

    def solver(p, form):
        prec = g.GKS2L_FP64 if form == "fp64" else g.GKS2L_FP32
        learned = form == "fp32_learned"
        kw = dict(indicator=g.GKS2L_INDICATOR_MLP, indicator_threshold=gate.THRESHOLD) if learned else {}
        par = g.default_params(g=p.g, chi=p.chi, cfl=p.cfl, precision=prec, **kw)
        s = g.Solver(p.mesh, par, p.b_vert, device=dev, stream=stream)
        s.set_state(p.avg, p.grad)
        if learned:
            s.set_mlp(gate_params)
        return s

    hbm = read_peaks().get("hbm_gbs", 6800.0)
    live_peaks = None

    def measure(name, headline):
        """All three forms of one workload: each autotuned, restarted from the
        initial state, W warm-up steps, K timed steps (FP64: fewer, then
        untimed steps up to the same count), its state after 2 (W + K)
        stages compared with the FP64 form's."""
        nonlocal live_peaks
        prob = make_workload(name)
        nt, ne = prob.mesh.n_tri, n_edges(prob)
        K, W = args.steps, args.warmup
        res = {}
        for form, learned in FORMS:
            with torch.cuda.stream(stream):
                s = solver(prob, form)
                shapes = s.autotune(1)
                s.set_state(prob.avg, prob.grad)
                k_form = K if form != "fp64" else max(2, K // 4)
                s.advance(2 * W)
                torch.cuda.synchronize(dev)
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                sampler = ClockSampler(local)
                reps = []
                with sampler:
                    torch.cuda.synchronize(dev)
                    if headline and form == "fp32_learned":
                        # a profiler started with capture off records the timed region
                        torch.cuda.profiler.start()
                    e0.record(stream)
                    s.advance(2 * k_form, sync=False)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    if headline and form == "fp32_learned":
                        torch.cuda.profiler.stop()
                    if headline and form == "fp32_learned":
                        # extra blocks of K steps, beside the value: the clock
                        # record covers them all (the state keeps advancing)
                        for _ in range(args.repeats):
                            r0 = torch.cuda.Event(enable_timing=True)
                            r1 = torch.cuda.Event(enable_timing=True)
                            r0.record(stream)
                            s.advance(2 * K, sync=False)
                            r1.record(stream)
                            torch.cuda.synchronize(dev)
                            reps.append(r0.elapsed_time(r1) / K)
                barrier()
                ms = max_over_ranks(e0.elapsed_time(e1) / k_form)
                st = s.stats()
                if st["status"] != 0:
                    raise RuntimeError("device status %d after the timed run (%s, %s)" % (st["status"], name, form))
                if reps:
                    # the comparison state: the same 2 (W + K) stages as the others
                    s.set_state(prob.avg, prob.grad)
                    s.advance(2 * (W + K))
                elif k_form < K:
                    s.advance(2 * (K - k_form))
                smooth = s.stats()["smooth_fraction"]
                a, _ = s.get_state()
                kern = s.profile_kernels(2)
                if headline and form == "fp32_learned":
                    live_peaks = s.alu_peaks()
                    PEAK_TFLOPS.update(live_peaks)
                res[form] = {"ms_per_step": ms, "steps": k_form, "clocks": sampler.summary(), "kernels": kern,
                             "state": a, "workspace": s.workspace_bytes, "shapes": shapes,
                             "smooth_fraction": smooth, "stages_compared": 2 * (W + K)}
                if reps:
                    res[form]["repeat_ms_per_step"] = reps
                # end to end through the C ABI with host (pinned) buffers
                if headline and form == "fp32_learned":
                    ha = torch.empty(6 * nt, dtype=torch.float64).pin_memory()
                    hg = torch.empty(12 * nt, dtype=torch.float64).pin_memory()
                    ha.copy_(torch.from_numpy(np.ascontiguousarray(prob.avg).ravel()))
                    hg.copy_(torch.from_numpy(np.ascontiguousarray(prob.grad).ravel()))
                    oa = torch.empty(6 * nt, dtype=torch.float64).pin_memory()
                    og = torch.empty(12 * nt, dtype=torch.float64).pin_memory()
                    n_e2e = K
                    io_bytes = {"h2d_bytes_per_step": 18 * 8 * nt, "d2h_bytes_per_step": 18 * 8 * nt}
                    # each step: the state in from pinned host memory, two
                    # stages, the state out, as one pipelined call over the
                    # steps (a step's copies overlap its neighbours' stages;
                    # the first call makes the staging buffers, untimed)
                    s.run_items([(ha, hg)], [(oa, og)], 2)
                    torch.cuda.synchronize(dev)
                    t0 = time.perf_counter()
                    s.run_items([(ha, hg)] * n_e2e, [(oa, og)] * n_e2e, 2)
                    torch.cuda.synchronize(dev)
                    el = max_over_ranks(time.perf_counter() - t0)
                    res[form]["e2e"] = dict({"value": ws * nt * 2 * n_e2e / el, "unit": UNIT,
                                             "api": "gks2l_run_items (pipelined host I/O)"}, **io_bytes)
                    # the same steps one call at a time: set_state, advance, get_state
                    t0 = time.perf_counter()
                    for _ in range(n_e2e):
                        s.set_state_host_ptr(ha.data_ptr(), hg.data_ptr())
                        s.advance(2, sync=False)
                        s.get_state_host_ptr(oa.data_ptr(), og.data_ptr())
                    torch.cuda.synchronize(dev)
                    el = max_over_ranks(time.perf_counter() - t0)
                    res[form]["e2e_sequential"] = dict({"value": ws * nt * 2 * n_e2e / el, "unit": UNIT,
                                                        "api": "gks2l_set_state, gks2l_advance, gks2l_get_state"},
                                                       **io_bytes)
                del s
                torch.cuda.empty_cache()
        out = {"workload": describe(name, prob), "n_tri": nt, "n_edges": ne, "forms": {}}
        for form, _ in FORMS:
            r = res[form]
            k = r["kernels"]
            sf = r["smooth_fraction"] if form == "fp32_learned" else 0.0
            if form == "fp32_learned" and r["shapes"][3] < 8:
                kern = {"recon": k["recon"], "edge_fused": k["edge"], "edge_deferred": k["iface"],
                        "update": k["update"], "gate": k["gate"], "step_begin": k["step_begin"]}
                names = ("recon", "edge_fused", "update")
            else:
                # the plain forms, and a gated run on the plain edge path
                kern = {"recon": k["recon"], "iface": k["iface"], "edge": k["edge"], "update": k["update"],
                        "step_begin": k["step_begin"]}
                if form == "fp32_learned":
                    kern["gate"] = k["gate"]
                names = ("recon", "iface", "edge", "update")
            units = {x: (nt if x in ("recon", "update", "gate") else ne) for x in kern}
            per = {x: roofline(form, x, units[x], kern[x], hbm, sf) for x in names}
            top = max(names, key=lambda x: kern[x])
            out["forms"][form] = {
                "value": replicas.job_rate(nt * 2, r["ms_per_step"], ws), "ms_per_step": r["ms_per_step"],
                "steps_timed": r["steps"], "l1_rel_vs_fp64_gpu": l1_rel(prob, r["state"], res["fp64"]["state"]),
                "stages_compared": r["stages_compared"], "smooth_fraction": r["smooth_fraction"],
                "kernel_ms": {x: round(v, 4) for x, v in kern.items()},
                "roofline_frac": {x: round(per[x]["frac"], 4) for x in names},
                "dominant_kernel": per[top]["kernel"], "launch_shapes": r["shapes"],
                "workspace_gb": round(r["workspace"] / 1e9, 2)}
            out["forms"][form]["_r"] = r
            out["forms"][form]["_top"] = (top, units[top], kern[top], per[top], kern)
        return out

    def measure_ensemble():
        """The batched ensemble (256 instances on jittered periodic meshes of
        log-uniform sizes): the instances sharded over the ranks by triangle
        count, each rank's share advanced as one ensemble (one CUDA graph per
        step over all its instances), FP32 with and without the gate. Also the
        graph's step time against the sum of its kernels' times run one by
        one: the most a single persistent launch could remove."""
        sizes_n = inputs.ensemble_sizes(256)
        mine = replicas.partition_instances([2 * n * n for n in sizes_n], ws)[rank]
        probs = [inputs.ensemble_member(int(sizes_n[i]), seed=2400 + i) for i in mine]
        nt = sum(p.mesh.n_tri for p in probs)
        nt_all = sum(2 * int(n) * int(n) for n in sizes_n)
        K, W = args.steps, args.warmup
        out = {"workload": "batched ensemble: 256 instances, jittered periodic unit squares of log-uniform "
                           "5k-200k triangles (%d in all), 8-mode Fourier bottom, smoothed interface, chi=0.98; "
                           "instances sharded over %d rank(s) by triangle count" % (nt_all, ws),
               "n_tri": nt_all, "instances": 256, "forms": {}}
        for form in ("fp32_learned", "fp32"):
            learned = form == "fp32_learned"
            kw = dict(indicator=g.GKS2L_INDICATOR_MLP, indicator_threshold=gate.THRESHOLD) if learned else {}
            par = g.default_params(g=probs[0].g, chi=probs[0].chi, cfl=probs[0].cfl, precision=g.GKS2L_FP32, **kw)
            with torch.cuda.stream(stream):
                s = g.Solver([p.mesh for p in probs], par, np.concatenate([p.b_vert for p in probs]),
                             device=dev, stream=stream)
                avg0 = np.concatenate([p.avg for p in probs], axis=1)
                grad0 = np.concatenate([p.grad for p in probs], axis=2)
                s.set_state(avg0, grad0)
                if learned:
                    s.set_mlp(gate_params)
                shapes = s.autotune(1)
                s.set_state(avg0, grad0)
                s.advance(2 * W)
                torch.cuda.synchronize(dev)
                barrier()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                s.advance(2 * K, sync=False)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                barrier()
                ms = max_over_ranks(e0.elapsed_time(e1) / K)
                st = s.stats()
                if st["status"] != 0:
                    raise RuntimeError("device status %d after the timed ensemble run" % st["status"])
                k = s.profile_kernels(2)
                ksum = k["step_begin"] + 2 * (k["recon"] + k["iface"] + k["edge"] + k["update"])
                out["forms"][form] = {"value": nt_all * 2 / (ms * 1e-3), "ms_per_step": ms,
                                      "kernel_sum_ms_per_step": ksum, "graph_minus_kernels_ms": ms - ksum,
                                      "smooth_fraction": st["smooth_fraction"], "launch_shapes": shapes,
                                      "kernel_ms": {x: round(v, 4) for x, v in k.items()}}
                del s
                torch.cuda.empty_cache()
        return out

    head = measure(args.workload, True)
    secondary = [measure(w, False) for w in args.secondary.split(",")
                 if w and w != args.workload and w != "ensemble"]
    ens = measure_ensemble() if "ensemble" in args.secondary.split(",") else None

    # the stated error on a smooth case that moves: the smooth periodic case
    # (512 triangles, 100 stages), each FP32 form against the plain FP64 form
    smooth = inputs.smooth_periodic(16)
    with torch.cuda.stream(stream):
        ref = solver(smooth, "fp64")
        ref.advance(100)
        a64, _ = ref.get_state()
        l1_smooth = {}
        for form, learned in FORMS[:2]:
            s = solver(smooth, form)
            s.advance(100)
            l1_smooth[form] = l1_rel(smooth, s.get_state()[0], a64)
            if learned:
                l1_smooth["smooth_fraction"] = s.stats()["smooth_fraction"]

    hf = head["forms"]["fp32_learned"]
    rh = hf["_r"]
    value = hf["value"]
    top, units, top_ms, roof, kern = hf["_top"]
    roof = dict(roof)
    tpu = TRAFFIC_PER_UNIT.get(top)
    roof["traffic"] = tpu * units if tpu else None
    fl_unit = recon_flops(rh["smooth_fraction"]) if top == "recon" else WORK_PER_UNIT[top][0]
    by_unit = recon_bytes(rh["smooth_fraction"]) if top == "recon" else WORK_PER_UNIT[top][1]
    # the bound's own measure: bytes for an HBM-bound kernel, flops otherwise
    roof["algorithmic_per_unit"] = by_unit if roof["bound"] == "hbm" else fl_unit
    roof["algorithmic_flops_per_unit"] = fl_unit
    roof["algorithmic_bytes_per_unit"] = by_unit
    roof["units_per_launch"] = units
    roof["launch_ms"] = top_ms
    ex = EXECUTED_FP32_PER_UNIT.get(top)
    roof["executed_fp32_per_unit"] = ex
    roof["overhead_executed_over_algorithmic"] = (ex / fl_unit) if ex else None
    roof["per_kernel"] = hf["roofline_frac"]
    timed = [x for x in kern if x != "step_begin"]
    ksum = sum(kern[x] for x in timed)
    share = {x: kern[x] / ksum for x in timed}
    launches_per_step = 1 + 2 * 5   # step start + (reconstruction, gate, fused edge, deferred edges, update) per stage

    def strip(w):
        return {"workload": w["workload"], "n_tri": w["n_tri"],
                "forms": {f: {k: v for k, v in d.items() if not k.startswith("_")} for f, d in w["forms"].items()},
                "speedup_over_fp64_gpu": w["forms"]["fp32_learned"]["value"] / w["forms"]["fp64"]["value"]}

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": rh["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64+bf16",
        "data": "synthetic (seeded jittered mesh, analytic initial data)",
        "config": {"workload": head["workload"],
                   "form": "FP32 moments/reconstruction with FP64 balance terms and sums, learned BF16 gate",
                   "l2": "inputs larger than L2 (operators and state %.1f GB)" % (rh["workspace"] / 1e9),
                   "parallelism": "replicas" if ws > 1 else "single GPU",
                   "launch_shapes": rh["shapes"]},
        "forms": strip(head)["forms"],
        "speedup_over_fp64_gpu": strip(head)["speedup_over_fp64_gpu"],
        "repeat_ms_per_step": rh.get("repeat_ms_per_step"),
        "repeat_median_ms_per_step": float(np.median(rh["repeat_ms_per_step"])) if rh.get("repeat_ms_per_step") else None,
        "secondary": [strip(w) for w in secondary],
        "ensemble": ens,
        "l1_rel_smooth_case_vs_fp64_gpu": l1_smooth,
        "gate": {"train_s": gate_train_s, "train_quality": gate_q, "smooth_fraction": rh["smooth_fraction"],
                 "threshold": gate.THRESHOLD},
        "kernel_ms": {k: round(v, 4) for k, v in kern.items()},
        "kernel_share": {k: round(v, 4) for k, v in share.items()},
        "roofline": roof,
        "alu_peaks_tflops": live_peaks,
        "clocks": rh["clocks"],
        "e2e": rh["e2e"],
        "e2e_sequential": rh.get("e2e_sequential"),
        "gpu_launches": launches_per_step * args.steps,
        "cpu_baseline": cpu,
    }
    if rank == 0:
        print(json.dumps(line))
    if ws > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
