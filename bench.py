#!/usr/bin/env python
"""Benchmark of the explicit MCT-2D-CEM step on one or more GB300s.

Workload (default): the 2048 x 2048 Q4 fragmentation plate -- 0.1 m square,
central hole of radius 5 mm, 50 MPa internal pressure pulse, Weibull G_c
(mean 3 J/m^2, shape 10, seed 2509).  A "step" is one whole explicit step:
piece forces, node update of every real node, phantom update, surface
evaluation, multi-tip tracking, and an energy record every 50 steps.
Metric: element-updates/s = active elements * steps / time.

--impl ours (default): the CUDA library.  After --warmup steps the run is
  advanced, untimed, past crack initiation until the tip list holds
  --min-tips tips; the --steps steps that follow are timed with CUDA events
  (graph replays).  The roofline of the node update comes from the same
  steps replayed from the timed window's saved start state with per-kernel
  CUDA events, 53 B per element-update (FP32-mixed) over its average launch
  time.  Beside it: the whole run from
  t = 0 to 60 us in both precisions (throughput of each, and the FP32 crack
  pattern against the FP64 one: Jaccard over time, fragments, branching
  time), end-to-end throughput through pipelined eight-step calls, and the
  CPU oracle on a bounded sample.
--impl reference: the CPU oracle as it stands (the only reference this
  method has), timed on a bounded sample on this host.
Multi-GPU (torchrun): one independent replica per GPU (the path does not
shard across GPUs); value = all ranks' element-updates / max rank time.

--workload notched_plate_100x40 / notched_plate_400x160: the single notched
  plates (1 mm and 0.25 mm elements, 1 MPa traction), L2-resident, so their
  throughput is latency- and L2-bound; use --min-tips 0.
--workload fragmentation_2048_dirichlet: the same plate under a 2 m/s
  outward edge velocity.
--workload specimens_64: 64 notched plates from 100 x 40 to 400 x 160 (seed
  1827), each run to 80 us with its own time step, stepped together as one
  batch (one launch per kernel kind for all specimens); the launch
  configuration comes from the autotuner on a separate copy of the batch.
  value = sum over specimens of active elements * steps / batch time.
"""
import argparse
import json
import math
import os
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "element-updates/s"
HBM_FALLBACK_GBS = 6800.0


def measured_peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def make_problem(workload):
    from paper_2509_01827_gb300 import inputs
    if workload == "fragmentation_2048_neumann":
        p = inputs.fragmentation(2048, mode="neumann", p0=50e6, seed=2509)
    elif workload == "fragmentation_2048_dirichlet":
        p = inputs.fragmentation(2048, mode="dirichlet", v0=2.0, seed=2509)
    elif workload in ("notched_plate_100x40", "notched_plate_400x160"):
        p = inputs.CONFIGS[workload]()
        # room for the cracks of the timed, profiled and end-to-end steps
        # beyond the configuration's own end time
        p.phantom_cap = max(p.phantom_cap, 4 * p.nx * p.ny)
        p.crack_cap = max(p.crack_cap, p.nx * p.ny)
    else:
        raise SystemExit(f"unknown workload {workload}")
    p.energy_every = 50
    return p


# ------------------------------------------------------------------ clocks
class ClockSampler:
    QUERY = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.QUERY}",
                                       "--format=csv,noheader,nounits", "-lms", "100"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except Exception:
            self.p.kill()
        self.f.flush()
        rows = []
        for line in open(self.f.name):
            c = [x.strip() for x in line.split(",")]
            if len(c) < 10:
                continue
            if self.uuid and self.uuid not in c[1]:
                continue
            rows.append(c)
        os.unlink(self.f.name)
        if not rows:
            return None
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in rows for n, v in zip(names, r[6:10]) if v.lower() == "active"})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows)}


# ------------------------------------------------------------------ oracle
def time_oracle(prob, budget_s=15.0, max_steps=60):
    """The CPU oracle as it stands, single thread, on a bounded sample of the
    workload: the first steps of the same run."""
    from oracle.oracle import from_problem
    t0 = time.perf_counter()
    s = from_problem(prob)
    setup = time.perf_counter() - t0
    t1 = time.perf_counter()
    s.step(1)
    one = time.perf_counter() - t1
    n = int(max(1, min(max_steps, budget_s / max(one, 1e-6)))) if one < budget_s else 0
    t2 = time.perf_counter()
    if n:
        s.step(n)
    rest = time.perf_counter() - t2
    steps = n + 1
    el = time.perf_counter() - t1
    del rest
    value = prob.n_active * steps / el
    return {"value": value, "unit": METRIC, "cores": 1, "kind": "oracle",
            "sample": f"first {steps} steps of the {prob.nx}x{prob.ny} run "
                      f"({prob.n_active} active elements), FP64, single thread; "
                      f"set-up {setup:.1f}s not timed", "seconds": round(el, 3)}


# ------------------------------------------------------------------ ranks
def max_over_ranks(x, world, device="cuda"):
    """The largest x over all ranks (x itself on one rank); NCCL on the GPU,
    any process group (gloo on the CPU in the tests)."""
    if world <= 1:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(units_per_rank, ms_per_rank, world, device="cuda"):
    """Whole-job throughput of independent replicas: the units of all ranks
    divided by the slowest rank's time.  Returns (units/s, max ms)."""
    ms = max_over_ranks(ms_per_rank, world, device)
    return world * units_per_rank / (ms * 1e-3), ms


# ------------------------------------------------------------------ ours
def bytes_per_update(precision):
    """Algorithmic bytes per element-update: the state one step must read and
    write per (real node, element) pair of the structured mesh."""
    if precision == "fp32":
        # u hi+lo read+write 32, v read+write 16, 1/m 4; element state 1
        return 53.0
    # u read+write 32, v read+write 32, 1/m 8; element state 1
    return 73.0


def measured_traffic(kernel_source):
    """DRAM bytes (read + write) of one node-update launch from the committed
    ncu summary, if it was taken on the current kernel source (its SHA-256
    is recorded beside the figure); None otherwise."""
    import hashlib
    path = os.path.join(ROOT, "profiles", "k_march32_fragmentation_2048.md")
    try:
        text = open(path).read()
        src = open(kernel_source, "rb").read()
    except OSError:
        return None, None
    vals = {}
    for line in text.splitlines():
        for key in ("traffic_bytes_per_launch:", "source_sha256:", "window:"):
            if line.strip().startswith(key):
                vals[key] = line.split(":", 1)[1].strip()
    if vals.get("source_sha256:") != hashlib.sha256(src).hexdigest():
        return None, None
    try:
        return float(vals["traffic_bytes_per_launch:"]), vals.get("window:")
    except (KeyError, ValueError):
        return None, None


def timed_steps(sol, n, stream):
    import torch
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sol.step(n)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1)


def advance_to_tips(sol, min_tips, max_steps, chunk=100):
    """Steps (untimed) until the tip list holds min_tips tips."""
    done = 0
    while done < max_steps and sol.counts()["n_tips"] < min_tips:
        sol.step(chunk)
        done += chunk
    return done


def accuracy_block(c32, c64, prob, dt, series_us=(5, 10, 20, 30, 40, 50, 60)):
    """FP32-mixed against FP64 crack patterns of the same run (Jaccard of the
    cracked-element sets over time, fragments, branching time and branch
    angle)."""
    from paper_2509_01827_gb300 import metrics
    out = {"jaccard_end": metrics.jaccard(c32["elem"], c64["elem"]),
           "cracked_fp32": int(len(c32["elem"])), "cracked_fp64": int(len(c64["elem"]))}
    ser = []
    for tus in series_us:
        s_ = int(round(tus * 1e-6 / dt))
        a = c32["elem"][c32["step"] <= s_]
        b = c64["elem"][c64["step"] <= s_]
        ser.append([tus, round(metrics.jaccard(a, b), 4)])
    out["jaccard_vs_time_us"] = ser
    for tag, c in (("fp32", c32), ("fp64", c64)):
        s_ = metrics.branching_step(c, prob.nx, prob.ny, prob.hx, prob.hy, prob.active)
        out[f"branching_t_us_{tag}"] = None if s_ is None else round(s_ * dt * 1e6, 3)
        ang, _ = metrics.branch_angle(c, prob.nx, prob.ny, prob.hx, prob.hy, prob.active)
        out[f"branch_angle_deg_{tag}"] = None if ang is None else round(ang, 2)
    return out


def run_ours(args, rank, world):
    import torch
    from paper_2509_01827_gb300 import build as _build
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, CEM_FP64, Solver

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    prec = CEM_FP32_MIXED if args.precision == "fp32" else CEM_FP64
    prob = make_problem(args.workload)
    sol = Solver(prob, precision=prec, device=dev)
    stream = sol._stream
    nact = prob.n_active
    # warm-up (also builds the CUDA graphs), then the run is advanced, untimed,
    # past crack initiation until the tip list holds --min-tips tips
    sol.step(args.warmup)
    adv = advance_to_tips(sol, args.min_tips, args.max_advance) if args.min_tips > 0 else 0
    torch.cuda.synchronize()
    # the state at the start of the timed window: its steps are replayed for
    # the per-kernel profile below
    start_blob = sol.save_state()
    c0 = sol.counts()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")  # lets ncu select the timed launches
    e0.record(stream)
    sol.step(args.steps)
    e1.record(stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    value, ms = replica_throughput(nact * args.steps, e0.elapsed_time(e1), world)
    if world > 1:
        torch.distributed.barrier()
    c1 = sol.counts()
    launches = c1["kernel_launches"] - c0["kernel_launches"]

    # per-kernel device time over the timed window's own steps, replayed from
    # its saved start state (kernels one after another, CUDA events on the
    # launching stream); the run then continues from the timed window's end
    nprof = max(1, min(args.profile_steps, args.steps, 4000))
    end_blob = sol.save_state()
    sol.load_state(start_blob)
    prof = sol.profile_steps(nprof)
    sol.load_state(end_blob)
    peaks = measured_peaks()
    hbm = peaks.get("hbm_gbs")
    peak_src = "measured" if hbm else "fallback"
    hbm = hbm or HBM_FALLBACK_GBS
    bpu = bytes_per_update(args.precision)
    bytes_launch = nact * bpu  # one node-update launch advances every active element once
    main_ms = prof["main"] / nprof
    achieved = bytes_launch / (main_ms * 1e-3) / 1e9
    share = prof["main"] / prof["total"] if prof["total"] > 0 else None
    traffic, traffic_window = (None, None)
    if args.precision == "fp32":
        traffic, traffic_window = measured_traffic(
            os.path.join(ROOT, "paper_2509_01827_gb300", "csrc", "step_fp32.cu"))
    if args.traffic is not None:
        traffic, traffic_window = args.traffic, "given on the command line"

    # end to end through the C ABI: one cem_step_async(8) per eight steps
    # from the host (each call reads back the previous call's per-step status
    # words, written to mapped pinned memory, while its own steps run), load
    # factors uploaded from pinned host memory, and a final cem_sync
    per_call = 8
    ne2e = per_call * max(1, min(args.steps, args.e2e_steps) // per_call)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ne2e // per_call):
        sol.step_async(per_call)
    sol.sync()
    e2e_val, _ = replica_throughput(nact * ne2e, (time.perf_counter() - t0) * 1e3, world)
    counts = sol.counts()
    sol.close()

    whole = companion = accuracy = None
    if args.whole_run and rank == 0 and world == 1:
        # the whole run from t = 0 to the workload's end time, in this
        # precision and in the other one (same inputs): throughput of each and
        # the crack-pattern agreement of the two
        other = CEM_FP64 if prec == CEM_FP32_MIXED else CEM_FP32_MIXED
        tabs = {}
        for pr in (prec, other):
            s2 = Solver(make_problem(args.workload), precision=pr, device=dev)
            s2.step(1)
            n2 = prob.steps - 1
            ms2 = timed_steps(s2, n2, s2._stream)
            rate = nact * n2 / (ms2 * 1e-3)
            tabs[pr] = s2.cracks()
            dt = s2.counts()["dt"]
            en = s2.energy()
            nfrag, _ = s2.fragments(labels=False)
            entry = {"precision": "fp64" if pr == CEM_FP64 else "fp32", "value": rate,
                     "unit": METRIC, "steps": n2, "t_end_us": round(s2.counts()["t"] * 1e6, 3),
                     "ms_per_step": ms2 / n2, "fragments_end": nfrag,
                     # dissipated energy U_d (J/m) and KE, SE, W_ext over time
                     "energy_series": [[round(float(en["t"][q]) * 1e6, 2)] +
                                       [float(en[k][q]) for k in ("U_d", "KE", "SE", "W_ext")]
                                       for q in range(0, len(en["t"]), max(1, len(en["t"]) // 12))]}
            if pr == prec:
                whole = entry
            else:
                companion = entry
            s2.close()
        if args.precision == "fp32":
            accuracy = accuracy_block(tabs[prec], tabs[other], prob, dt)
            accuracy["fragments_fp32"] = whole["fragments_end"]
            accuracy["fragments_fp64"] = companion["fragments_end"]
            accuracy["reference"] = ("the FP64 mode of this library on the same run "
                                     "(bit-identical to the CPU oracle in the parity tests)")

    if rank != 0:
        return None
    cfg = {"workload": args.workload, "mesh": f"{prob.nx}x{prob.ny} Q4",
           "active_elements": nact, "nodes": prob.n_nodes,
           "precision": "fp32-mixed (FP32 element math, compensated FP32 displacement)"
           if args.precision == "fp32" else "fp64",
           "energy_every": prob.energy_every,
           "l2": f"inputs larger than L2: state {bpu * nact / 1e6:.0f} MB > 129 MB",
           "parallelism": f"replicas x{world}",
           "timed_window": f"{args.steps} steps after the run was advanced untimed past "
                           f"initiation to >= {args.min_tips} tips",
           "t_start_us": round(c0["t"] * 1e6, 3), "tips_start": c0["n_tips"],
           "cracked_start": c0["n_cracked"], "advanced_steps": adv,
           "t_end_us": round(c1["t"] * 1e6, 3), "tips_end": c1["n_tips"],
           "cracked_elements_end": c1["n_cracked"]}
    if accuracy:
        cfg["crack_pattern_accuracy"] = accuracy
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": cfg,
        "roofline": {"bound": "hbm", "achieved": achieved, "peak": hbm, "unit": "GB/s",
                     "frac": achieved / hbm, "traffic": traffic,
                     "traffic_window": traffic_window,
                     "kernel": "node update (k_march32)" if args.precision == "fp32"
                     else "tile update (k_main64)", "peak_source": peak_src,
                     "algorithmic_bytes_per_launch": bytes_launch,
                     "bytes_per_element_update": bpu,
                     "avg_launch_ms": main_ms, "share_of_step": share,
                     "profiled_steps": nprof,
                     "profiled_window": "the timed window's first profiled_steps steps, replayed "
                                        "from its saved start state, kernels one after another",
                     "per_kernel_ms": prof,
                     **({} if args.precision == "fp32" else {
                         "note": "the FP64 mode is bound by the FP64 pipe, not by HBM: 0.96 of "
                                 "its measured instruction rate (ncu summary of k_main64); this "
                                 "line states its HBM fraction only"})},
        "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": 16,
                "d2h_bytes_per_step": 76, "steps": ne2e,
                "how": "one cem_step_async(8) call per 8 steps from the host (an "
                       "eight-step graph): every step's status word (76 B) is written by "
                       "the last block of its split writes into a ring in mapped pinned "
                       "host memory; the next call reads them back while its steps run, "
                       "a final cem_sync; load "
                       "factors uploaded from pinned memory in 4096-step tables (16 B per "
                       "step)"},
        "gpu_launches": launches,
        "clocks": clk,
    }
    del counts
    if args.precision == "fp64":
        line["roofline"]["note"] = ("the FP64 tile kernel is bound by the FP64 pipe, "
                                    "not by HBM")
    if whole:
        line["whole_run"] = whole
    if companion:
        line["companion"] = companion
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle(make_problem(args.workload), args.cpu_budget)
    return line


def run_batch(args, rank, world):
    """The 64-specimen sweep as one batch (see the module docstring)."""
    import torch
    from paper_2509_01827_gb300 import build as _build, inputs
    from paper_2509_01827_gb300.cem import CEM_FP32_MIXED, CEM_FP64, Batch, Solver

    dev = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(dev)
    if rank == 0 or world == 1:
        _build.build()
    if world > 1:
        torch.distributed.barrier()
    prec = CEM_FP32_MIXED if args.precision == "fp32" else CEM_FP64
    probs = inputs.batch_specimens(64)
    for p in probs:
        p.energy_every = 50
    steps = [p.steps for p in probs]
    total_updates = sum(p.n_active * n for p, n in zip(probs, steps))

    def make():
        ms = [Solver(p, precision=prec, device=dev) for p in probs]
        return ms, Batch(ms, step_end=steps)

    # autotune on a throwaway copy (its timed steps advance that copy)
    ms_t, bt = make()
    tile_rows, grid = bt.autotune(max(1, args.autotune_steps))
    bt.close()
    for m in ms_t:
        m.close()

    members, b = make()
    b.set_config(tile_rows, grid)
    b.step(args.warmup)
    torch.cuda.synchronize()
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    clocks = ClockSampler(uuid)
    if world > 1:
        torch.distributed.barrier()
    torch.cuda.synchronize()
    c0 = b.counts()
    clocks.start()
    time.sleep(0.3)
    nrun = max(steps) - args.warmup
    if args.batch_steps > 0:
        nrun = min(nrun, args.batch_steps)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    torch.cuda.nvtx.range_push("timed")
    e0.record(b._stream)
    b.step(nrun)
    e1.record(b._stream)
    torch.cuda.nvtx.range_pop()
    torch.cuda.synchronize()
    time.sleep(0.2)
    clk = clocks.stop()
    ms = e0.elapsed_time(e1)
    c1 = b.counts()
    launches = c1["kernel_launches"] - c0["kernel_launches"]
    timed_updates = sum(p.n_active * max(0, min(n - args.warmup, nrun)) for p, n in zip(probs, steps))
    value, ms = replica_throughput(timed_updates, ms, world)
    cracked = c1["n_cracked"]
    b.close()
    for m in members:
        m.close()

    # end to end: a fresh batch, one cem_step(batch, 1) per step from the host
    members, b = make()
    b.set_config(tile_rows, grid)
    ne2e = max(1, min(args.e2e_steps, max(steps)))
    upd = sum(p.n_active * min(n, ne2e) for p, n in zip(probs, steps))
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(ne2e):
        b.step(1)
    e2e_val, _ = replica_throughput(upd, (time.perf_counter() - t0) * 1e3, world)
    b.close()
    for m in members:
        m.close()

    # the same specimens stepped one after another, each alone (a sample)
    nsolo = min(len(probs), max(1, args.solo_sample))
    solo_upd, solo_ms = 0, 0.0
    for p, n in list(zip(probs, steps))[:nsolo]:
        s = Solver(p, precision=prec, device=dev)
        s.step(1)
        torch.cuda.synchronize()
        f0 = torch.cuda.Event(enable_timing=True)
        f1 = torch.cuda.Event(enable_timing=True)
        f0.record(s._stream)
        s.step(n - 1)
        f1.record(s._stream)
        torch.cuda.synchronize()
        solo_ms += f0.elapsed_time(f1)
        solo_upd += p.n_active * (n - 1)
        s.close()
    if rank != 0:
        return None
    line = {
        "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": world,
        "steps": nrun, "warmup": args.warmup, "ms_per_step": ms / nrun,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32" if args.precision == "fp32" else "f64", "data": "synthetic",
        "config": {"workload": "specimens_64", "specimens": len(probs),
                   "meshes": "notched plates 100x40 .. 400x160 (s ~ U(1, 4), seed 1827)",
                   "active_elements_total": sum(p.n_active for p in probs),
                   "steps_per_specimen": [min(steps), max(steps)],
                   "element_updates": total_updates, "energy_every": 50,
                   "precision": args.precision, "tile_rows": tile_rows, "grid_main": grid,
                   "l2": "state of all specimens about 0.1 GB: close to L2 (129 MB), "
                         "no flush between steps",
                   "parallelism": f"batch of 64, replicas x{world}",
                   "cracked_elements_end": cracked},
        "roofline": None,
        "e2e": {"value": e2e_val, "unit": METRIC, "h2d_bytes_per_step": 16 * len(probs),
                "d2h_bytes_per_step": 76 * len(probs), "steps": ne2e,
                "how": "one cem_step(batch, 1) call per step from the host"},
        "gpu_launches": launches,
        "clocks": clk,
        "solo_sequential": {"value": solo_upd / (solo_ms * 1e-3), "unit": METRIC,
                            "specimens": nsolo,
                            "how": "the first specimens stepped alone, one after another"},
    }
    if not args.no_cpu_baseline:
        line["cpu_baseline"] = time_oracle(probs[0], args.cpu_budget)
        line["cpu_baseline"]["sample"] = "specimen 0 only: " + line["cpu_baseline"]["sample"]
    return line


def run_reference(args, rank):
    if rank != 0:
        return None
    if args.workload == "specimens_64":
        from paper_2509_01827_gb300 import inputs
        prob = inputs.batch_specimens(64)[0]
    else:
        prob = make_problem(args.workload)
    per = []
    t_all = time.perf_counter()
    for _ in range(max(1, args.steps_reference)):
        per.append(time_oracle(prob, args.cpu_budget / max(1, args.steps_reference)))
    wall = time.perf_counter() - t_all
    vals = [p["value"] for p in per]
    value = float(np.median(vals))
    cb = dict(per[-1])
    cb["value"] = value
    # the oracle's time for one step of the whole mesh, from its throughput
    ms_step = 1e3 * prob.n_active / value if value > 0 else None
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": METRIC, "n_gpus": 1,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms_step,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": args.workload, "mesh": f"{prob.nx}x{prob.ny} Q4",
                       "active_elements": prob.n_active},
            "cpu_baseline": cb, "wall_s": wall,
            "e2e": {"value": value, "unit": METRIC, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=1000)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64"])
    ap.add_argument("--workload", default="fragmentation_2048_neumann")
    ap.add_argument("--profile-steps", type=int, default=1000,
                    help="steps of the timed window replayed with per-kernel timing (at most --steps)")
    ap.add_argument("--e2e-steps", type=int, default=300)
    ap.add_argument("--whole-run", type=int, default=1,
                    help="also time the whole run in both precisions and compare crack patterns")
    ap.add_argument("--min-tips", type=int, default=100,
                    help="advance the run untimed until the tip list holds this many tips")
    ap.add_argument("--max-advance", type=int, default=6000)
    ap.add_argument("--cpu-budget", type=float, default=15.0)
    ap.add_argument("--steps-reference", type=int, default=1)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--autotune-steps", type=int, default=5)
    ap.add_argument("--solo-sample", type=int, default=8)
    ap.add_argument("--batch-steps", type=int, default=0,
                    help="specimens_64: time only this many batch steps (0: the whole run)")
    ap.add_argument("--traffic", type=float, default=None,
                    help="ncu DRAM bytes per launch of the node update, overriding the "
                         "committed summary")
    args = ap.parse_args()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if args.impl == "reference":
        line = run_reference(args, rank)
    else:
        if world > 1:
            import torch
            torch.distributed.init_process_group("nccl")
        if args.workload == "specimens_64":
            line = run_batch(args, rank, world)
        else:
            line = run_ours(args, rank, world)
        if world > 1:
            import torch
            torch.distributed.destroy_process_group()
    if line is not None:
        print(json.dumps(line))


if __name__ == "__main__":
    main()
