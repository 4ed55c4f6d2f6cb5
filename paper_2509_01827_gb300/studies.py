"""Crack-pattern studies of Sec. 4 on the solver, one JSON line per case.

    python -m paper_2509_01827_gb300.studies compact_tension [--n 100]
    python -m paper_2509_01827_gb300.studies kalthoff [--n 200,400]
    python -m paper_2509_01827_gb300.studies ceiling [--n 64]
    python -m paper_2509_01827_gb300.studies sensitivity [--n 64]
    python -m paper_2509_01827_gb300.studies tri_throughput [--n 1024]

compact_tension: the Dirichlet compact-tension plate (Sec. 4.3) at the three
loading rates of Sec. 4.3, FP64 and FP32-mixed, with the dissipated energy U_d
(Figs. of Sec. 4.3 plot it against time), the grown splits, the branching
time, the fragments and the FP32-vs-FP64 Jaccard of the cracked sets.

kalthoff: the upper half of the Kalthoff-Winkler plate (Sec. 4.1) in the
multiple-tips and single-tip scopes, with the direction of the crack grown
from the notch tip in three rings around it (Sec. 4.1 compares crack angles).

ceiling: how far the crack map the surrogate learns is fixed by its input.
On n runs of the surrogate's data set (test seeds 10^6 + q), the Jaccard
index at 80 us of the FP32-mixed map (the training target) against the FP64
map, and of the FP64 and FP32 maps against runs whose G_c field is raised by
one FP32 ulp everywhere.

sensitivity: how finely the crack map depends on the G_c field.  On n runs of
the surrogate's data set, the Jaccard index at 80 us of the FP32-mixed map
against the maps of the same run with G_c replaced by: the value the
surrogate's BF16 input channel holds ((G_c - 3) / 0.36 rounded to BF16 and
mapped back); the same in two BF16 words (the rounded value and its rounded
remainder); G_c times 1 + r, r uniform in +-1e-4, +-1e-3, +-1e-2 (Philox
stream 7); an independent field (another seed, same traction and notch).

tri_throughput: FP64 and FP32-mixed element-updates/s of the unstructured
constant-strain triangle path (cem_tri_mesh_create) on an n x n jittered plate of 2 n^2
triangles with tractions and a random initial state, CUDA events around
repeated cem_step calls, and the mesh's sizes for the roofline.
"""
import argparse
import json
import time

import numpy as np

from . import inputs, metrics


def _run(p, precision, chunk=1000):
    from .cem import Solver
    import torch
    g = Solver(p, precision=precision)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    left = p.steps
    while left:
        n = min(chunk, left)
        g.step(n)
        left -= n
    torch.cuda.synchronize()
    el = time.perf_counter() - t0
    out = dict(cracks=g.cracks(), counts=g.counts(), seconds=el, fragments=g.fragments(labels=False)[0],
               energy=g.energy())
    g.close()
    return out


def _summary(p, r, dt):
    c = r["cracks"]
    grown = c["step"] >= 0
    bs = metrics.branching_step(c, p.nx, p.ny, p.hx, p.hy, p.active)
    return dict(steps=p.steps, seconds=round(r["seconds"], 3), grown=int(np.sum(grown)),
                tips_end=int(r["counts"]["n_tips"]), U_d=float(np.sum(c["ud"])),
                branching_t_us=None if bs is None else round(bs * dt * 1e6, 3),
                fragments=int(r["fragments"]))


def compact_tension(n=100):
    from .cem import CEM_FP32_MIXED, CEM_FP64
    for v0 in (1.375, 3.318, 3.993):
        p = inputs.compact_tension(n, v0=v0)
        p.energy_every = 0
        dt = inputs.estimate_dt(p)
        r64 = _run(p, CEM_FP64)
        r32 = _run(p, CEM_FP32_MIXED)
        line = dict(study="compact_tension", n=n, v0=v0, t_end_us=round(p.steps * dt * 1e6, 2),
                    fp64=_summary(p, r64, dt), fp32=_summary(p, r32, dt),
                    jaccard_fp32_fp64=metrics.jaccard(r64["cracks"]["elem"], r32["cracks"]["elem"]))
        print(json.dumps(line), flush=True)


def kalthoff(ns=(200, 400)):
    from .cem import CEM_FP32_MIXED, CEM_FP64
    L, notch_y, notch_len = 0.1, 0.025, 0.05
    rings = ((2e-3, 10e-3), (5e-3, 25e-3), (10e-3, 40e-3))
    for n in ns:
        for scope, name in ((inputs.SCOPE_NBHD, "mct"), (inputs.SCOPE_TIPS, "sct")):
            p = inputs.kalthoff(n, L=L, notch_y=notch_y, notch_len=notch_len, scope=scope)
            p.energy_every = 0
            dt = inputs.estimate_dt(p)
            line = dict(study="kalthoff", n=n, scope=name, t_end_us=round(p.steps * dt * 1e6, 2))
            for tag, prec in (("fp64", CEM_FP64), ("fp32", CEM_FP32_MIXED)):
                r = _run(p, prec)
                s = _summary(p, r, dt)
                tip = ((notch_len), notch_y)  # the notch tip: end of the pre-cracked row
                s["angles_deg"] = [None if a is None else round(a, 1) for a in
                                   (metrics.crack_angle(r["cracks"], p.nx, p.hx, p.hy, tip, r0, r1)
                                    for r0, r1 in rings)]
                s["first_growth_us"] = (None if s["grown"] == 0 else
                                        round(float(np.min(r["cracks"]["step"][r["cracks"]["step"] >= 0]))
                                              * dt * 1e6, 2))
                line[tag] = s
            print(json.dumps(line), flush=True)


def ceiling(n=64):
    from .cem import CEM_FP32_MIXED, CEM_FP64
    J = {"fp32_vs_fp64": [], "fp64_vs_gc_ulp": [], "fp32_vs_gc_ulp": []}
    for q in range(n):
        seed = 10**6 + q
        p, _ = inputs.surrogate_run(seed)
        u, _ = inputs.surrogate_run(seed)
        u.gc = np.nextafter(u.gc, np.float32(np.inf)).astype(np.float32)
        c64 = _run(p, CEM_FP64)["cracks"]["elem"]
        c32 = _run(p, CEM_FP32_MIXED)["cracks"]["elem"]
        u64 = _run(u, CEM_FP64)["cracks"]["elem"]
        u32 = _run(u, CEM_FP32_MIXED)["cracks"]["elem"]
        line = dict(study="ceiling", seed=seed, n64=len(c64), n32=len(c32),
                    fp32_vs_fp64=metrics.jaccard(c64, c32), fp64_vs_gc_ulp=metrics.jaccard(c64, u64),
                    fp32_vs_gc_ulp=metrics.jaccard(c32, u32))
        for k in J:
            J[k].append(line[k])
        print(json.dumps(line), flush=True)
    print(json.dumps(dict(study="ceiling_summary", runs=n,
                          **{k: dict(mean=float(np.mean(v)), min=float(np.min(v)),
                                     p10=float(np.percentile(v, 10))) for k, v in J.items()})), flush=True)


def bf16_round(a):
    """Round-to-nearest-even of float32 values to BF16, returned as float32."""
    u = np.asarray(a, np.float32).view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32)


def sensitivity(n=64):
    from .cem import CEM_FP32_MIXED
    from .train_surrogate import GC_SD
    keys = ["bf16_input", "bf16_two_words", "rel_1e-4", "rel_1e-3", "rel_1e-2", "other_field"]
    J = {k: [] for k in keys}
    for q in range(n):
        seed = 10**6 + q
        p, _ = inputs.surrogate_run(seed)
        ref = _run(p, CEM_FP32_MIXED)["cracks"]["elem"]
        gc = np.asarray(p.gc, np.float32)
        v = ((gc.astype(np.float64) - 3.0) / GC_SD).astype(np.float32)
        hi = bf16_round(v)
        lo = bf16_round(v - hi)
        r = 2.0 * inputs.uniform01(len(gc), seed, stream=7) - 1.0
        other = inputs.weibull_gc(len(gc), 3.0, 10.0, seed + 10**7)
        fields = {"bf16_input": 3.0 + GC_SD * hi.astype(np.float64),
                  "bf16_two_words": 3.0 + GC_SD * (hi.astype(np.float64) + lo.astype(np.float64)),
                  "rel_1e-4": gc * (1.0 + 1e-4 * r), "rel_1e-3": gc * (1.0 + 1e-3 * r),
                  "rel_1e-2": gc * (1.0 + 1e-2 * r), "other_field": other}
        line = dict(study="sensitivity", seed=seed, n32=len(ref))
        for k in keys:
            p.gc = np.asarray(fields[k], np.float32)
            line[k] = metrics.jaccard(ref, _run(p, CEM_FP32_MIXED)["cracks"]["elem"])
            J[k].append(line[k])
        print(json.dumps(line), flush=True)
    print(json.dumps(dict(study="sensitivity_summary", runs=n,
                          **{k: dict(mean=float(np.mean(v)), min=float(np.min(v)),
                                     p10=float(np.percentile(v, 10))) for k, v in J.items()})), flush=True)


def tri_throughput(n=1024, steps=200, warmup=10):
    import torch
    from .cem import CEM_FP32_MIXED, CEM_FP64, TriSolver
    p = inputs.tri_plate(n, n, lx=0.1, ly=0.1, jitter=0.2, traction=1e6, random_state=1e-3,
                         steps=steps)
    ed = inputs.tri_edges(p.conn)
    for name, prec in (("fp64", CEM_FP64), ("fp32", CEM_FP32_MIXED)):
        g = TriSolver(p, precision=prec)
        g.step(warmup)
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(g._stream)
        g.step(steps)
        e1.record(g._stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / steps
        line = dict(study="tri_throughput", precision=name, n=n, nodes=int(p.n_nodes),
                    elements=int(p.n_elems), edges=int(len(ed["n1"])),
                    incidences=int(6 * len(ed["n1"]) - 3 * int(np.sum(ed["e2"] < 0))),
                    steps=steps, ms_per_step=ms, element_updates_per_s=p.n_elems / (ms * 1e-3))
        g.close()
        print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("study", choices=["compact_tension", "kalthoff", "ceiling", "sensitivity",
                                      "tri_throughput"])
    ap.add_argument("--n", default=None)
    a = ap.parse_args()
    from . import build
    build.build()
    if a.study == "compact_tension":
        compact_tension(int(a.n or 100))
    elif a.study == "ceiling":
        ceiling(int(a.n or 64))
    elif a.study == "sensitivity":
        sensitivity(int(a.n or 64))
    elif a.study == "tri_throughput":
        tri_throughput(int(a.n or 1024))
    else:
        kalthoff(tuple(int(x) for x in (a.n or "200,400").split(",")))


if __name__ == "__main__":
    main()
