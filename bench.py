"""Benchmark: element matrices/s of the prism degree sweep (p = 1..7).

One step integrates, for every degree p = 1..7, E_p jittered straight-edged
prisms with random SPD diffusion, convection, reaction and source
coefficients (E_p = round(2e9 / (8 (NS^2 + NS))), ~2 GB of FP64 output per
degree), full non-symmetric A_e and b_e.  `value` is element matrices per
second over the whole sweep (sum E_p / step time), device-timed with CUDA
events, inputs resident in HBM; the L2 is flushed between timed steps.

Lines printed (one JSON line from rank 0):
  --impl ours (default): the CUDA library through its C ABI;
  --impl reference: the FP64 CPU oracle on the host cores, on a bounded
    per-degree sample of the same workload, extrapolated to the sweep.
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
sys.path.insert(0, ROOT)

from paper_1310_1191_gb300 import inputs  # noqa: E402

SWEEP_E = {1: 5952381, 2: 730994, 3: 152439, 4: 43860, 5: 15623, 6: 6475, 7: 3004}
# oracle sample per degree for the CPU baseline (~1-3 s of host work each)
CPU_SAMPLE = {1: 400000, 2: 40000, 3: 4000, 4: 600, 5: 96, 6: 32, 7: 16}
# nominal ALU peaks: 152 SMs x 2.07 GHz x lanes x 2 flops
PEAK_F32 = 152 * 2.07e9 * 128 * 2 / 1e12   # 80.5 TFLOP/s
PEAK_F64 = 1.25                            # TFLOP/s, GB300 FP64 (nominal)


def ns_of(p):
    return (p + 1) ** 2 * (p + 2) // 2


def nq_of(p):
    return (p + 1) ** 3


def flops_per_elem(p):
    """Algorithmic flops per element: 8 NQ NS^2 (contraction) + 2 NQ NS (load
    vector) + 32 NQ NS (weighted tile, dense 4x4 count) + 150 NQ (geometry)."""
    n, q = ns_of(p), nq_of(p)
    return 8 * q * n * n + 2 * q * n + 32 * q * n + 150 * q


def bytes_per_elem(p, osz):
    """Algorithmic HBM bytes per element: coords 144 + coefficients 88 in,
    A (NS^2) + b (NS) out."""
    n = ns_of(p)
    return 232 + osz * (n * n + n)


class Clocks:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
             "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
             "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), "--query-gpu=" + q,
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for l in self.lines:
            f = [x.strip() for x in l.split(",")]
            if len(f) < 8:
                continue
            try:
                sm.append(float(f[0]))
                mx.append(float(f[1]))
            except ValueError:
                continue
            for n, v in zip(names, f[4:8]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_baseline(sweep, sample=CPU_SAMPLE):
    """The FP64 oracle, as it stands, on a bounded per-degree sample of the
    sweep; the sweep time is extrapolated from the per-element times."""
    import oracle
    oracle.build()
    t_total, desc = 0.0, []
    for p in sweep:
        n = min(sample[p], sweep[p])
        X = inputs.prism_mesh(sweep[p])[:n] if n < sweep[p] else inputs.prism_mesh(sweep[p])
        C = inputs.coefficients(n)
        t0 = time.perf_counter()
        oracle.integrate(1, p, X, C)
        dt = time.perf_counter() - t0
        t_total += dt / n * sweep[p]
        desc.append("p%d:%d" % (p, n))
    units = sum(sweep.values())
    return {"value": units / t_total, "unit": "element matrices/s", "cores": oracle.max_threads(),
            "kind": "oracle",
            "sample": "first n prisms of each degree's mesh (%s), FP64 full A_e+b_e; sweep time "
                      "extrapolated per degree" % ",".join(desc)}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sweep = dict(SWEEP_E)
    samp = dict(CPU_SAMPLE)
    t0 = time.perf_counter()
    vals = []
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(sweep, samp)
        vals.append(cb["value"])
    el = time.perf_counter() - t0
    v = statistics.median(vals)
    units = sum(sweep.values())
    line = {"impl": "reference", "metric": "element matrices/s (prism sweep p=1..7)", "value": v,
            "unit": "element matrices/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": units / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "prism degree sweep p=1..7, E_p=%s" % list(sweep.values()),
                       "precision": "f64", "layout": "full"},
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": "element matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": el}
    print(json.dumps(line), flush=True)


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_1310_1191_gb300 import _lib as lib
    from paper_1310_1191_gb300 import build as _build

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    _build.build()
    lib.load()
    prec = lib.FEM_F64 if args.precision == "f64" else lib.FEM_F32
    dt = torch.float64 if prec == lib.FEM_F64 else torch.float32
    osz = 8 if prec == lib.FEM_F64 else 4
    sweep = {p: (max(1, SWEEP_E[p] // args.scale_down)) for p in range(1, 8)}
    tables = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    stream = torch.cuda.Stream(device=dev)
    data = {}
    for p, E in sweep.items():
        X = inputs.prism_mesh(E)
        C = inputs.coefficients(E)
        n = ns_of(p)
        data[p] = dict(
            X=torch.from_numpy(X).to(dev), C=torch.from_numpy(C).to(dev),
            A=torch.empty((E, n * n), dtype=dt, device=dev),
            b=torch.empty((E, n), dtype=dt, device=dev),
            st=torch.empty((E,), dtype=torch.int32, device=dev), Xh=X, Ch=C)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def step(events=None):
        with torch.cuda.stream(stream):
            for p, d in data.items():
                if events is not None:
                    events[p][0].record(stream)
                lib.fem_integrate(tables, p, sweep[p], d["X"], d["C"], sweep[p], prec,
                                  lib.FEM_OUT_FULL, d["A"], d["b"], d["st"], stream)
                if events is not None:
                    events[p][1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    bad = sum(int((d["st"] != 0).sum().item()) for d in data.values())
    per_p = {p: [] for p in sweep}
    step_ms = []
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        for _ in range(args.steps):
            with torch.cuda.stream(stream):
                flush.zero_()
            ev = {p: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
                  for p in sweep}
            s0, s1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            s0.record(stream)
            step(ev)
            s1.record(stream)
            s1.synchronize()
            step_ms.append(s0.elapsed_time(s1))
            for p in sweep:
                per_p[p].append(ev[p][0].elapsed_time(ev[p][1]))
    torch.cuda.synchronize()
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.barrier()
        total_ms = t.item()
    units = sum(sweep.values()) * args.steps * world
    value = units / (total_ms / 1e3)

    # dominant kernel and its roofline
    mean_p = {p: statistics.mean(v) for p, v in per_p.items()}
    pdom = max(mean_p, key=mean_p.get)
    fl = flops_per_elem(pdom) * sweep[pdom]
    achieved = fl / (mean_p[pdom] / 1e3) / 1e12
    peak = PEAK_F64 if prec == lib.FEM_F64 else PEAK_F32
    per_degree = {}
    for p in sweep:
        t_s = mean_p[p] / 1e3
        tf = flops_per_elem(p) * sweep[p] / t_s / 1e12
        gbs = bytes_per_elem(p, osz) * sweep[p] / t_s / 1e9
        t_roof = max(flops_per_elem(p) / (peak * 1e12), bytes_per_elem(p, osz) / 6790.3e9)
        per_degree[str(p)] = {"elements": sweep[p], "ms": round(mean_p[p], 4),
                              "elem_per_s": sweep[p] / t_s, "tflops": round(tf, 3),
                              "gbs": round(gbs, 1),
                              "roofline_frac": round(t_roof * sweep[p] / t_s, 4)}

    # end to end: host buffers in pinned memory, copies inside the timed region
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(lib, tables, sweep, data, prec, dt, stream, args.e2e_steps)

    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(sweep)
    clocks = clk.summary()
    if rank == 0:
        line = {
            "metric": "element matrices/s (prism sweep p=1..7)", "value": value,
            "unit": "element matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": {"workload": "prism degree sweep p=1..7 (jittered prisms, random SPD D, b, "
                                   "c, f), E_p=%s" % list(sweep.values()),
                       "precision": args.precision, "layout": "full",
                       "l2": "flushed between timed steps (256 MB write)"},
            "gpu_launches": 7 * args.steps,
            "per_degree": per_degree,
            "roofline": {"bound": "alu", "kernel": "fma_kernel p=%d" % pdom,
                         "achieved": round(achieved, 4), "peak": peak, "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4), "traffic": None,
                         "peak_source": "nominal %s ALU peak (unit counts x clock)" % args.precision},
            "flagged_elements": bad,
            "clocks": clocks,
            "e2e": e2e, "cpu_baseline": cb,
        }
        print(json.dumps(line), flush=True)
    tables.close()
    if world > 1:
        dist.destroy_process_group()


def measure_e2e(lib, tables, sweep, data, prec, dt, stream, steps):
    """Same sweep with host (pinned) inputs and outputs; H2D of the inputs and
    D2H of A and b are inside the timed region."""
    import torch
    host = {}
    h2d = d2h = 0
    for p, d in data.items():
        host[p] = dict(X=torch.from_numpy(d["Xh"]).pin_memory(), C=torch.from_numpy(d["Ch"]).pin_memory(),
                       A=torch.empty(d["A"].shape, dtype=dt).pin_memory(),
                       b=torch.empty(d["b"].shape, dtype=dt).pin_memory())
        h2d += host[p]["X"].numel() * 8 + host[p]["C"].numel() * 8
        d2h += host[p]["A"].numel() * host[p]["A"].element_size() + host[p]["b"].numel() * host[p]["b"].element_size()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        with torch.cuda.stream(stream):
            for p, d in data.items():
                h = host[p]
                d["X"].copy_(h["X"], non_blocking=True)
                d["C"].copy_(h["C"], non_blocking=True)
                lib.fem_integrate(tables, p, sweep[p], d["X"], d["C"], sweep[p], prec,
                                  lib.FEM_OUT_FULL, d["A"], d["b"], d["st"], stream)
                h["A"].copy_(d["A"], non_blocking=True)
                h["b"].copy_(d["b"], non_blocking=True)
        stream.synchronize()
    el = time.perf_counter() - t0
    return {"value": sum(sweep.values()) * steps / el, "unit": "element matrices/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "torch pinned copies around fem_integrate"}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="f64", choices=["f64", "f32"])
    ap.add_argument("--scale-down", type=int, default=1, help="divide element counts (debug)")
    ap.add_argument("--e2e-steps", type=int, default=2)
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
