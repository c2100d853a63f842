"""Benchmark: element matrices/s of the prism degree sweep (p = 1..7).

Headline (`value`): one step integrates, for every degree p = 1..7, E_p
jittered straight-edged prisms with random SPD diffusion, convection,
reaction and source coefficients (E_p = round(2e9 / (8 (NS^2 + NS))), about
2 GB of FP64 output per degree), full non-symmetric A_e and b_e, in FP64
(--precision f32 for the FP32 kernels).  `value` is element matrices per
second over the whole sweep (sum E_p / step time), device-timed with CUDA
events on the launching stream, inputs resident in HBM, L2 flushed between
timed steps.  `e2e` is the same sweep through the host-buffer entry point
fem_integrate_host (pinned host inputs and outputs, copies inside the timed
region).

`workloads` (rank 0, unless --no-extras) reports the other workloads, each
timed the same way: P1 tetrahedra, the FP32 sweep, the tensor-core BF16x3 /
FP16x3 forms at p = 4..7 (errors against the GPU FP64 path), the 500k-prism
mixed-degree mesh (graph + autotuned persistent launch vs per-degree loop),
and the nonlinear-law workload with the exact law and the trained network.

--impl reference times the FP64 CPU oracle on the host cores on a bounded
per-degree sample of the same sweep, extrapolated to the sweep.
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
# oracle sample per degree for the CPU baseline (at least four elements per
# host core at every degree; a few seconds of host work each)
CPU_SAMPLE = {1: 200000, 2: 20000, 3: 2000, 4: 300, 5: 64, 6: 64, 7: 64}
# ALU peaks derived from unit counts and clocks (152 SMs x 2.07 GHz), used
# only when the FMA probe cannot run:
PEAK_F32 = 152 * 2.07e9 * 128 * 2 / 1e12   # 128 FP32 lanes per SM: 80.5 TFLOP/s
PEAK_F64 = 152 * 2.07e9 * 2 * 2 / 1e12     # 2 FP64 FMA per SM per clock: 1.26 TFLOP/s
HBM_FALLBACK, BF16_FALLBACK = 6800.0, 1900.0
# DRAM bytes (read + write) per launch of the dominant kernel, from one ncu
# capture of the full-size FP64 p = 7 launch (dram__bytes_read.sum +
# dram__bytes_write.sum of fma_kernel_pair2<double>, 3004 prisms, mirrored
# tile pairs)
TRAFFIC = {("f64", 7): 53.60e6 + 1.9698e9}
TRAFFIC_SOURCE = ("ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none "
                  "-k regex:fma_kernel -s 6 -c 1 of the full-size FP64 p=7 launch "
                  "(bench.py --steps 1 --warmup 1 --no-cpu --no-e2e --no-extras)")


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), float(d["bf16_tflops"]), "measured"
    except Exception:
        return HBM_FALLBACK, BF16_FALLBACK, "fallback"


def measure_fma_peaks(lib, dev, stream, sm_mhz=2070.0):
    """FP64 and FP32 multiply-add throughput measured with the library's FMA
    probe, the better of its two loop forms (independent chains; the
    contraction's inner loop, register-tile outer products fed from shared
    memory), 8 CTAs of 256 threads per SM, launches of about 50 ms (best of 3
    after a warm-up launch, CUDA events on the launching stream).  Each CTA records its SM clock cycles, so the
    probe gives multiply-adds per SM per clock; the peak (TFLOP/s, a
    multiply-add = 2 flops) is that rate at sm_mhz, the SM clock the
    measured kernels ran at (the probe itself may run at a lower,
    power-capped clock)."""
    import torch
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    n = sms * 8 * 256
    out = torch.empty(n, dtype=torch.float64, device=dev)
    clk = torch.zeros((n // 256, 2), dtype=torch.int64, device=dev)
    res = {"sm_mhz_used": sm_mhz}
    # (form, iterations, multiply-adds per thread and iteration): chains, outer products
    forms = {"f64": ((0, 12000, 8), (1, 200, 32 * 16)), "f32": ((0, 800000, 8), (1, 3200, 32 * 64))}
    for name, fp64 in (("f64", True), ("f32", False)):
        best = None
        for form, iters, per_it in forms[name]:
            for rep in range(4):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                lib.fem_probe_fma(fp64, form, iters, n, out, clk, stream)
                e1.record(stream)
                e1.synchronize()
                if rep:
                    s = e0.elapsed_time(e1) / 1e3
                    c = clk.double()
                    mhz = float((c[:, 0] / c[:, 1]).mean()) * 1e3
                    fmas = float(per_it) * iters * n
                    per_clk = fmas / (s * mhz * 1e6) / sms
                    if best is None or per_clk > best[0]:
                        best = (per_clk, 2.0 * fmas / s / 1e12, mhz, form)
        res[name] = 2.0 * best[0] * sms * sm_mhz * 1e6 / 1e12
        res[name + "_fma_per_sm_clk"] = round(best[0], 3)
        res[name + "_probe_tflops"] = round(best[1], 4)
        res[name + "_probe_mhz"] = round(best[2], 1)
        res[name + "_probe_form"] = "chains" if best[3] == 0 else "outer products"
    return res


def ns_of(p):
    return (p + 1) ** 2 * (p + 2) // 2


def geom_fp64_ops(p):
    """FP64 operations (a multiply-add = 1) of the prism geometry per element
    in the FP32 and tensor-core paths: adj J rows 0, 1 and det J per point
    (15), the zeta-level factors J[:,0], J[:,1], adj row 2 (18 per level),
    J[:,2] per triangle point (12) and the edge record (21)."""
    N = p + 1
    return 15 * N ** 3 + 18 * N + 12 * N * N + 21


def nq_of(p):
    return (p + 1) ** 3


def flops_per_elem(p):
    """Algorithmic flops per element: 8 NQ NS^2 (contraction) + 2 NQ NS (load
    vector) + 32 NQ NS (weighted tile, dense 4x4 count) + 150 NQ (geometry)."""
    n, q = ns_of(p), nq_of(p)
    return 8 * q * n * n + 2 * q * n + 32 * q * n + 150 * q


# Output tiles (or, with one tile, micro-tiles) per side of the FMA kernels'
# shapes that take mirrored pairs (the tile below the diagonal from the one
# above it plus the antisymmetric convection part, a contraction over 2 NQ
# instead of 4 NQ): FP64 p = 4 and 5 (25 x 25 and 21 x 21 micro-tiles of one
# tile), p = 6 (two tiles of 98) and p = 7 (three of 96), FP32 p = 7.
MIRROR_TILES = {8: {4: 25, 5: 21, 6: 2, 7: 3}, 4: {7: 3}}


def executed_flops_per_elem(p, osz):
    """Flops the kernel executes per element: the algorithmic count with the
    contraction term scaled by the mirrored pairs' share of the dense work,
    (T (T + 1) / 2 full tiles + T (T - 1) / 2 half tiles) / T^2."""
    t = MIRROR_TILES.get(osz, {}).get(p)
    if not t:
        return flops_per_elem(p)
    n, q = ns_of(p), nq_of(p)
    ratio = (t * (t + 1) / 2 * 4 + t * (t - 1) / 2 * 2) / (4 * t * t)
    return flops_per_elem(p) - 8 * q * n * n * (1 - ratio)


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
        X = inputs.prism_mesh(sweep[p])[:n]
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


def sweep_config(sweep, precision):
    """The workload description shared by both arms' JSON lines."""
    return {"workload": "prism degree sweep p=1..7 (jittered prisms, random SPD D, b, c, f), E_p=%s"
                        % list(sweep.values()),
            "precision": precision, "layout": "full",
            "l2": "flushed between timed steps (256 MB write)",
            "sharding": "per rank E_p prisms: rank r integrates prisms r E_p .. (r+1) E_p - 1 "
                        "of an (N E_p)-prism mesh; no data-path collective"}


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    sweep = dict(SWEEP_E)
    t0 = time.perf_counter()
    vals = []
    cb = None
    for _ in range(max(1, args.steps)):
        cb = cpu_baseline(sweep)
        vals.append(cb["value"])
    el = time.perf_counter() - t0
    v = statistics.median(vals)
    units = sum(sweep.values())
    line = {"impl": "reference", "metric": "element matrices/s (prism sweep p=1..7)", "value": v,
            "unit": "element matrices/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": units / v * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": sweep_config(sweep, "f64"),
            "cpu_baseline": dict(cb, value=v),
            "e2e": {"value": v, "unit": "element matrices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0},
            "wall_s": el}
    print(json.dumps(line), flush=True)


def _timed(stream, fn, reps, warm=1):
    """Device time (ms) per call of fn on stream: warm-up calls, then reps calls
    bracketed by CUDA events."""
    import torch
    for _ in range(warm):
        with torch.cuda.stream(stream):
            fn()
    stream.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    with torch.cuda.stream(stream):
        for _ in range(reps):
            fn()
    e1.record(stream)
    e1.synchronize()
    return e0.elapsed_time(e1) / reps


def measure_sweep(lib, tables, sweep, data, prec, stream, steps, warmup, flush):
    """Per-step and per-degree device times of the sweep."""
    import torch

    def step(events=None):
        with torch.cuda.stream(stream):
            for p, d in data.items():
                if events is not None:
                    events[p][0].record(stream)
                lib.fem_integrate_uniform(tables, p, sweep[p], d["X"], d["C"], sweep[p], prec,
                                  lib.FEM_OUT_FULL, d["A"], d["b"], d["st"], stream)
                if events is not None:
                    events[p][1].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    per_p = {p: [] for p in sweep}
    step_ms = []
    for _ in range(steps):
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
    return step_ms, {p: statistics.mean(v) for p, v in per_p.items()}


def per_degree_table(sweep, mean_p, osz, peak, hbm, fp64_peak=None):
    """Per degree: time, rate and the fraction of the roofline time, the
    largest of the contraction at its ALU peak, the bytes at the HBM peak and
    (FP32 path, fp64_peak given) the FP64 geometry at the FP64 pipe rate."""
    out = {}
    for p in sweep:
        t_s = mean_p[p] / 1e3
        tf = flops_per_elem(p) * sweep[p] / t_s / 1e12
        gbs = bytes_per_elem(p, osz) * sweep[p] / t_s / 1e9
        terms = {"alu": flops_per_elem(p) / (peak * 1e12), "hbm": bytes_per_elem(p, osz) / (hbm * 1e9)}
        if fp64_peak:
            terms["fp64_geometry"] = geom_fp64_ops(p) / (fp64_peak / 2 * 1e12)
        bound = max(terms, key=terms.get)
        out[str(p)] = {"elements": sweep[p], "ms": round(mean_p[p], 4), "elem_per_s": sweep[p] / t_s,
                       "tflops": round(tf, 3), "gbs": round(gbs, 1),
                       "roofline_frac": round(terms[bound] * sweep[p] / t_s, 4), "bound": bound}
        ex = executed_flops_per_elem(p, osz)
        if ex < flops_per_elem(p):  # mirrored tile pairs: less work than the algorithmic count
            out[str(p)]["executed_work_ratio"] = round(ex / flops_per_elem(p), 4)
            out[str(p)]["executed_alu_frac"] = round(ex / (peak * 1e12) * sweep[p] / t_s, 4)
    return out


def shard_inputs(E, rank=0, world=1):
    """Inputs of one rank under weak scaling: the whole mesh has world * E
    prisms and rank r integrates prisms r E .. (r+1) E - 1 (coordinates and
    coefficients generated for that slice only; world = 1: the E-prism mesh)."""
    if world == 1:
        return inputs.prism_mesh(E), inputs.coefficients(E)
    dims = inputs.prism_grid_dims(world * E)
    return inputs.prism_mesh(E, dims=dims, first=rank * E), inputs.coefficients(E, first=rank * E)


def max_over_ranks(x, world):
    """Largest value of x over the ranks (x itself for one rank)."""
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(x)], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def make_sweep_data(sweep, dev, dt, host=None, rank=0, world=1):
    """Device inputs/outputs of the sweep (this rank's shard); host arrays
    generated once and reused."""
    import torch
    data = {}
    for p, E in sweep.items():
        if host is not None and p in host:
            X, C = host[p]
        else:
            X, C = shard_inputs(E, rank, world)
            if host is not None:
                host[p] = (X, C)
        n = ns_of(p)
        data[p] = dict(X=torch.from_numpy(X).to(dev), C=torch.from_numpy(C).to(dev),
                       A=torch.empty((E, n * n), dtype=dt, device=dev),
                       b=torch.empty((E, n), dtype=dt, device=dev),
                       st=torch.empty((E,), dtype=torch.int32, device=dev), Xh=X, Ch=C)
    return data


def measure_e2e(lib, tables, sweep, data, prec, steps, world=1):
    """The sweep through fem_integrate_host: pinned host inputs/outputs, copies
    in the timed region."""
    import torch
    dt = torch.float64 if prec == lib.FEM_F64 else torch.float32
    host = {}
    h2d = d2h = 0
    for p, d in data.items():
        host[p] = dict(X=torch.from_numpy(d["Xh"]).pin_memory(),
                       C=torch.from_numpy(d["Ch"]).pin_memory(),
                       A=torch.empty(tuple(d["A"].shape), dtype=dt).pin_memory(),
                       b=torch.empty(tuple(d["b"].shape), dtype=dt).pin_memory())
        h2d += host[p]["X"].numel() * 8 + host[p]["C"].numel() * 8
        d2h += (host[p]["A"].numel() + host[p]["b"].numel()) * host[p]["A"].element_size()
    for p, h in host.items():  # warm-up (staging allocation)
        lib.fem_integrate_host(tables, p, min(sweep[p], 1000), h["X"], h["C"], sweep[p], prec,
                               lib.FEM_OUT_FULL, h["A"], h["b"])
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        for p, h in host.items():
            lib.fem_integrate_host(tables, p, sweep[p], h["X"], h["C"], sweep[p], prec,
                                   lib.FEM_OUT_FULL, h["A"], h["b"])
    el = max_over_ranks(time.perf_counter() - t0, world)
    return {"value": world * sum(sweep.values()) * steps / el, "unit": "element matrices/s",
            "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "steps": steps,
            "path": "fem_integrate_host (C ABI, pinned host buffers, 2-slot copy/compute pipeline)"}


# ---------------------------------------------------------------- other workloads

def wl_tets(lib, stream, dev, reps):
    import torch
    X = inputs.tet_mesh(16)
    E = X.shape[0]
    C = inputs.coefficients(E, kind="laplace")
    t = lib.fem_tables_build(lib.FEM_TET4, 1, 1)
    Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
    A = torch.empty((E, 16), dtype=torch.float64, device=dev)
    b = torch.empty((E, 4), dtype=torch.float64, device=dev)
    ms = _timed(stream, lambda: lib.fem_integrate_uniform(t, 1, E, Xd, Cd, E, 0, 0, A, b, None, stream), reps, 3)
    vol = float(b.sum().item())
    t.close()
    return {"workload": "P1 tets, unit cube 16^3 x 6 = 24576 elements, Laplace, FP64",
            "ms": round(ms, 4), "elem_per_s": E / ms * 1e3, "sum_b": vol}


def wl_tensor(lib, tables, stream, dev, reps, bf16_peak, E=200000, degrees=(4, 5, 6, 7), hbm=HBM_FALLBACK,
              fp64_peak=PEAK_F64):
    """Tensor-core forms at p = 4..7, 200k prisms each; errors against the GPU
    FP64 path (itself within 1e-12 of the oracle) on the first 512 elements."""
    import torch
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
    out = {}
    S = min(512, E)
    for p in degrees:
        n = ns_of(p)
        A64 = torch.empty((S, n * n), dtype=torch.float64, device=dev)
        lib.fem_integrate_uniform(tables, p, S, Xd, Cd, E, 0, 0, A64, None, None, stream)
        stream.synchronize()
        ref = A64.view(S, n, n)
        A = torch.empty((E, n * n), dtype=torch.float32, device=dev)
        b = torch.empty((E, n), dtype=torch.float32, device=dev)
        row = {}
        for name, prec in (("bf16x3", lib.FEM_BF16X3), ("f16x3", lib.FEM_F16X3)):
            ms = _timed(stream, lambda: lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, prec, 0, A, b, None,
                                                          stream), reps)
            err = ((A[:S].double().view(S, n, n) - ref).flatten(1).norm(dim=1) /
                   ref.flatten(1).norm(dim=1)).cpu().numpy()
            fl = 8.0 * nq_of(p) * n * n * E
            terms = {"tensor_x3": 3 * fl / (bf16_peak * 1e12), "hbm": bytes_per_elem(p, 4) * E / (hbm * 1e9),
                     "fp64_geometry": geom_fp64_ops(p) * E / (fp64_peak / 2 * 1e12)}
            bound = max(terms, key=terms.get)
            row[name] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3,
                         "alg_tflops": round(fl / ms / 1e9, 1),
                         "hw_tflops_x3": round(3 * fl / ms / 1e9, 1),
                         "frac_of_bf16_peak_x3": round(3 * fl / ms / 1e9 / bf16_peak, 4),
                         "roofline_frac": round(terms[bound] / (ms / 1e3), 4), "bound": bound,
                         "err_max": float(err.max()), "err_median": float(np.median(err))}
        ms32 = _timed(stream, lambda: lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, 1, 0, A, b, None,
                                                        stream), 1)
        row["f32_fma"] = {"ms": round(ms32, 3), "elem_per_s": E / ms32 * 1e3}
        out[str(p)] = row
        del A, b, A64
        torch.cuda.empty_cache()
    return {"workload": "prisms p=4..7, 200000 elements per degree, full A_e + b_e (FP32 out)",
            "per_degree": out, "error_reference": "GPU FP64 path, first 512 elements"}


def wl_elastic(lib, tables, stream, dev, reps, scale_down=1, degrees=range(1, 8)):
    """Linear elastostatics (the paper's model problem), about 2 GB of FP64
    output per degree; FP64, FP32 and the BF16x3 / FP16x3 tensor-core forms.  GFLOP/s also in the paper's count of
    63 flops per 3x3 block and point (63 NQ NS^2 per element)."""
    import torch
    out = {}
    for p in degrees:
        n = ns_of(p)
        E = max(1, round(2e9 / (8 * (9 * n * n + 3 * n))) // scale_down)
        X = inputs.prism_mesh(E)
        C = inputs.elastic_coefficients(E)
        Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
        row = {"elements": E}
        S = min(E, 64)
        ref = None
        for name, prec, dt in (("f64", lib.FEM_F64, torch.float64), ("f32", lib.FEM_F32, torch.float32),
                               ("bf16x3", lib.FEM_BF16X3, torch.float32), ("f16x3", lib.FEM_F16X3, torch.float32)):
            A = torch.empty((E, 9 * n * n), dtype=dt, device=dev)
            b = torch.empty((E, 3 * n), dtype=dt, device=dev)
            ms = _timed(stream, lambda: lib.fem_integrate_elastic(tables, p, E, Xd, Cd, E, prec, A, b, None,
                                                                  stream), reps)
            alg = 9 * 6.0 * nq_of(p) * n * n  # 9 blocks, K = 3 NQ
            row[name] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3,
                         "tflops": round(alg * E / ms / 1e9, 3),
                         "paper_count_gflops": round(63.0 * nq_of(p) * n * n * E / ms / 1e6, 1)}
            if ref is None:
                ref = A[:S].clone()
            else:
                row[name]["err_max_vs_f64"] = float(((A[:S].double() - ref).norm(dim=1) / ref.norm(dim=1)).max())
            del A, b
        out[str(p)] = row
        torch.cuda.empty_cache()
    return {"workload": "linear elastostatics, isotropic E U[1,10], nu U[0.05,0.45], body force; "
                        "prisms, about 2 GB FP64 output per degree; A^e[3][3][NS][NS] + b^e[3][NS]",
            "per_degree": out}


# FP64 pipe rate of GB300: 2 FP64 operations per clock per SM (a multiply-add
# is one), 152 SMs at 2.07 GHz; the 1.26 TFLOP/s FP64 peak counts each
# multiply-add as 2 flops
FP64_PIPE_GOPS = 2 * 152 * 2.07


def apply_fp64_ops(p):
    """FP64 operations per element of the FP64 apply kernel (multiply-add = 1),
    counted from its loops: zeta contractions and the transposed b-direction
    sums (4 N NS each), the b-direction sums per column (N^2 (4 NT - N)), the
    a-direction sums both ways (2 NQ (5 N - 2)), 57 per point for adj J, det J
    and v = G_Q u, and the element's geometry factors (33 N + 18 N^2 + 29)."""
    N = p + 1
    NT, NQ = N * (N + 1) // 2, N ** 3
    NS = NT * N
    return 8 * N * NS + N * N * (4 * NT - N) + 2 * NQ * (5 * N - 2) + 57 * NQ + 33 * N + 18 * N * N + 29


def wl_apply(lib, tables, stream, dev, reps, hbm, scale_down=1, degrees=range(1, 8)):
    """Matrix-free operator apply y_e = A_e x_e (fem_apply), prisms p = 1..7,
    about 1 GB of algorithmic FP64 traffic per degree (x and y, coordinates,
    11 coefficients, status), every operand larger than L2.  HBM roofline per
    degree; the FP64 result is checked against the formed matrices
    (fem_integrate FP64, then A_e x_e) on the first elements, FP32 against FP64."""
    import torch
    out = {}
    for p in degrees:
        n = ns_of(p)
        E = max(1, round(1e9 / (8 * (2 * n + 29))) // scale_down)
        X = inputs.prism_mesh(E)
        C = inputs.coefficients(E)
        x = inputs.dof_vectors(E, n)
        Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
        st = torch.empty(E, dtype=torch.int32, device=dev)
        row = {"elements": E}
        S = min(E, 32)
        y64 = None
        for name, prec, dt, osz in (("f64", lib.FEM_F64, torch.float64, 8), ("f32", lib.FEM_F32, torch.float32, 4)):
            xd = torch.from_numpy(x).to(dev, dt)
            y = torch.empty_like(xd)
            ms = _timed(stream, lambda: lib.fem_apply(tables, p, E, Xd, Cd, E, prec, xd, y, st, stream), reps)
            nbytes = (2 * osz * n + 8 * 29 + 4) * E
            gbs = nbytes / ms / 1e6
            row[name] = {"ms": round(ms, 4), "elem_per_s": E / ms * 1e3, "gbs": round(gbs, 1),
                         "hbm_frac": round(gbs / hbm, 4)}
            if prec == lib.FEM_F64:
                gops = apply_fp64_ops(p) * E / ms / 1e6
                row[name]["fp64_ops_per_elem"] = apply_fp64_ops(p)
                row[name]["roofline"] = {"bound": "alu", "achieved": round(gops, 1), "peak": FP64_PIPE_GOPS,
                                         "unit": "G FP64 ops/s", "frac": round(gops / FP64_PIPE_GOPS, 4)}
            if y64 is None:
                y64 = y[:S].clone()
                A = torch.empty((S, n * n), dtype=torch.float64, device=dev)
                lib.fem_integrate_uniform(tables, p, S, Xd, Cd, E, lib.FEM_F64, lib.FEM_OUT_FULL, A, None, None, stream)
                stream.synchronize()
                yf = torch.bmm(A.view(S, n, n), xd[:S].unsqueeze(2)).squeeze(2)
                row[name]["err_max_vs_formed"] = float(((y64 - yf).norm(dim=1) / yf.norm(dim=1)).max())
                del A
            else:
                row[name]["err_max_vs_f64"] = float(((y[:S].double() - y64).norm(dim=1) / y64.norm(dim=1)).max())
            row[name]["flagged"] = int((st != 0).sum().item())
            del xd, y
        out[str(p)] = row
        del Xd, Cd, st
        torch.cuda.empty_cache()
    return {"workload": "matrix-free operator apply y_e = A_e x_e (sum factorisation), jittered prisms, "
                        "random D/b/c, x_e ~ U[-1,1]; about 1 GB of FP64 traffic per degree",
            "per_degree": out}


def _copy_ms(stream, pairs, reps=2):
    """Device time (ms) of the host<->device copies dst.copy_(src) in pairs."""
    return _timed(stream, lambda: [d.copy_(s, non_blocking=True) for d, s in pairs], reps)


NTRI_TABLE1 = {1: 3, 2: 6, 3: 12, 4: 16, 5: 25, 6: 33, 7: 42}


def flops_per_elem_rule(p, nq):
    """flops_per_elem with a rule of nq points."""
    n = ns_of(p)
    return 8 * nq * n * n + 2 * nq * n + 32 * nq * n + 150 * nq


def wl_table1(lib, stream, dev, reps, fma, hbm, bf16_peak, scale_down=1, degrees=range(1, 8),
              collapsed_ms=None):
    """The paper's prism rules (Table 1: N_Q = (p+1) x 3 ... 42 points, a
    symmetric degree-2p triangle rule x Gauss-Legendre) at the sweep's element
    counts, FP64, FP32 and BF16x3, with the same roofline terms as the sweep
    (counted with the rule's N_Q); collapsed_ms: {precision: {p: ms}} of the
    collapsed rule's runs for the speed ratio."""
    import torch
    t1 = lib.fem_tables_build_ex(lib.FEM_PRISM6, lib.FEM_RULE_TABLE1, 1, 7)
    out = {}
    for p in degrees:
        E = max(1, SWEEP_E[p] // scale_down)
        n, q = ns_of(p), (p + 1) * NTRI_TABLE1[p]
        X, C = inputs.prism_mesh(E), inputs.coefficients(E)
        Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
        row = {"elements": E, "nq": q, "nq_collapsed": (p + 1) ** 3,
               "work_ratio_collapsed_over_table1": round((p + 1) ** 3 / q, 3)}
        for name, prec, dt in (("f64", lib.FEM_F64, torch.float64), ("f32", lib.FEM_F32, torch.float32),
                               ("bf16x3", lib.FEM_BF16X3, torch.float32)):
            A = torch.empty((E, n * n), dtype=dt, device=dev)
            b = torch.empty((E, n), dtype=dt, device=dev)
            ms = _timed(stream, lambda: lib.fem_integrate_uniform(t1, p, E, Xd, Cd, E, prec, lib.FEM_OUT_FULL, A, b,
                                                                  None, stream), reps)
            fl = flops_per_elem_rule(p, q)
            osz = 8 if prec == lib.FEM_F64 else 4
            terms = {"hbm": bytes_per_elem(p, osz) * E / (hbm * 1e9)}
            if name == "bf16x3":
                terms["tensor_x3"] = 3 * 8.0 * q * n * n * E / (bf16_peak * 1e12)
            else:
                terms["alu"] = fl * E / ((fma["f64"] if name == "f64" else fma["f32"]) * 1e12)
            if name != "f64":
                terms["fp64_geometry"] = (15 * q + 18 * (p + 1) + 12 * NTRI_TABLE1[p] + 21) * E / (fma["f64"] / 2 * 1e12)
            bound = max(terms, key=terms.get)
            r = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3, "tflops": round(fl * E / ms / 1e9, 3),
                 "roofline_frac": round(terms[bound] / (ms / 1e3), 4), "bound": bound}
            if collapsed_ms and name in collapsed_ms and p in collapsed_ms[name]:
                r["speedup_vs_collapsed"] = round(collapsed_ms[name][p] / ms, 3)
            row[name] = r
            del A, b
        out[str(p)] = row
        torch.cuda.empty_cache()
    # the paper's model problem with its own rule: linear elastostatics, about
    # 2 GB of FP64 output per degree; GFLOP/s also in the paper's count (63
    # flops per 3x3 block and point, 63 N_Q NS^2 per element)
    el = {}
    for p in degrees:
        n, q = ns_of(p), (p + 1) * NTRI_TABLE1[p]
        E = max(1, round(2e9 / (8 * (9 * n * n + 3 * n))) // scale_down)
        X, C = inputs.prism_mesh(E), inputs.elastic_coefficients(E)
        Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
        row = {"elements": E, "nq": q}
        for name, prec, dt in (("f64", lib.FEM_F64, torch.float64), ("f32", lib.FEM_F32, torch.float32),
                               ("bf16x3", lib.FEM_BF16X3, torch.float32)):
            A = torch.empty((E, 9 * n * n), dtype=dt, device=dev)
            b = torch.empty((E, 3 * n), dtype=dt, device=dev)
            ms = _timed(stream, lambda: lib.fem_integrate_elastic(t1, p, E, Xd, Cd, E, prec, A, b, None, stream),
                        reps)
            row[name] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3,
                         "tflops": round(9 * 6.0 * q * n * n * E / ms / 1e9, 3),
                         "paper_count_gflops": round(63.0 * q * n * n * E / ms / 1e6, 1)}
            del A, b
        el[str(p)] = row
        torch.cuda.empty_cache()
    t1.close()
    return {"workload": "prism degree sweep with the paper's rules (Table 1 N_Q = 6, 18, 48, 80, 150, 231, 336), "
                        "same element counts, coefficients and outputs as the headline sweep; and linear "
                        "elastostatics with that rule (about 2 GB of FP64 output per degree)",
            "per_degree": out, "elasticity": el}


def wl_split(lib, tables, stream, dev, reps, scale_down=1, degrees=range(1, 8)):
    """Split geometry (the paper's NOJAC variants: det J and J^{-1} per point
    stored, then read) against the fused kernels (JAC), FP64, at the sweep's
    element counts; and the per-stage host<->device times of the paper's
    Tables 6/7 (pinned host buffers, over NVLink-C2C)."""
    import torch
    out = {}
    for p in degrees:
        E = max(1, SWEEP_E[p] // scale_down)
        n, q = ns_of(p), nq_of(p)
        X, C = inputs.prism_mesh(E), inputs.coefficients(E)
        Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
        A = torch.empty((E, n * n), dtype=torch.float64, device=dev)
        b = torch.empty((E, n), dtype=torch.float64, device=dev)
        T = torch.empty((E, q, 10), dtype=torch.float64, device=dev)
        st = torch.empty((E,), dtype=torch.int32, device=dev)
        F, L = lib.FEM_F64, lib.FEM_OUT_FULL
        fused = _timed(stream, lambda: lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, F, L, A, b, st, stream), reps)
        A_ref = A[:: max(1, E // 64)].clone()
        terms = _timed(stream, lambda: lib.fem_jacobian_terms(tables, p, E, Xd, T, st, stream), reps)
        nojac = _timed(stream, lambda: lib.fem_integrate_terms(tables, p, E, T, Cd, E, F, L, A, b, st, stream),
                       reps)
        stream.synchronize()
        dev_rel = float(((A[:: max(1, E // 64)] - A_ref).norm() / A_ref.norm()).item())
        Xh, Ch = torch.from_numpy(X).pin_memory(), torch.from_numpy(C).pin_memory()
        Th = torch.empty(T.shape, dtype=T.dtype).pin_memory()
        Ah = torch.empty(A.shape, dtype=A.dtype).pin_memory()
        bh = torch.empty(b.shape, dtype=b.dtype).pin_memory()
        h2d_jac = _copy_ms(stream, [(Xd, Xh), (Cd, Ch)])
        h2d_nojac = _copy_ms(stream, [(T, Th), (Cd, Ch)])
        d2h = _copy_ms(stream, [(Ah, A), (bh, b)])
        init = _timed(stream, lambda: (A.zero_(), b.zero_()), 2)
        tb = E * q * 80
        out[str(p)] = {
            "elements": E,
            "fused_jac_ms": round(fused, 3), "terms_pass_ms": round(terms, 3),
            "nojac_integrate_ms": round(nojac, 3), "nojac_total_ms": round(terms + nojac, 3),
            "nojac_over_jac": round((terms + nojac) / fused, 3),
            "nojac_integrate_over_jac": round(nojac / fused, 3),
            "terms_bytes": tb, "terms_pass_gbs": round((tb + E * 144) / terms / 1e6, 1),
            "max_rel_diff_nojac_vs_jac": dev_rel,
            "stages_ms": {"input_transfer_jac": round(h2d_jac, 3), "input_transfer_nojac": round(h2d_nojac, 3),
                          "output_memory_init": round(init, 3), "output_transfer": round(d2h, 3)},
        }
        del Xd, Cd, A, b, T, st, Xh, Ch, Th, Ah, bh, A_ref
        torch.cuda.empty_cache()
    return {"workload": "prism degree sweep element counts, FP64, full A_e + b_e; JAC = fused geometry, "
                        "NOJAC = device terms pass (det J, J^-1 per point, 80 B) + integration reading them; "
                        "stages: pinned host buffers <-> HBM",
            "per_degree": out}


def wl_batched(lib, tables, stream, dev, reps, E=500000):
    import torch
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    P = inputs.mixed_degrees(E)
    Xd, Cd = torch.from_numpy(X).to(dev), torch.from_numpy(C).to(dev)
    offA, offb, totA, totb = lib.fem_output_offsets(lib.FEM_PRISM6, P, 0)
    A = torch.empty(totA, dtype=torch.float32, device=dev)
    b = torch.empty(totb, dtype=torch.float32, device=dev)
    # error sample: the first elements of each degree, against the FP32 result
    sample = [int(np.flatnonzero(P == p)[k]) for p in range(1, 8) for k in range(8)]
    res, ref = {}, None
    for name, prec, flags in (("graph_autotuned", lib.FEM_F32, lib.FEM_PLAN_AUTOTUNE),
                              ("per_degree_loop", lib.FEM_F32, lib.FEM_PLAN_LOOP),
                              ("per_degree_loop_autotuned", lib.FEM_F32, lib.FEM_PLAN_LOOP | lib.FEM_PLAN_AUTOTUNE),
                              ("graph_concurrent_branches", lib.FEM_F32, lib.FEM_PLAN_CONCURRENT),
                              ("graph_concurrent_bf16x3", lib.FEM_BF16X3, lib.FEM_PLAN_CONCURRENT),
                              ("graph_concurrent_bf16x3_autotuned", lib.FEM_BF16X3,
                               lib.FEM_PLAN_CONCURRENT | lib.FEM_PLAN_AUTOTUNE),
                              ("graph_concurrent_f16x3", lib.FEM_F16X3, lib.FEM_PLAN_CONCURRENT)):
        plan = lib.fem_plan_create(tables, P, prec, 0, flags, None)
        ms = _timed(stream, lambda: lib.fem_plan_execute(plan, Xd, Cd, E, A, b, None, stream), reps, 2)
        res[name] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3,
                     "variants": [plan.variant(p)[0] for p in range(1, 8)]}
        if flags & lib.FEM_PLAN_AUTOTUNE:  # the autotuner's candidate times per degree (ms)
            res[name]["tuned_ms"] = {str(p): [round(float(x), 3) for x in plan.variant(p)[1]] for p in range(1, 8)}
        stream.synchronize()
        blocks = [A[int(offA[e]):int(offA[e]) + ns_of(int(P[e])) ** 2].double() for e in sample]
        if ref is None:
            ref = blocks
        else:
            res[name]["err_max_vs_f32"] = max(float((x - r).norm() / r.norm()) for x, r in zip(blocks, ref))
        plan.close()
    return {"workload": "500000 prisms, seeded degrees p=1..7 (weights .25 .2 .15 .15 .1 .1 .05), FP32 outputs; "
                        "variants per degree: 0/1 persistent shapes, 2 uniform-degree FP32 kernel, 3 tensor cores",
            "bins": np.bincount(P, minlength=8)[1:].tolist(), **res}


def wl_surrogate(lib, tables, stream, dev, reps, E=1000000):
    import torch
    p, NS, NQ = 3, 40, 64
    X = inputs.prism_mesh(E)
    C = inputs.coefficients(E)
    U = inputs.field_coefficients(E, NS).astype(np.float32)
    Xd, Cd, Ud = (torch.from_numpy(a).to(dev) for a in (X, C, U))
    pil = torch.empty((20000, NQ, 2), dtype=torch.float32, device=dev)
    lib.fem_field_samples(tables, p, 20000, Xd, Ud, pil, stream)
    stream.synchronize()
    box = lib.fem_box_from_samples(pil.cpu().numpy())
    N = 10_000_000
    us = torch.empty((N, 2), dtype=torch.float32, device=dev)
    k = torch.empty(N, dtype=torch.float32, device=dev)
    lib.fem_law_samples(N, box, inputs.SEED_SURROGATE, us, k, stream)
    m = lib.fem_mlp_create(box, inputs.SEED_SURROGATE)
    t0 = time.perf_counter()
    L1 = lib.fem_mlp_train(m, N, us, k, 5000, 8192, 1e-3, 1, stream=stream)
    L2 = lib.fem_mlp_train(m, N, us, k, 2000, 8192, 3e-4, 2, stream=stream)
    train_s = time.perf_counter() - t0
    A = torch.empty((E, NS * NS), dtype=torch.float32, device=dev)
    b = torch.empty((E, NS), dtype=torch.float32, device=dev)
    st = torch.empty(E, dtype=torch.int32, device=dev)
    S = 256
    A64 = torch.empty((S, NS * NS), dtype=torch.float64, device=dev)
    lib.fem_integrate_law(tables, p, S, Xd, Cd, E, Ud, lib.FEM_LAW_EXACT, None, 0, 0, A64, None, None, stream)
    stream.synchronize()
    ref = A64.view(S, NS, NS)
    res = {}
    for name, fn in (
            ("constant_D", lambda: lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, 1, 0, A, b, st, stream)),
            ("exact_law", lambda: lib.fem_integrate_law(tables, p, E, Xd, Cd, E, Ud, lib.FEM_LAW_EXACT, None,
                                                        1, 0, A, b, st, stream)),
            ("network", lambda: lib.fem_integrate_law(tables, p, E, Xd, Cd, E, Ud, lib.FEM_LAW_MLP, m, 1, 0,
                                                      A, b, st, stream)),
            ("constant_D_bf16x3", lambda: lib.fem_integrate_uniform(tables, p, E, Xd, Cd, E, lib.FEM_BF16X3, 0, A, b, st,
                                                            stream)),
            ("exact_law_bf16x3", lambda: lib.fem_integrate_law(tables, p, E, Xd, Cd, E, Ud, lib.FEM_LAW_EXACT, None,
                                                               lib.FEM_BF16X3, 0, A, b, st, stream)),
            ("network_bf16x3", lambda: lib.fem_integrate_law(tables, p, E, Xd, Cd, E, Ud, lib.FEM_LAW_MLP, m,
                                                             lib.FEM_BF16X3, 0, A, b, st, stream))):
        ms = _timed(stream, fn, reps)
        row = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3}
        if not name.startswith("constant_D"):
            err = ((A[:S].double().view(S, NS, NS) - ref).flatten(1).norm(dim=1) /
                   ref.flatten(1).norm(dim=1)).cpu().numpy()
            row.update(err_max=float(err.max()), err_median=float(np.median(err)))
        if name.startswith("network"):
            row["fallback_elements"] = int(((st & 8) != 0).sum().item())
        res[name] = row
    # the law's cost against the network's: the exact law with more Newton
    # steps (k unchanged once converged), and the network with the hardware
    # tanh approximation; the crossover is the step count at which the
    # exact law costs as much as the network (linear in the steps)
    for prec, tag in ((1, ""), (lib.FEM_BF16X3, "_bf16x3")):
        steps_ms = {8: res["exact_law" + tag]["ms"]}
        for steps in (16, 32):
            law = lib.coef_law(lib.FEM_LAW_EXACT, Ud, newton_steps=steps)
            ms = _timed(stream, lambda: lib.fem_integrate(tables, E, Xd, None, p, Cd, E, law, prec, 0, A, b, st,
                                                          stream), reps)
            steps_ms[steps] = ms
            res["exact_law_newton%d%s" % (steps, tag)] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3}
        law = lib.coef_law(lib.FEM_LAW_MLP, Ud, m, hw_tanh=True)
        ms = _timed(stream, lambda: lib.fem_integrate(tables, E, Xd, None, p, Cd, E, law, prec, 0, A, b, st, stream),
                    reps)
        err = ((A[:S].double().view(S, NS, NS) - ref).flatten(1).norm(dim=1) /
               ref.flatten(1).norm(dim=1)).cpu().numpy()
        res["network_hw_tanh" + tag] = {"ms": round(ms, 3), "elem_per_s": E / ms * 1e3,
                                        "err_max": float(err.max()), "err_median": float(np.median(err))}
        slope = (steps_ms[32] - steps_ms[8]) / 24.0  # ms per Newton step
        for net in ("network", "network_hw_tanh"):
            t_net = res[net + tag]["ms"]
            res["crossover_newton_steps_" + net + tag] = (round(8 + (t_net - steps_ms[8]) / slope, 1)
                                                          if slope > 0 else None)
    m.close()
    return {"workload": "1000000 prisms p=3, FP32, D = k(u, |grad u|) I per point, 40 field "
                        "coefficients per element", "box": [float(x) for x in box],
            "training": {"samples": N, "steps": 7000, "batch": 8192, "seconds": round(train_s, 3),
                         "loss_first": float(L1[:20].mean()), "loss_last": float(L2[-100:].mean())},
            "error_reference": "GPU FP64 path with the exact law, first 256 elements",
            "network_over_exact_time": round(res["network"]["ms"] / res["exact_law"]["ms"], 3),
            "network_over_exact_time_bf16x3": round(res["network_bf16x3"]["ms"] / res["exact_law_bf16x3"]["ms"], 3),
            **res}


def run_only(args):
    """One workload alone (for profiling and quick checks); prints its JSON."""
    import torch

    from paper_1310_1191_gb300 import _lib as lib
    from paper_1310_1191_gb300 import build as _build
    _build.build()
    lib.load()
    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    hbm, bf16_peak, _ = measured_peaks()
    fma = measure_fma_peaks(lib, dev, stream)
    tables = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    reps = args.steps
    if args.only == "tets":
        out = wl_tets(lib, stream, dev, reps)
    elif args.only == "tc":
        degs = tuple(int(x) for x in args.degrees.split(",")) if args.degrees else (4, 5, 6, 7)
        out = wl_tensor(lib, tables, stream, dev, reps, bf16_peak, E=args.elements or 200000, degrees=degs,
                        hbm=hbm, fp64_peak=fma["f64"])
    elif args.only == "mixed":
        out = wl_batched(lib, tables, stream, dev, reps, E=args.elements or 500000)
    elif args.only == "law":
        out = wl_surrogate(lib, tables, stream, dev, reps, E=args.elements or 1000000)
    elif args.only == "elastic":
        degs = tuple(int(x) for x in args.degrees.split(",")) if args.degrees else range(1, 8)
        out = wl_elastic(lib, tables, stream, dev, reps, args.scale_down, degs)
    elif args.only == "apply":
        degs = tuple(int(x) for x in args.degrees.split(",")) if args.degrees else range(1, 8)
        out = wl_apply(lib, tables, stream, dev, reps, hbm, args.scale_down, degs)
    elif args.only == "table1":
        degs = tuple(int(x) for x in args.degrees.split(",")) if args.degrees else range(1, 8)
        out = wl_table1(lib, stream, dev, reps, fma, hbm, bf16_peak, args.scale_down, degs)
    elif args.only == "split":
        degs = tuple(int(x) for x in args.degrees.split(",")) if args.degrees else range(1, 8)
        out = wl_split(lib, tables, stream, dev, reps, args.scale_down, degs)
    else:  # sweep at one precision
        prec = lib.FEM_F64 if args.precision == "f64" else lib.FEM_F32
        dt = torch.float64 if prec == lib.FEM_F64 else torch.float32
        sweep = {p: (max(1, SWEEP_E[p] // args.scale_down)) for p in range(1, 8)}
        if args.degrees:
            sweep = {p: sweep[p] for p in (int(x) for x in args.degrees.split(","))}
        data = make_sweep_data(sweep, dev, dt)
        flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
        step_ms, mean_p = measure_sweep(lib, tables, sweep, data, prec, stream, reps, args.warmup, flush)
        peak = fma["f64"] if prec == lib.FEM_F64 else fma["f32"]
        out = {"elem_per_s": sum(sweep.values()) * reps / (sum(step_ms) / 1e3), "fma_peaks": fma,
               "per_degree": per_degree_table(sweep, mean_p, 8 if prec == lib.FEM_F64 else 4, peak, hbm,
                                              None if prec == lib.FEM_F64 else fma["f64"])}
    print(json.dumps({"only": args.only, "result": out}), flush=True)
    tables.close()


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
    hbm, bf16_peak, peak_src = measured_peaks()
    stream = torch.cuda.Stream(device=dev)
    with Clocks(torch.cuda.current_device()) as pclk:
        try:
            fma = measure_fma_peaks(lib, dev, stream)
            fma_src = "measured"
        except Exception:
            fma, fma_src = {"f64": PEAK_F64, "f32": PEAK_F32}, "derived from unit counts x 2.07 GHz"
    probe_clocks = pclk.summary()
    prec = lib.FEM_F64 if args.precision == "f64" else lib.FEM_F32
    dt = torch.float64 if prec == lib.FEM_F64 else torch.float32
    osz = 8 if prec == lib.FEM_F64 else 4
    sweep = {p: (max(1, SWEEP_E[p] // args.scale_down)) for p in range(1, 8)}
    tables = lib.fem_tables_build(lib.FEM_PRISM6, 1, 7)
    host_inputs = {}
    data = make_sweep_data(sweep, dev, dt, host_inputs, rank, world)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    with Clocks(torch.cuda.current_device()) as clk:
        step_ms, mean_p = measure_sweep(lib, tables, sweep, data, prec, stream, args.steps,
                                        args.warmup, flush)
    torch.cuda.synchronize()
    clocks = clk.summary()
    if fma_src == "measured":  # the probe's rate per SM clock at the sweep's median SM clock
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        f_k = clocks.get("sm_mhz") or 2070.0
        fma["sm_mhz_used"] = f_k
        for k in ("f64", "f32"):
            fma[k] = 2.0 * fma[k + "_fma_per_sm_clk"] * sms * f_k * 1e6 / 1e12
    bad = sum(int((d["st"] != 0).sum().item()) for d in data.values())
    total_ms = sum(step_ms)
    if world > 1:
        total_ms = max_over_ranks(total_ms, world)
        dist.barrier()
    units = sum(sweep.values()) * args.steps * world
    value = units / (total_ms / 1e3)

    peak = fma["f64"] if prec == lib.FEM_F64 else fma["f32"]
    pdom = max(mean_p, key=mean_p.get)
    achieved = flops_per_elem(pdom) * sweep[pdom] / (mean_p[pdom] / 1e3) / 1e12
    per_degree = per_degree_table(sweep, mean_p, osz, peak, hbm,
                                  None if prec == lib.FEM_F64 else fma["f64"])
    e2e = None
    if not args.no_e2e:
        e2e = measure_e2e(lib, tables, sweep, data, prec, args.e2e_steps, world)
    workloads = {}
    collapsed_ms = None
    if rank == 0 and not args.no_extras:
        del data
        torch.cuda.empty_cache()
        reps = 3
        workloads["tets_f64"] = wl_tets(lib, stream, dev, reps)
        if prec == lib.FEM_F64:
            d32 = make_sweep_data(sweep, dev, torch.float32, host_inputs)
            sm32, mp32 = measure_sweep(lib, tables, sweep, d32, lib.FEM_F32, stream, reps, 2, flush)
            workloads["sweep_f32"] = {"elem_per_s": sum(sweep.values()) * reps / (sum(sm32) / 1e3),
                                      "per_degree": per_degree_table(sweep, mp32, 4, fma["f32"], hbm,
                                                                     fma["f64"])}
            collapsed_ms = {"f64": dict(mean_p), "f32": dict(mp32)}
            del d32
            torch.cuda.empty_cache()
        workloads["tensor_core"] = wl_tensor(lib, tables, stream, dev, reps, bf16_peak, hbm=hbm,
                                             fp64_peak=fma["f64"])
        workloads["table1_rules"] = wl_table1(lib, stream, dev, reps, fma, hbm, bf16_peak,
                                              collapsed_ms=collapsed_ms if prec == lib.FEM_F64 else None)
        workloads["mixed_degree"] = wl_batched(lib, tables, stream, dev, reps)
        workloads["nonlinear_law"] = wl_surrogate(lib, tables, stream, dev, reps)
        workloads["elasticity"] = wl_elastic(lib, tables, stream, dev, reps)
        workloads["split_geometry"] = wl_split(lib, tables, stream, dev, 2)
        workloads["operator_apply"] = wl_apply(lib, tables, stream, dev, reps, hbm)
    cb = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cb = cpu_baseline(sweep)
    if rank == 0:
        line = {
            "metric": "element matrices/s (prism sweep p=1..7)", "value": value,
            "unit": "element matrices/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": args.precision, "data": "synthetic",
            "config": sweep_config(sweep, args.precision),
            "gpu_launches": 7 * args.steps,
            "per_degree": per_degree,
            "roofline": {"bound": "alu", "kernel": "fma_kernel p=%d" % pdom,
                         "achieved": round(achieved, 4), "peak": round(peak, 4), "unit": "TFLOP/s",
                         "frac": round(achieved / peak, 4),
                         "executed_work_ratio": round(executed_flops_per_elem(pdom, osz) / flops_per_elem(pdom), 4),
                         "executed_frac": round(achieved / peak * executed_flops_per_elem(pdom, osz)
                                                / flops_per_elem(pdom), 4),
                         "note": "achieved counts the algorithmic flops of the dense contraction; the kernel "
                                 "takes mirrored tile pairs (the tile below the diagonal from the one above "
                                 "plus the antisymmetric convection part) and executes executed_work_ratio of "
                                 "them, so frac can exceed 1; executed_frac is the FP64 pipe's share of the work "
                                 "it does",
                         "traffic": TRAFFIC.get((args.precision, pdom)),
                         "traffic_source": TRAFFIC_SOURCE if (args.precision, pdom) in TRAFFIC else None,
                         "peak_source": "%s FMA peak %s: fem_probe_fma's multiply-adds per SM per clock "
                                        "(the better of independent chains and register-tile outer products from shared "
                                        "memory, 8 CTAs x 256 threads per SM, "
                                        "best of 3 launches of about 50 ms, SM clock from clock64 and "
                                        "globaltimer in every CTA) x SMs x the timed region's median SM "
                                        "clock; HBM %s %.0f GB/s" % (args.precision, fma_src, peak_src, hbm)},
            "fma_peaks": dict(fma, source=fma_src, nvidia_smi_clocks=probe_clocks),
            "flagged_elements": bad,
            "clocks": clocks,
            "e2e": e2e, "cpu_baseline": cb, "workloads": workloads,
        }
        print(json.dumps(line), flush=True)
    tables.close()
    if world > 1:
        dist.destroy_process_group()


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
    ap.add_argument("--no-extras", action="store_true")
    ap.add_argument("--only", choices=["sweep", "tets", "tc", "mixed", "law", "elastic", "split", "apply", "table1"],
                    help="run one workload alone (profiling); prints its own JSON")
    ap.add_argument("--elements", type=int, default=0, help="elements for --only tc/mixed/law")
    ap.add_argument("--degrees", default="", help="comma-separated degrees for --only sweep/tc")
    args = ap.parse_args()
    if args.only:
        run_only(args)
    elif args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
