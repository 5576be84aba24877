"""Benchmark of the cell-wise matrix-free operator library on GB300.

Default workload (one step): Laplace + mass apply with assembly (y = S A x) of degree 4 on a
64^3-cell curved unit cube (sinusoidal vertex displacement of amplitude 0.1 h, metric stored as
7 FP64 values per quadrature point), FP64 storage. The step is the apply kernel followed by the
three DSS axis passes. Inputs (x 262 MB, metric 1.84 GB, y 262 MB) exceed the 129 MB L2, so no
flush is needed between steps.

Extra measurements in the same JSON line: the same workload in FP32 / BF16-metric / BF16, a
degree sweep p=1..7 at ~2^27 cell-wise values (FP64, FP32 and BF16 Laplace), the Poisson CG
time-to-1e-10 (plain FP64 Jacobi-PCG vs FP64 iterative refinement around an FP32 inner CG), the
same Poisson problem solved with the V-cycle-preconditioned CG (FP64 and FP32 cycles), the
multi-block cube in cube (assembled apply with the inter-block DSS, and its Jacobi-PCG solve), and
the batched apply (16 RHS on Q5 64^3 + 48 uneven problems in one persistent launch).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-sweep] [--no-cg]
                  [--no-batched] [--no-mg] [--no-mblock] [--no-mixed] [--no-e2e] [--no-cpu] [--no-tune] [--variant C,S] [--cg-mode M]
                  [--cells N] [--prec P]

--impl reference times the FP64 CPU oracle (explicit element matrices) on a bounded cell sample of
the same workload on the host cores.
"""
import argparse
import json
import os
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402

P, NCELL, KIND = 4, 64, 3
WORKLOAD = "laplace+mass apply+DSS, Q4 (125 DoFs/cell), 5 Gauss pts/dir, 64^3 curved cells, metric 7 x 8 B/qp (FP64 values held as rounded float pairs)"
METRIC = "cell-wise DoF/s of apply at p=2..7 (FP64 vs mixed); CG time-to-1e-10 on 1 GB300"
SWEEP_N = {1: 256, 2: 171, 3: 128, 4: 102, 5: 85, 6: 73, 7: 64}


def flops_per_value(n, kind):
    """Algorithmic FP64-equivalent flops per cell-wise value of the collocation apply on curved
    cells: K: 12n+9 MADs + 2 adds; M: 6n+1 MADs; K+M: 12n+10 MADs + 3 adds."""
    return {1: 24 * n + 20, 2: 12 * n + 2, 3: 24 * n + 23}[kind]


def bytes_per_value(prec, kind):
    """Algorithmic HBM bytes per cell-wise value: read x, write y, read the metric once."""
    vs = {0: 8, 1: 8, 2: 4, 3: 4, 4: 2}[prec]
    gs = {0: 8, 1: 8, 2: 4, 3: 2, 4: 2}[prec]
    nc = {1: 6, 2: 1, 3: 7}[kind]
    return 2 * vs + nc * gs


def peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return d.get("hbm_gbs", 6800.0), "measured"
    return 6800.0, "fallback"


# DRAM bytes per cell of the double-float K+M p=4 apply kernel by variant (cells/CTA, staging):
# dram__bytes_read.sum + dram__bytes_write.sum from one ncu capture per variant of a 40^3-cell case
# (64,000 cells), to be scaled by the cell count of a launch. Variants not listed report null.
DF64_KM_P4_TRAFFIC_PER_CELL = {
    (8, 0): (512.066560e6 + 55.982592e6) / 64000,
    (8, 2): (512.073984e6 + 55.491072e6) / 64000,
    (4, 2): (512.065792e6 + 55.499776e6) / 64000,
}

# FP32 issue-rate roofline for double-float arithmetic: 152 SMs x 128 FP32 lanes x 2.07 GHz,
# 12 FP32 instructions per emulated FP64 multiply-add (2 flops).
DF64_PEAK_TFLOPS = 152 * 128 * 2.07e9 / 12 * 2 / 1e12


class ClockSampler:
    """Samples nvidia-smi SM clocks and throttle reasons while running (for the timed region)."""

    def __init__(self, index=0):
        self.index, self.proc, self.lines = index, None, []

    def __enter__(self):
        q = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.hw_slowdown,"
             "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
             "clocks_event_reasons.sw_power_cap")
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={q}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                self.proc.wait(2)
            except Exception:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 7:
                continue
            try:
                sm.append(float(f[0]))
                mx = float(f[1])
            except ValueError:
                continue
            for nm, v in zip(names, f[3:7]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    return rank, local, world


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(v, world):
    """Largest value over the ranks (step times: the slowest replica sets the job's time)."""
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    dev = "cuda" if dist.get_backend() == "nccl" else "cpu"
    t = torch.tensor([v], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------- oracle error samples ----
class SampleBook:
    """GPU outputs of the timed legs on a seeded sample of cells, kept so that the CPU-oracle leg can
    report each result's error against the FP64 oracle after the GPU work (the oracle is never run
    inside the GPU arm). Every entry is (where in the JSON line, mesh size N, degree p, kind, input
    seed, sampled cells, sampled LOCAL output)."""

    def __init__(self, ncells=48):
        self.ncells = ncells
        self.entries = []

    def cells(self, N, seed):
        rng = np.random.default_rng(1000 + seed)
        E = N ** 3
        pick = rng.choice(E, min(self.ncells, E), replace=False)
        return np.unique(np.concatenate([pick, [0, N - 1, E - N, E - 1]]))

    def add(self, where, N, p, kind, seed, y):
        """y: the LOCAL output of the operator (device tensor, any precision)."""
        import torch
        cells = self.cells(N, p)
        n3 = (p + 1) ** 3
        idx = torch.from_numpy(cells).to(y.device)
        got = y.view(-1, n3).index_select(0, idx).to(torch.float64).cpu().numpy()
        self.entries.append((where, N, p, kind, seed, cells, got))


def oracle_errors(book, out):
    """Relative error max|y - y_oracle| / max|y_oracle| of every sampled output against the oracle's
    LOCAL apply (explicit element matrices) on the same cells and the same input, written beside the
    result it belongs to as ``rel_err_vs_oracle``."""
    import oracle
    oracle.build()
    refs = {}
    for where, N, p, kind, seed, cells, got in book.entries:
        key = (N, p, kind, seed)
        if key not in refs:
            mesh = synth.box_mesh(N, perturb=0.1)
            n3 = (p + 1) ** 3
            ug = synth.global_vector(mesh, p, seed=seed)
            gidx = oracle.global_index(mesh, p).reshape(mesh.ncells, n3)
            x = np.zeros(mesh.ncells * n3)
            x.reshape(mesh.ncells, n3)[cells] = ug[gidx[cells]]
            del gidx, ug
            refs[key] = oracle.apply_local(mesh, p, kind, x, cells)
            del x
        ref = refs[key]
        err = float(np.abs(got - ref).max() / np.abs(ref).max())
        d = out
        for k in where:
            d = d[k]
        d["rel_err_vs_oracle"] = err
        d["oracle_sample_cells"] = int(len(cells))


# ---------------------------------------------------------------------------- GPU arm ----
def event_pair():
    import torch
    return torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)


def time_apply(cw, op, x, y, steps, warmup, stream, assemble=True):
    """Times `steps` steps with events on the launching stream; returns (ms per step, ms per apply
    kernel). A step is one cw_apply call: CW_APPLY_ASSEMBLE (the operator kernel, which also sums the
    x-interfaces inside its tiles, then the remaining DSS passes) or CW_APPLY_LOCAL. The kernel time
    comes from events around CW_APPLY_LOCAL launches of the same kernel on the same buffers, timed
    right after the steps (the assembled launch adds only the in-tile x sums to it)."""
    import torch
    flags = cw.CW_APPLY_ASSEMBLE if assemble else cw.CW_APPLY_LOCAL
    sid = stream.cuda_stream
    for _ in range(warmup):
        cw.cw_apply(op.handle, x, y, flags, stream=sid)
    torch.cuda.synchronize()
    t0, t1 = event_pair()
    ev = [event_pair() for _ in range(steps)]
    with torch.cuda.stream(stream):
        t0.record(stream)
        for _ in range(steps):
            cw.cw_apply(op.handle, x, y, flags, stream=sid)
        t1.record(stream)
        for a, b in ev:
            a.record(stream)
            cw.cw_apply(op.handle, x, y, cw.CW_APPLY_LOCAL, stream=sid)
            b.record(stream)
    torch.cuda.synchronize()
    step_ms = t0.elapsed_time(t1) / steps
    kern_ms = sum(a.elapsed_time(b) for a, b in ev) / steps
    return step_ms, kern_ms


def host_link(xh, yh, x, y, stream, reps=5):
    """Host link rates with whole-vector pinned copies (CUDA events): H2D, D2H and both at once on two
    streams; bound_ms = the bytes of one host-buffer step over the two-way rate."""
    import torch
    s2 = torch.cuda.Stream()

    def timed(fn):
        fn()
        torch.cuda.synchronize()
        a, b = event_pair()
        a.record(stream)
        for _ in range(reps):
            fn()
        b.record(stream)
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    def h2d():
        with torch.cuda.stream(stream):
            x.copy_(xh, non_blocking=True)

    def d2h():
        with torch.cuda.stream(stream):
            yh.copy_(y, non_blocking=True)

    def both():
        ev = torch.cuda.Event()
        ev.record(stream)
        s2.wait_event(ev)
        with torch.cuda.stream(stream):
            x.copy_(xh, non_blocking=True)
        with torch.cuda.stream(s2):
            yh.copy_(y, non_blocking=True)
        ev2 = torch.cuda.Event()
        ev2.record(s2)
        stream.wait_event(ev2)

    nb = x.numel() * x.element_size()
    t_in, t_out, t_both = timed(h2d), timed(d2h), timed(both)
    return {"h2d_gbs": round(nb / t_in / 1e6, 1), "d2h_gbs": round(nb / t_out / 1e6, 1),
            "both_gbs": round(2 * nb / t_both / 1e6, 1), "bound_ms": round(t_both, 3)}


def gpu_arm(args, rank, local, world):
    import torch

    import paper_2607_03413_gb300 as cw
    torch.cuda.set_device(local)
    cw.load()
    hbm, hbm_src = peaks()
    stream = torch.cuda.Stream()
    mesh = synth.box_mesh(args.cells, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, P, KIND, cw.CW_GEOM_METRIC, args.prec)
    n = P + 1
    ug = torch.from_numpy(synth.global_vector(mesh, P, seed=rank)).cuda()
    x = op.gather(ug)
    y = op.empty()
    if args.variant:
        op.set_variant(*[int(v) for v in args.variant.split(",")])
    elif args.tune:
        op.autotune(x, y, reps=3)  # picks cells-per-CTA and TMA staging (before the timed region)
    variant = op.variant()
    torch.cuda.synchronize()

    barrier(world)
    torch.cuda.synchronize()
    with ClockSampler(local) as clk:
        step_ms, kern_ms = time_apply(cw, op, x, y, args.steps, args.warmup, stream)
    barrier(world)
    torch.cuda.synchronize()
    step_ms = max_over_ranks(step_ms, world)
    clocks = clk.summary()
    book = args.book
    if book is not None:
        book.add(("headline",), args.cells, P, KIND, rank, y)  # y holds the LOCAL output after timing
    units = op.L * world
    value = units / (step_ms * 1e-3)

    e2e = None
    if args.e2e:
        # end to end through the C ABI with host buffers: H2D of x, apply + DSS, D2H of y per step
        xh = torch.empty(op.L, dtype=op.vec_dtype, pin_memory=True)
        xh.copy_(x.cpu())
        yh = torch.empty(op.L, dtype=op.vec_dtype, pin_memory=True)

        def e2e_step():  # the public host-buffer entry point: chunked H2D / apply pipeline, DSS, D2H
            cw.cw_apply_host(op.handle, xh, yh, cw.CW_APPLY_ASSEMBLE, stream=stream.cuda_stream)
        for _ in range(args.warmup):
            e2e_step()
        torch.cuda.synchronize()
        barrier(world)
        a, b = event_pair()
        a.record(stream)
        for _ in range(args.steps):
            e2e_step()
        b.record(stream)
        torch.cuda.synchronize()
        e2e_ms = max_over_ranks(a.elapsed_time(b) / args.steps, world)
        e2e = {"value": units / (e2e_ms * 1e-3), "unit": "DoF/s", "ms_per_step": e2e_ms,
               "h2d_bytes_per_step": op.L * x.element_size(), "d2h_bytes_per_step": op.L * x.element_size(),
               "api": "cw_apply_host (pinned host x and y, CW_APPLY_ASSEMBLE)",
               "link": host_link(xh, yh, x, y, stream)}

    fl = flops_per_value(n, KIND) * op.L
    achieved_tflops = fl / (kern_ms * 1e-3) / 1e12
    by = bytes_per_value(0, KIND) * op.L
    traffic = None
    if args.prec == 0 and (variant[0], variant[1]) in DF64_KM_P4_TRAFFIC_PER_CELL:
        traffic = round(DF64_KM_P4_TRAFFIC_PER_CELL[(variant[0], variant[1])] * args.cells ** 3)
    roof = {"bound": "alu", "achieved": round(achieved_tflops, 3), "peak": round(DF64_PEAK_TFLOPS, 3),
            "unit": "TFLOP/s", "frac": round(achieved_tflops / DF64_PEAK_TFLOPS, 4), "traffic": traffic,
            "traffic_note": "bytes per launch, ncu on a 40^3 case of the same variant scaled by cells (null for "
                            "variants not profiled)",
            "kernel": f"apply_metric_kernel_capped<N=5, cells/CTA={variant[0]}, staged={variant[1]}, double-float>",
            "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2.07 GHz / 12 instructions per double-float MAD",
            "hbm": {"achieved": round(by / (kern_ms * 1e-3) / 1e9, 1), "peak": hbm, "unit": "GB/s",
                    "frac": round(by / (kern_ms * 1e-3) / 1e9 / hbm, 4), "peak_source": hbm_src}}
    out = {
        "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64 storage, double-float (f32 pair) arithmetic",
        "data": "synthetic: seeded uniform[-1,1] continuous global vector gathered to cells; curved "
                "64^3 unit-cube mesh (0.1h sinusoidal displacement)",
        "config": {"workload": WORKLOAD, "degree": P, "cells": args.cells ** 3, "cellwise_values": op.L,
                   "kind": "laplace+mass", "assemble": True, "parallelism": f"replicas x{world}",
                   "l2": "inputs larger than L2 (2.4 GB per step), no flush"},
        "apply_kernel_ms": kern_ms,
        "unique_dofs_per_s": (args.cells * P + 1) ** 3 * world / (step_ms * 1e-3),
        "roofline": roof,
        "clocks": clocks,
        "e2e": e2e,
        "gpu_launches": 4 * args.steps,
        "headline": {"what": "the timed step's operator, LOCAL output of the same kernel on the same input"},
    }
    del x, y
    op.close()

    # mixed precision on the same workload
    mixed = {}
    for name, prec in ([("f64_native", cw.CW_PREC_F64_NATIVE), ("f32", cw.CW_PREC_F32),
                        ("f32_bf16metric", cw.CW_PREC_F32_BF16G), ("bf16", cw.CW_PREC_BF16)] if args.mixed else []):
        o = cw.Operator(M, P, KIND, cw.CW_GEOM_METRIC, prec)
        xx = o.gather(ug)
        yy = o.empty()
        o.autotune(xx, yy, reps=3)
        sm, km = time_apply(cw, o, xx, yy, args.steps, args.warmup, stream)
        gbs = bytes_per_value(prec, KIND) * o.L / (km * 1e-3) / 1e9
        mixed[name] = {"dofs_per_s": o.L / (sm * 1e-3), "ms_per_step": sm, "apply_kernel_ms": km,
                       "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4)}
        if book is not None:
            book.add(("mixed", name), args.cells, P, KIND, rank, yy)
        o.close()
    if mixed:
        out["mixed"] = mixed

    # stored vs recomputed metric on the same workload: the recomputed operator reads 21
    # trilinear-map coefficients per cell instead of 7 metric values per quadrature point
    recomp = {}
    for name, prec in ([("f64", cw.CW_PREC_F64), ("f32", cw.CW_PREC_F32), ("bf16", cw.CW_PREC_BF16)]
                       if args.mixed else []):
        o = cw.Operator(M, P, KIND, cw.CW_GEOM_RECOMPUTE, prec)
        xx = o.gather(ug)
        yy = o.empty()
        o.autotune(xx, yy, reps=3)
        sm, km = time_apply(cw, o, xx, yy, args.steps, args.warmup, stream)
        sv = {cw.CW_PREC_F64: 8, cw.CW_PREC_F32: 4, cw.CW_PREC_BF16: 2}[prec]
        sg = 8 if prec == cw.CW_PREC_F64 else 4
        gbs = (2 * sv + 21 * sg / n ** 3) * o.L / (km * 1e-3) / 1e9
        recomp[name] = {"dofs_per_s": o.L / (sm * 1e-3), "ms_per_step": sm, "apply_kernel_ms": km,
                        "hbm_gbs": round(gbs, 1), "hbm_frac": round(gbs / hbm, 4), "variant": o.variant()}
        if book is not None:
            book.add(("recomputed_metric", name), args.cells, P, KIND, rank, yy)
        o.close()
    if recomp:
        out["recomputed_metric"] = recomp

    # the other operator kinds of the same workload (FP64, double-float): stored and recomputed metric
    kinds = {}
    for kname, kind in ((("laplace", cw.CW_LAPLACE), ("mass", cw.CW_MASS)) if args.mixed else ()):
        kinds[kname] = {}
        for gname, geom in (("stored", cw.CW_GEOM_METRIC), ("recomputed", cw.CW_GEOM_RECOMPUTE)):
            o = cw.Operator(M, P, kind, geom, cw.CW_PREC_F64)
            xx = o.gather(ug)
            yy = o.empty()
            o.autotune(xx, yy, reps=3)
            sm, km = time_apply(cw, o, xx, yy, args.steps, args.warmup, stream)
            kinds[kname][gname] = {"dofs_per_s": o.L / (sm * 1e-3), "ms_per_step": sm, "apply_kernel_ms": km}
            if book is not None:
                book.add(("kinds_f64", kname, gname), args.cells, P, kind, rank, yy)
            o.close()
    if kinds:
        out["kinds_f64"] = kinds

    # the small Cartesian case (Q2, 8^3 affine cells, Laplace, FP64): latency per call, LOCAL and
    # ASSEMBLE, back-to-back calls on one stream
    if args.mixed:
        m8 = synth.box_mesh(8)
        M8 = cw.Mesh.from_synth(m8)
        o = cw.Operator(M8, 2, cw.CW_LAPLACE, cw.CW_GEOM_AFFINE, cw.CW_PREC_F64)
        xx = o.gather(torch.from_numpy(synth.global_vector(m8, 2, seed=0)).cuda())
        yy = o.empty()
        lat = {}
        for name, fl in (("local_us", cw.CW_APPLY_LOCAL), ("assemble_us", cw.CW_APPLY_ASSEMBLE)):
            for _ in range(20):
                cw.cw_apply(o.handle, xx, yy, fl, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            a, b = event_pair()
            a.record(stream)
            for _ in range(200):
                cw.cw_apply(o.handle, xx, yy, fl, stream=stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            lat[name] = round(a.elapsed_time(b) / 200 * 1e3, 2)
        out["small_affine"] = {"workload": "Laplace apply, Q2, 8^3 Cartesian cells, FP64, 13,824 cell-wise values",
                               **lat}
        o.close()
        M8.close()

    if args.sweep:
        out["sweep"] = degree_sweep(cw, stream, hbm, args)
    if args.cg:
        out["cg"] = cg_bench(cw, args)
    if args.mg:
        out["mg"] = mg_bench(cw, args, stream)
    if args.mblock:
        out["multiblock"] = mblock_bench(cw, args, stream)
    if args.batched:
        out["batched"] = batched_bench(cw, args, stream)
    return out


def degree_sweep(cw, stream, hbm, args):
    import torch
    res = {}
    for p, N in SWEEP_N.items():
        mesh = synth.box_mesh(N, perturb=0.1)
        M = cw.Mesh.from_synth(mesh)
        ug = torch.from_numpy(synth.global_vector(mesh, p, seed=0)).cuda()
        row = {}
        for name, prec in [("f64", cw.CW_PREC_F64), ("f32", cw.CW_PREC_F32), ("bf16", cw.CW_PREC_BF16)]:
            o = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec)
            x = o.gather(ug)
            y = o.empty()
            o.autotune(x, y, reps=2)
            sm, km = time_apply(cw, o, x, y, max(3, args.steps // 2), 2, stream, assemble=False)
            gbs = bytes_per_value(prec, 1) * o.L / (km * 1e-3) / 1e9
            row[name] = {"dofs_per_s": o.L / (km * 1e-3), "hbm_frac": round(gbs / hbm, 4)}
            if args.book is not None:
                args.book.add(("sweep", f"p{p}", name), N, p, 1, 0, y)
            del x, y
            o.close()
        res[f"p{p}"] = {"cells": N ** 3, "values": N ** 3 * (p + 1) ** 3, **row}
        del ug
        M.close()
    return res


def batched_bench(cw, args, stream):
    """Config 5: 16 right-hand sides on one Q5 64^3 curved mesh plus 48 independent problems
    (N_i^3 cells, N_i in 8..48, degrees 2,3,5,7 in turn, seeded displacements), Laplace, applied in
    one persistent launch replayed from a CUDA graph, after the per-degree tile autotuner. The same
    work as 16 + 48 separate per-operator launches is timed alongside."""
    import torch
    probs = synth.batched_problem_list(48, seed=0)
    out = {"workload": "16 RHS x Q5 64^3 + 48 uneven problems (8^3..48^3, p in {2,3,5,7}), Laplace"}
    for name, prec in [("f32", cw.CW_PREC_F32), ("f64", cw.CW_PREC_F64)]:
        keep, ops, xs, ys, nrhs = [], [], [], [], []
        big = synth.box_mesh(64, perturb=0.1)
        Mb = cw.Mesh.from_synth(big)
        opb = cw.Operator(Mb, 5, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec)
        xb = torch.empty((16, opb.L), dtype=opb.vec_dtype, device="cuda")
        for r in range(16):
            opb.gather(torch.from_numpy(synth.global_vector(big, 5, seed=r)).cuda(), xb[r])
        keep.append(Mb)
        ops.append(opb)
        xs.append(xb)
        ys.append(torch.empty_like(xb))
        nrhs.append(16)
        for pr in probs:
            m = synth.box_mesh(pr["n"], perturb=0.1, freq=pr["freq"], direction=pr["direction"])
            M = cw.Mesh.from_synth(m)
            o = cw.Operator(M, pr["p"], cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec)
            x = o.gather(torch.from_numpy(synth.global_vector(m, pr["p"], seed=pr["seed"])).cuda())
            keep.append(M)
            ops.append(o)
            xs.append(x.view(1, -1))
            ys.append(torch.empty_like(x).view(1, -1))
            nrhs.append(1)
        B = cw.Batch(ops, nrhs, xs, ys)
        modes = {}
        for mname, mode in (("single_kernel", cw.CW_BATCH_SINGLE), ("grouped", cw.CW_BATCH_GROUPED)):
            B.set_mode(mode)
            B.autotune(reps=2)
            for _ in range(args.warmup):
                B.launch(graph=True, stream=stream.cuda_stream)
            torch.cuda.synchronize()
            a, b = event_pair()
            a.record(stream)
            for _ in range(args.steps):
                B.launch(graph=True, stream=stream.cuda_stream)
            b.record(stream)
            torch.cuda.synchronize()
            mms = a.elapsed_time(b) / args.steps
            modes[mname] = {"ms_per_launch": mms, "dofs_per_s": B.values / (mms * 1e-3),
                            "variants": {f"p{d}": B.variant(d) for d in (2, 3, 5, 7)}}
        ms = modes["grouped"]["ms_per_launch"]
        # the same work as separate launches (each op with its own autotuned variant)
        for o, x, y in zip(ops, xs, ys):
            o.autotune(x[0], y[0], reps=2)

        def unbatched():
            for o, x, y, R in zip(ops, xs, ys, nrhs):
                for r in range(R):
                    cw.cw_apply(o.handle, x[r], y[r], cw.CW_APPLY_LOCAL, stream=stream.cuda_stream)
        for _ in range(2):
            unbatched()
        torch.cuda.synchronize()
        a.record(stream)
        for _ in range(max(3, args.steps // 4)):
            unbatched()
        b.record(stream)
        torch.cuda.synchronize()
        ms_u = a.elapsed_time(b) / max(3, args.steps // 4)
        out[name] = {"values": B.values, "ms_per_launch": ms, "dofs_per_s": B.values / (ms * 1e-3),
                     "modes": modes, "unbatched_ms": ms_u, "unbatched_dofs_per_s": B.values / (ms_u * 1e-3)}
        B.close()
        del ops, xs, ys, keep
        torch.cuda.synchronize()
    return out


def cg_bench(cw, args):
    """Poisson -Laplace u = f, u = sin(pi x) sin(pi y) sin(pi z), homogeneous Dirichlet, Q3 on the
    128^3 curved mesh (134,217,728 cell-wise values): time to relative residual 1e-10 (measured
    with the native-FP64 operator) from u = 0, for each solver mode; one warm-up solve at a
    loose tolerance first."""
    import torch
    N, p = 128, 3
    mesh = synth.box_mesh(N, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = op.load_vector(0)
    u = torch.empty_like(b)
    res = {"workload": f"Poisson Q{p}, {N}^3 curved cells, {op.L} cell-wise values, Jacobi-PCG, rtol 1e-10",
           "unit": "s",
           "tolerance_measure": "||m G^T(b - A u)|| / ||m G^T b|| with A the IEEE FP64 operator (native FP64 "
                                "arithmetic, metric stored as IEEE doubles)"}
    names = [("ir_f32", cw.CW_CG_IR_F32), ("ir_bf16_metric", cw.CW_CG_IR_BF16), ("f64_doublefloat", cw.CW_CG_F64),
             ("f64_native", cw.CW_CG_F64_NATIVE)]
    if args.cg_mode >= 0:  # one mode only (profiling cases)
        names = [nm for nm in names if nm[1] == args.cg_mode]
    for name, mode in names:
        op.cg_solve(b, u, rtol=1e-3, maxit=200, mode=mode, check=False)  # warm-up: allocations, graphs
        torch.cuda.synchronize()
        _, st, rc = op.cg_solve(b, u, rtol=1e-10, maxit=20000, mode=mode, check=False)
        res[name] = {"seconds": st.seconds, "iterations": st.iterations, "outer": st.outer_iterations,
                     "rel_residual": st.rel_residual, "status": int(rc),
                     "ms_per_iteration": 1e3 * st.seconds / max(1, st.iterations),
                     # the returned u's residual measured again with each FP64 operator of the library
                     "rel_residual_ieee_fp64_operator": op.residual(b, u, cw.CW_PREC_F64_NATIVE),
                     "rel_residual_doublefloat_operator": op.residual(b, u, cw.CW_PREC_F64)}
    if len(names) == 4:
        res["speedup_ir_f32_vs_f64_native"] = res["f64_native"]["seconds"] / res["ir_f32"]["seconds"]
        res["speedup_ir_f32_vs_f64_doublefloat"] = res["f64_doublefloat"]["seconds"] / res["ir_f32"]["seconds"]
    op.close()
    M.close()
    return res


def mg_bench(cw, args, stream):
    """The Poisson problem of the CG leg (Q3, u = sin(pi x) sin(pi y) sin(pi z)) on a 128^3 mesh that
    is the 5-fold uniform refinement of a curved 4^3 mesh (0.1 h sinusoidal displacement of the coarse
    vertices; every level's mesh nested in the next, as geometric multigrid requires): CG preconditioned
    by one V-cycle (6 levels, 2 + 2 fused Jacobi sweeps, omega 0.7, dense coarse solve on 4^3 cells)
    with the cycle in double-float FP64 and in FP32, against the fastest Jacobi solve (FP64 refinement
    around an FP32 inner CG) on the same mesh; time to relative residual 1e-10 (IEEE FP64 operator)."""
    import torch
    p, n0, nl = 3, 4, 6
    ms = [synth.box_mesh(n0, perturb=0.1)]
    for _ in range(nl - 1):
        ms.append(synth.refine(ms[-1]))
    Ms = [cw.Mesh.from_synth(m) for m in ms]
    fine = cw.Operator(Ms[-1], p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0)
    b = fine.load_vector(0)
    u = torch.empty_like(b)
    res = {"workload": f"Poisson Q{p}, {ms[-1].nx}^3 cells refined {nl - 1} times from a curved {n0}^3 mesh, "
                       f"{fine.L} cell-wise values, rtol 1e-10", "unit": "s", "levels": nl}
    for name, prec in (("mg_f64_cycle", cw.CW_PREC_F64), ("mg_f32_cycle", cw.CW_PREC_F32)):
        ops = [cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec, cw.CW_BC_DIRICHLET0) for M in Ms[:-1]]
        ops.append(fine if prec == cw.CW_PREC_F64 else
                   cw.Operator(Ms[-1], p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec, cw.CW_BC_DIRICHLET0))
        t0 = time.perf_counter()
        mg = cw.Multigrid(ops, nu1=2, nu2=2, omega=0.7)
        setup_s = time.perf_counter() - t0
        mg.pcg_solve(fine, b, u, rtol=1e-3, maxit=50, check=False)  # warm-up: solver scratch, graph capture
        torch.cuda.synchronize()
        _, st, rc = mg.pcg_solve(fine, b, u, rtol=1e-10, maxit=200, check=False)
        # one V-cycle alone on the finest level (zero initial guess), CUDA events on its stream
        xb = ops[-1].empty()
        xb.copy_(b.to(xb.dtype))
        zb = ops[-1].empty()
        with torch.cuda.stream(stream):
            for _ in range(3):
                cw.cw_mg_vcycle(mg.handle, xb, zb, True, stream=stream.cuda_stream)
            e0, e1 = event_pair()
            e0.record(stream)
            for _ in range(10):
                cw.cw_mg_vcycle(mg.handle, xb, zb, True, stream=stream.cuda_stream)
            e1.record(stream)
        torch.cuda.synchronize()
        res[name] = {"seconds": st.seconds, "iterations": st.iterations, "outer": st.outer_iterations,
                     "rel_residual": st.rel_residual, "status": int(rc),
                     "ms_per_iteration": 1e3 * st.seconds / max(1, st.iterations),
                     "vcycle_ms": e0.elapsed_time(e1) / 10, "setup_s": round(setup_s, 3),
                     "rel_residual_ieee_fp64_operator": fine.residual(b, u, cw.CW_PREC_F64_NATIVE),
                     "rel_residual_doublefloat_operator": fine.residual(b, u, cw.CW_PREC_F64)}
        del xb, zb
        mg.close()
        for o in ops:
            if o is not fine:
                o.close()
    if args.mg_jacobi:
        fine.cg_solve(b, u, rtol=1e-3, maxit=200, mode=cw.CW_CG_IR_F32, check=False)
        torch.cuda.synchronize()
        _, st, rc = fine.cg_solve(b, u, rtol=1e-10, maxit=20000, mode=cw.CW_CG_IR_F32, check=False)
        res["jacobi_ir_f32"] = {"seconds": st.seconds, "iterations": st.iterations, "outer": st.outer_iterations,
                                "rel_residual": st.rel_residual, "status": int(rc)}
        best = min(res["mg_f64_cycle"]["seconds"], res["mg_f32_cycle"]["seconds"])
        res["speedup_mg_vs_jacobi_ir_f32"] = res["jacobi_ir_f32"]["seconds"] / best
    fine.close()
    for M in Ms:
        M.close()
    return res


def mblock_bench(cw, args, stream):
    """The 7-block cube in cube (inner cube [-0.5, 0.5]^3 and six frustum shells out to [-1, 1]^3, the
    stand-in for the paper's curved multi-block ball), 48^3 cells per block, Q3 Laplace, FP64 double-float
    (49.5 M cell-wise values): assembled apply (every block's operator, then the structured DSS inside the
    blocks and the unstructured inter-block DSS), the inter-block DSS alone, and the Jacobi-PCG solve of
    the sine problem to 1e-10."""
    import torch
    p, n = 3, 48
    mbm = synth.cube_in_cube(n, seed=0)
    Ms = [cw.Mesh.from_synth(m) for m in mbm.blocks]
    ops = [cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64, cw.CW_BC_DIRICHLET0) for M in Ms]
    for o in ops:
        xo = o.empty()
        o.autotune(o.gather(torch.zeros(o.NG, dtype=torch.float64, device="cuda")), xo, reps=2)
    mb = cw.MultiBlock(ops)
    x = torch.empty(mb.L, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    mb.dss(x, average=True)  # a continuous input
    y = mb.empty()

    def timed(fn, reps):
        for _ in range(3):
            fn()
        torch.cuda.synchronize()
        a, b = event_pair()
        a.record()
        for _ in range(reps):
            fn()
        b.record()
        torch.cuda.synchronize()
        return a.elapsed_time(b) / reps

    apply_ms = timed(lambda: mb.apply(x, y, assemble=True), args.steps)
    local_ms = timed(lambda: mb.apply(x, y, assemble=False), args.steps)
    dss_ms = timed(lambda: mb.dss(y), args.steps)
    b = torch.cat([o.load_vector(0) for o in ops])
    u, st, rc = mb.cg_solve(b, rtol=1e-10, maxit=20000, check=False)
    out = {"workload": f"7-block cube in cube, {n}^3 cells per block, Q{p} Laplace, {mb.L} cell-wise values, FP64",
           "assembled_apply_ms": apply_ms, "dofs_per_s": mb.L / (apply_ms * 1e-3),
           "local_apply_ms": local_ms, "dss_ms": dss_ms, "shared_dofs_face_line_vertex": mb.shared_dofs(),
           "cg": {"seconds": st.seconds, "iterations": st.iterations, "rel_residual": st.rel_residual,
                  "status": int(rc)}}
    mb.close()
    for o in ops:
        o.close()
    return out


def batch_profile(cw, n, variant, launches=3):
    """Profiling case: one grouped batch of 16 right-hand sides on a Q5 n^3 curved mesh (FP32 Laplace)
    with the given variant of degree 5 (cells-per-CTA choice + 2 * staging mode), launched a few times;
    returns the mean launch time in ms."""
    import torch
    mesh = synth.box_mesh(n, perturb=0.1)
    M = cw.Mesh.from_synth(mesh)
    op = cw.Operator(M, 5, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F32)
    x = torch.empty((16, op.L), dtype=torch.float32, device="cuda").uniform_(-1, 1)
    y = torch.empty_like(x)
    B = cw.Batch([op], [16], [x], [y])
    B.set_variant(5, variant)
    B.launch()
    torch.cuda.synchronize()
    a, e = event_pair()
    a.record()
    for _ in range(launches):
        B.launch()
    e.record()
    torch.cuda.synchronize()
    ms = a.elapsed_time(e) / launches
    B.close()
    op.close()
    return ms


def apply_profile(cw, n, prec, geom, variant, launches=4):
    """Profiling case: local applies of the bench step's operator (Q4 Laplace+mass) on an n^3 curved
    mesh in one precision and geometry mode, with a fixed kernel variant ("cells,stage") or the
    default; returns the mean time per apply in ms."""
    import torch
    mesh = synth.box_mesh(n, perturb=0.1)
    op = cw.Operator(cw.Mesh.from_synth(mesh), P, KIND, geom, prec)
    x = op.gather(torch.from_numpy(synth.global_vector(mesh, P, seed=0)).cuda())
    y = op.empty()
    if variant:
        op.set_variant(*[int(v) for v in variant.split(",")])
    op.apply(x, y)
    torch.cuda.synchronize()
    a, e = event_pair()
    a.record()
    for _ in range(launches):
        op.apply(x, y)
    e.record()
    torch.cuda.synchronize()
    return a.elapsed_time(e) / launches


def mblock_profile(cw, n, launches=3):
    """Profiling case: the 7-block cube in cube with n^3 cells per block, Q3 Laplace, FP64 double-float:
    assembled multi-block applies (every block's operator, the structured DSS inside the blocks, then the
    unstructured inter-block DSS), launched a few times; returns the mean time per apply in ms."""
    import torch
    mbm = synth.cube_in_cube(n, seed=0)
    ops = [cw.Operator(cw.Mesh.from_synth(m), 3, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, cw.CW_PREC_F64,
                       cw.CW_BC_DIRICHLET0) for m in mbm.blocks]
    mb = cw.MultiBlock(ops)
    x = torch.empty(mb.L, dtype=torch.float64, device="cuda").uniform_(-1, 1)
    mb.dss(x, average=True)
    y = mb.empty()
    mb.apply(x, y, assemble=True)
    torch.cuda.synchronize()
    a, e = event_pair()
    a.record()
    for _ in range(launches):
        mb.apply(x, y, assemble=True)
    e.record()
    torch.cuda.synchronize()
    return a.elapsed_time(e) / launches


def mg_cycle_profile(cw, n, prec, cycles=3):
    """Profiling case: V-cycles alone (zero initial guess) on a Q3 hierarchy whose finest mesh has n^3
    cells (6 levels, refined from a curved (n/32)^3 mesh), in one precision; no solver. Returns the mean
    cycle time in ms."""
    import torch
    p, nl = 3, 6
    ms = [synth.box_mesh(n // 32, perturb=0.1)]
    for _ in range(nl - 1):
        ms.append(synth.refine(ms[-1]))
    Ms = [cw.Mesh.from_synth(m) for m in ms]
    ops = [cw.Operator(M, p, cw.CW_LAPLACE, cw.CW_GEOM_METRIC, prec, cw.CW_BC_DIRICHLET0) for M in Ms]
    mg = cw.Multigrid(ops)
    b = ops[-1].empty()
    b.copy_(torch.from_numpy(synth.cellwise_random(ms[-1], p, seed=0)).to(b.dtype))
    z = ops[-1].empty()
    for _ in range(2):
        mg.vcycle(b, z)
    torch.cuda.synchronize()
    a, e = event_pair()
    a.record()
    for _ in range(cycles):
        mg.vcycle(b, z)
    e.record()
    torch.cuda.synchronize()
    ms_cycle = a.elapsed_time(e) / cycles
    mg.close()
    for o in ops:
        o.close()
    return ms_cycle


# ------------------------------------------------------------------------- CPU oracle ----
def oracle_sample_rate(target_s, seed=0):
    """Times the oracle apply (explicit element matrices, K+M, p=4) on a cell sample of the 64^3
    curved workload; the sample grows until one timing takes about target_s seconds."""
    import oracle
    oracle.build()
    mesh = synth.box_mesh(NCELL, perturb=0.1)
    rng = np.random.default_rng(seed)
    x = synth.cellwise_random(mesh, P, seed=seed)
    ncell = 16
    while True:
        cells = np.sort(rng.choice(mesh.ncells, ncell, replace=False))
        t0 = time.perf_counter()
        oracle.apply_local(mesh, P, KIND, x, cells)
        dt = time.perf_counter() - t0
        if dt >= target_s or ncell >= mesh.ncells:
            return ncell * (P + 1) ** 3 / dt, ncell, dt
        ncell = min(mesh.ncells, int(ncell * max(2.0, min(8.0, target_s / max(dt, 1e-3)))))


def cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count()


def reference_arm(args, rank, world):
    if rank != 0:
        return None
    # calibrate a per-step sample of about 2 s, then time warmup + steps of it
    import oracle
    rate, ncell, dt = oracle_sample_rate(2.0)
    mesh = synth.box_mesh(NCELL, perturb=0.1)
    x = synth.cellwise_random(mesh, P, seed=1)
    rng = np.random.default_rng(1)
    times = []
    for s in range(args.warmup + args.steps):
        cells = np.sort(rng.choice(mesh.ncells, ncell, replace=False))
        t0 = time.perf_counter()
        oracle.apply_local(mesh, P, KIND, x, cells)
        if s >= args.warmup:
            times.append(time.perf_counter() - t0)
    ms = 1e3 * float(np.mean(times))
    value = ncell * (P + 1) ** 3 / (ms * 1e-3)
    samp = f"{ncell} random cells of the 64^3 mesh per step (element matrices built per cell), OpenMP"
    return {"impl": "reference", "metric": METRIC, "value": value, "unit": "DoF/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": WORKLOAD, "degree": P, "cells": NCELL ** 3, "parallelism": "host cores"},
            "cpu_baseline": {"value": value, "unit": "DoF/s", "cores": cores(), "kind": "oracle",
                             "sample": samp},
            "e2e": {"value": value, "unit": "DoF/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}


def oracle_cg_time(n=16, p=3):
    """The oracle's assembled Jacobi-PCG (scipy sparse, host cores) on the Poisson problem at the
    largest mesh it solves in a few seconds: the same method as the GPU solve, 16^3 curved cells Q3."""
    import oracle as orc
    orc.build()
    orc.lib()
    mesh = synth.box_mesh(n, perturb=0.1)
    t0 = time.perf_counter()
    b = orc.load_vector(mesh, p, orc.PROBLEM_SINE)
    A = orc.assemble_global(mesh, p, 1)
    t1 = time.perf_counter()
    _, its, rel, _ = orc.pcg_assembled(A, orc.scatter_add(mesh, p, b), orc.boundary_mask_global(mesh, p), tol=1e-10)
    t2 = time.perf_counter()
    return {"workload": f"Poisson Q{p}, {n}^3 curved cells, assembled Jacobi-PCG to 1e-10",
            "assembly_s": round(t1 - t0, 3), "solve_s": round(t2 - t1, 3), "iterations": its,
            "rel_residual": rel}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="gb300")
    ap.add_argument("--no-sweep", dest="sweep", action="store_false")
    ap.add_argument("--no-cg", dest="cg", action="store_false")
    ap.add_argument("--no-batched", dest="batched", action="store_false")
    ap.add_argument("--no-mg", dest="mg", action="store_false")
    ap.add_argument("--no-mblock", dest="mblock", action="store_false")
    ap.add_argument("--no-mg-jacobi", dest="mg_jacobi", action="store_false",
                    help="multigrid leg without the Jacobi comparison solve")
    ap.add_argument("--profile-mg", type=int, default=0,
                    help="profiling case: only V-cycles on an N^3 Q3 hierarchy (FP32), then exit")
    ap.add_argument("--profile-apply", type=int, default=0,
                    help="profiling case: local applies of the step's operator on an N^3 mesh (--prec, --geom, --variant)")
    ap.add_argument("--geom", type=int, default=1, help="CW_GEOM_* of --profile-apply (1 stored metric, 2 recomputed)")
    ap.add_argument("--profile-mblock", type=int, default=0,
                    help="profiling case: assembled applies on the 7-block cube in cube, N^3 cells per block")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling case: only a 16-RHS grouped batch on a Q5 N^3 mesh (FP32), then exit")
    ap.add_argument("--batch-variant", type=int, default=2, help="degree-5 variant of --profile-batch")
    ap.add_argument("--no-mixed", dest="mixed", action="store_false")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-cpu", dest="cpu", action="store_false")
    ap.add_argument("--no-tune", dest="tune", action="store_false", help="default kernel variant, no autotuning")
    ap.add_argument("--variant", default="", help="cells_per_cta,stage of the main step's kernel (profiling cases)")
    ap.add_argument("--cg-mode", type=int, default=-1, help="CW_CG_* mode: time this solver mode only (profiling cases)")
    ap.add_argument("--cells", type=int, default=NCELL, help="cells per direction (profiling cases)")
    ap.add_argument("--prec", type=int, default=0, help="CW_PREC_* of the main step (profiling cases)")
    ap.add_argument("--cpu-seconds", type=float, default=15.0)
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.impl == "reference":
        # rank 0 alone times the oracle; other ranks exit without work
        rank, world = int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1"))
        out = reference_arm(args, rank, world)
        if out is not None:
            print(json.dumps(out))
        return
    if args.profile_batch:
        import torch
        import paper_2607_03413_gb300 as cw
        torch.cuda.set_device(0)
        cw.load()
        print(json.dumps({"profile": "batch_16rhs_q5", "cells": args.profile_batch ** 3, "variant": args.batch_variant,
                          "ms_per_launch": batch_profile(cw, args.profile_batch, args.batch_variant)}))
        return
    if args.profile_apply:
        import torch
        import paper_2607_03413_gb300 as cw
        torch.cuda.set_device(0)
        cw.load()
        print(json.dumps({"profile": "apply", "cells": args.profile_apply ** 3, "prec": args.prec, "geom": args.geom,
                          "variant": args.variant,
                          "ms_per_apply": apply_profile(cw, args.profile_apply, args.prec, args.geom, args.variant)}))
        return
    if args.profile_mblock:
        import torch
        import paper_2607_03413_gb300 as cw
        torch.cuda.set_device(0)
        cw.load()
        print(json.dumps({"profile": "mblock_apply", "cells_per_block": args.profile_mblock ** 3,
                          "ms_per_apply": mblock_profile(cw, args.profile_mblock)}))
        return
    if args.profile_mg:
        import torch
        import paper_2607_03413_gb300 as cw
        torch.cuda.set_device(0)
        cw.load()
        print(json.dumps({"profile": "mg_cycle", "cells": args.profile_mg ** 3,
                          "f32_cycle_ms": mg_cycle_profile(cw, args.profile_mg, cw.CW_PREC_F32)}))
        return
    rank, local, world = dist_init(args)
    args.book = SampleBook() if (rank == 0 and world == 1 and args.cpu) else None
    out = gpu_arm(args, rank, local, world)
    if rank == 0 and world == 1 and args.cpu:
        oracle_errors(args.book, out)
        rate, ncell, dt = oracle_sample_rate(args.cpu_seconds)
        out["cpu_baseline"] = {"value": rate, "unit": "DoF/s", "cores": cores(), "kind": "oracle",
                               "sample": f"{ncell} random cells of the 64^3 curved mesh, K+M p=4, "
                                         f"element matrices built and applied per cell ({dt:.1f} s)"}
        if args.cg:
            out["cpu_baseline"]["cg"] = oracle_cg_time()
    if rank == 0 and out is not None:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
