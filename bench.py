#!/usr/bin/env python
"""Benchmark: SIPG dG assembly throughput on GB300.

One step = one pass of the whole hot path on device-resident inputs
(dg_assemble_step): geometry kernels, then the element kernels (volume +
own faces + load vector) and the interface kernels, writing every block of
the BSR matrix and the load vector.

Default workload: 2D advection-diffusion-reaction on 65,536 Voronoi cells,
p ~ U{1..4}, a = 10^U(-2,2), b = (1, 0.5), c = 1 (seeded, synthetic).
Headline form: FP32 contractions on FP32 geometry records equal to the
rounded FP64 ones; the FP64 form is timed in the same run and the FP32
matrix error against it is reported.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
For N > 1 launch under torch.distributed.run; every rank assembles its own
replica of the workload (weak scaling, no collective on the data path).
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

# The pass runs its degree groups on forked streams, and a recorded pass
# branches the same way.  With the driver's default of 8 hardware work queues
# a process that has used more streams than that can put two branches on one
# queue, where they run one after the other: measured 0.552 instead of
# 0.538 ms per adr2d_65k step.  Set before CUDA is initialised.
os.environ.setdefault("CUDA_DEVICE_MAX_CONNECTIONS", "32")

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

L2_FLUSH_BYTES = 256 << 20  # > 129 MB L2
METRIC = "dG assembly elements/s & matrix GB/s vs roofline; reduced vs FP64 form at fixed err"
# reduced forms of the timed pass: binding constant and arithmetic type
PRECS = {"fp32": "DG_PREC_FP32", "bf16x3": "DG_PREC_BF16X3", "tf32x3": "DG_PREC_TF32X3"}
DTYPES = {"fp32": "f32", "bf16x3": "bf16x3 (f32 accumulate)", "tf32x3": "tf32x3 (f32 accumulate)"}
WORKLOADS = {
    "adr2d_65k": ("adr2d_65k: 2D advection-diffusion-reaction, 65,536 clipped Voronoi cells (5 Lloyd steps), "
                  "p~U{1..4}, a=10^U(-2,2), b=(1,0.5), c=1, sin-product source, penalty 10 p^2/h"),
    "poisson2d_1k": ("poisson2d_1k: 2D Poisson, 1,024 clipped Voronoi cells (5 Lloyd steps), p=2, a=1, b=0, c=0, "
                     "f from u=sin(pi x)sin(pi y), penalty 10 p^2/h"),
    "diff3d_32k": ("diff3d_32k: 3D diffusion, 64^3 cubes x 6 Kuhn tets (1,572,864 tets) agglomerated by k-means "
                   "into 32,768 polyhedra, p=3, a=10^U(-2,2), b=0, c=0, penalty 10 p^2/h"),
    "diff3d_8k": ("diff3d_8k: the diff3d_32k recipe on 40^3 cubes x 6 Kuhn tets (384,000 tets) agglomerated into "
                  "8,192 polyhedra, p=3 (the small case of the 3D kernel profiles)"),
    "learned2d_262k": ("learned2d_262k: 2D ADR on 262,144 clipped Voronoi cells (3-12 vertices), p=3, a=10^U(-2,2), "
                       "b=(1,0.5), c=1; learned 28-point volume rules (24->128->128->84 BF16 network trained on "
                       "1,048,576 polygons of 16 independent meshes, then 3 FP64 Gauss-Newton steps, sub-triangle "
                       "fallback), assembled in FP32"),
    "batch2d_256": ("batch2d_256: 256 independent 2D clipped-Voronoi meshes (5 Lloyd steps), cell counts "
                    "log-uniform in 512..16,384, per-mesh p~U{1..5}, a=10^U(-2,2), b=(1,0.5), c=1, one recorded "
                    "pass over the whole batch"),
    "slab2d_65k_p": ("slab2d_65k_p: one space-time slab (Sec. 2.3) over the adr2d_65k mesh and problem, prisms "
                     "kappa x (0, 0.01], space P_p (space-time total degree <= p, p~U{1..4}), FP32: the slab "
                     "matrix and load vector with the previous slab's trace"),
    "slab2d_65k_pq": ("slab2d_65k_pq: as slab2d_65k_p in the space PQ_p (degree <= p in t and in x)"),
    "adr3d_varcoef": ("adr3d_varcoef: the 3D test problem of Sec. 4.2 (A=0.01 I, b=(1+x,1+y,1+z), c=3+xyz, "
                      "u=sin(pi x)sin(pi y)sin(pi z)) on 50^3 cubes x 6 Kuhn tets (750,000 tets) grown into polyhedra "
                      "of about 4 tets (seeded greedy region growing across faces), p=3, FP32: the row pass without b "
                      "and c, then the variable-coefficient kernels"),
    "adr3d_varcoef_12k": ("adr3d_varcoef_12k: the adr3d_varcoef recipe on 20^3 cubes x 6 Kuhn tets (48,000 tets), "
                          "the small case of the variable-coefficient kernel profiles"),
}


class _Batch:
    """The batch workload as one object: members plus their concatenated
    coordinates and coefficients (for the host-memory path)."""

    def __init__(self, members):
        self.members = members
        self.dim = 2
        self.ne = sum(w.ne for w in members)
        self.problem = members[0].problem
        self.a = np.concatenate([w.a for w in members])
        self.p = np.concatenate([w.p for w in members])

        class _M:
            pass

        self.mesh = _M()
        self.mesh.x = np.concatenate([w.mesh.x for w in members])
        self.mesh.y = np.concatenate([w.mesh.y for w in members])
WORKLOAD = WORKLOADS["adr2d_65k"]


def make_workload(name):
    from paper_2007_04881_gb300 import configs

    if name in ("adr2d_65k", "slab2d_65k_p", "slab2d_65k_pq"):
        return configs.adr2d()
    if name == "poisson2d_1k":
        return configs.poisson2d()
    if name == "diff3d_32k":
        return configs.diff3d()
    if name == "diff3d_8k":
        return configs.diff3d(n=40, clusters=8192)
    if name == "batch2d_256":
        return _Batch(configs.batch2d())
    if name == "learned2d_262k":
        return configs.learned2d()
    if name == "adr3d_varcoef":
        return configs.adr3d_varcoef()
    if name == "adr3d_varcoef_12k":
        return configs.adr3d_varcoef(n=20)
    raise SystemExit(f"unknown workload {name}")


def emit(line: dict) -> None:
    """Print the bench line; with --jsonl, also append it (with the time and
    the command line) to that run log, one JSON object per line."""
    print(json.dumps(line))
    path = getattr(emit, "jsonl", None)
    if path:
        rec = dict(line, logged_at=time.strftime("%Y-%m-%dT%H:%M:%S"), argv=sys.argv[1:])
        with open(path, "a") as f:
            f.write(json.dumps(rec) + "\n")


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except Exception:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "sm_max_mhz": 2070.0}, "fallback"


def fp32_alu_peak_tflops(sm_mhz: float, sms: int) -> float:
    # 128 FP32 FMA lanes per SM, 2 flops per FMA
    return sms * 128 * 2 * sm_mhz * 1e6 / 1e12


def device_sms() -> int:
    import torch

    return int(torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)


FP64_PEAK_TFLOPS = 1.25  # GB300 FP64, the nominal figure of the profiling recipe


class ClockSampler:
    """nvidia-smi clock / throttle sampling during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index: int):
        self.dev = device_index
        self.proc = None
        self.path = os.path.join("/tmp", f"dg_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        out = {"sm_mhz": None, "sm_max_mhz": None, "reasons": [], "samples": 0}
        if self.proc is None:
            return out
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.f.close()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [x.strip() for x in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        os.unlink(self.path)
        if sm:
            out.update(sm_mhz=statistics.median(sm), sm_max_mhz=max(smax), reasons=sorted(reasons), samples=len(sm))
        return out


def dist_setup(use_cuda: bool):
    import torch

    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if ws > 1:
        import torch.distributed as dist

        if use_cuda:
            torch.cuda.set_device(local)
        dist.init_process_group("nccl" if use_cuda else "gloo")
    return ws, rank, local


def barrier(ws):
    if ws > 1:
        import torch.distributed as dist

        dist.barrier()


def max_over_ranks(x: float, ws: int) -> float:
    if ws == 1:
        return x
    import torch
    import torch.distributed as dist

    t = torch.tensor([x], dtype=torch.float64, device="cuda")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def workload_config(wl, info, name):
    return {
        "workload": WORKLOADS[name],
        "elements": int(info.ne),
        "interfaces": int(info.ninterfaces),
        "boundary_faces": int(info.nbfaces),
        "sub_triangles": int(info.nsub),
        "quad_points_volume": int(info.nqvol),
        "quad_points_face": int(info.nqface),
        "bsr_blocks": int(info.nnzb),
        "matrix_entries": int(info.nvals),
        "dofs": int(info.ndofs),
        "l2": "flushed between timed steps (256 MiB write, outside the timed region)",
    }


# ---------------------------------------------------------------------------
# reference arm: the FP64 CPU oracle on a bounded sample per step
# ---------------------------------------------------------------------------


def run_reference(args):
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    if args.workload.startswith("slab2d"):
        return run_reference_slab(args, ws)
    import oracle as O
    from paper_2007_04881_gb300 import configs

    wl = make_workload(args.workload)
    batch_ne = None
    if isinstance(wl, _Batch):  # the oracle samples the largest member
        batch_ne = wl.ne
        wl = max(wl.members, key=lambda w: w.ne)
    om = O.Mesh(wl.mesh)
    # the variable-coefficient workload: the oracle with the Sec. 4.2 fields
    coef = {"coef": 1} if args.workload.startswith("adr3d_varcoef") else {}
    pb = O.make_problem(wl.dim, **wl.problem, **coef)
    p = wl.p.astype(np.int32)
    cores = os.cpu_count() or 1
    # per step: a contiguous sample of elements and the same share of interfaces
    per_step = args.ref_sample
    rng = np.random.default_rng(7)
    times = []
    tot = 0
    for it in range(args.warmup + args.steps):
        e0 = int(rng.integers(0, wl.ne - per_step))
        el = np.arange(e0, e0 + per_step, dtype=np.int32)
        i0 = int(round(e0 * om.ni / wl.ne))
        ni = int(round(per_step * om.ni / wl.ne))
        ifs = np.arange(i0, min(i0 + ni, om.ni), dtype=np.int32)
        t = time.perf_counter()
        om.assemble(p, wl.a, pb, elems=el, ifaces=ifs, nthreads=cores)
        dt = time.perf_counter() - t
        if it >= args.warmup:
            times.append(dt)
            tot += per_step
    T = sum(times)
    value = tot / T
    sample = (f"{per_step} consecutive elements (diagonal blocks + load vector) and the proportional "
              f"{int(round(per_step * om.ni / wl.ne))} interfaces (off-diagonal block pairs) per step, "
              f"FP64, OpenMP over {cores} threads")
    line = {
        "impl": "reference",
        "metric": METRIC,
        "value": value,
        "unit": "elements/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": 1e3 * T / max(1, len(times)),
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "elements": int(batch_ne or wl.ne), "interfaces": int(om.ni),
                   "boundary_faces": int(om.nbf), "sample_per_step": per_step},
        "cpu_baseline": {"value": value, "unit": "elements/s", "cores": cores, "kind": "oracle", "sample": sample},
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)
    return 0


def run_reference_slab(args, ws):
    """Reference arm of the slab workloads: the slab oracle, one bounded
    sample per step (at most 3 timed steps: each is seconds of plain numpy)."""
    space_name = "PQ" if args.workload.endswith("_pq") else "P"
    steps = min(args.steps, 3)
    slab_cpu_sample(space_name)  # warm-up
    runs = [slab_cpu_sample(space_name) for _ in range(steps)]
    value = sum(r["value"] for r in runs) / len(runs)
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": "elements/s", "n_gpus": ws,
        "steps": steps, "warmup": 1, "ms_per_step": 1e3 * 40 / value, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "elements": 65536, "sample_per_step": runs[0]["sample"]},
        "cpu_baseline": dict(runs[0], value=value),
        "e2e": {"value": value, "unit": "elements/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    emit(line)
    return 0


def cpu_baseline_sample(wl, seconds_target=12.0):
    """The oracle as it stands, on a bounded sample of the workload, timed on
    the host cores (rank 0, N=1 only)."""
    import oracle as O

    cores = os.cpu_count() or 1
    om = O.Mesh(wl.mesh)
    pb = O.make_problem(wl.dim, **wl.problem)
    p = wl.p.astype(np.int32)
    n = min(2048, wl.ne // 2)
    el = np.arange(n, dtype=np.int32)
    ifs = np.arange(int(round(n * om.ni / wl.ne)), dtype=np.int32)
    t = time.perf_counter()
    om.assemble(p, wl.a, pb, elems=el, ifaces=ifs, nthreads=cores)
    dt = time.perf_counter() - t
    # grow the sample to ~seconds_target of CPU work (bounded by the mesh)
    n2 = int(min(wl.ne, max(n, n * seconds_target / max(dt, 1e-3))))
    el = np.arange(n2, dtype=np.int32)
    ifs = np.arange(int(round(n2 * om.ni / wl.ne)), dtype=np.int32)
    t = time.perf_counter()
    ob = om.assemble(p, wl.a, pb, elems=el, ifaces=ifs, nthreads=cores)
    dt = time.perf_counter() - t
    # one thread, on a sample of about a third of the OpenMP run's CPU time per core
    n1 = max(16, min(n2, int(n2 * 4.0 / max(dt * cores, 1e-3))))
    el1 = np.arange(n1, dtype=np.int32)
    ifs1 = np.arange(int(round(n1 * om.ni / wl.ne)), dtype=np.int32)
    t = time.perf_counter()
    om.assemble(p, wl.a, pb, elems=el1, ifaces=ifs1, nthreads=1)
    dt1 = time.perf_counter() - t
    line = {
        "value": n2 / dt,
        "unit": "elements/s",
        "cores": cores,
        "kind": "oracle",
        "sample": f"first {n2} of {wl.ne} elements (diagonal blocks + load vector) and {ifs.size} of {om.ni} "
                  f"interfaces, FP64, {dt:.1f} s on {cores} threads",
        "one_thread": {"value": n1 / dt1, "unit": "elements/s",
                       "sample": f"first {n1} elements and {ifs1.size} interfaces, {dt1:.1f} s on 1 thread"},
    }
    return line, (om, ob)


def oracle_error(mesh, vals, rhs, om, ob):
    """Largest block max-norm relative difference between the library's
    result (host arrays) and the oracle's sampled blocks."""
    from math import comb

    row_ptr, col, blk_off, dof_off = mesh.dg_bsr_pattern()
    nb = np.array([comb(int(q) + mesh.dim, mesh.dim) for q in mesh.p])

    def block(r, c):
        cols = col[row_ptr[r]:row_ptr[r + 1]]
        k = row_ptr[r] + int(np.searchsorted(cols, c))
        return vals[blk_off[k]:blk_off[k + 1]].reshape(nb[r], nb[c])

    def rel(g, o):
        s = np.abs(o).max()
        return float(np.abs(g - o).max() / s) if s > 0 else float(np.abs(g).max())

    ed = max(rel(block(int(e), int(e)), ob["diag"][i]) for i, e in enumerate(ob["elems"]))
    er = max(rel(rhs[dof_off[int(e)]:dof_off[int(e) + 1]], ob["rhs"][i]) for i, e in enumerate(ob["elems"]))
    eo = 0.0
    for k, i in enumerate(ob["ifaces"]):
        e0, e1 = int(om.if_e0[i]), int(om.if_e1[i])
        eo = max(eo, rel(block(e0, e1), ob["a01"][k]), rel(block(e1, e0), ob["a10"][k]))
    return {"diag_block_rel_max": ed, "offdiag_block_rel_max": eo, "rhs_rel_max": er,
            "sample": f"{len(ob['elems'])} elements and {len(ob['ifaces'])} interfaces of the oracle sample"}


# ---------------------------------------------------------------------------
# our arm
# ---------------------------------------------------------------------------


def time_steps(torch, stream, step, flush, steps, ctx=None):
    """Per-step CUDA-event times (ms); L2 flushed between steps, untimed.
    With ctx, also collects the library's per-launch timings."""
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
    stats = {}
    for i in range(steps):
        flush.zero_()
        ev[i][0].record(stream)
        step()
        ev[i][1].record(stream)
        if ctx is not None:
            for name, ms, fl, by in ctx.dg_kernel_stats():
                s = stats.setdefault(name, [0.0, 0, fl, by])
                s[0] += ms
                s[1] += 1
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in ev], stats


def run_ours(args):
    # mesh generation (process pools for the batch) before any CUDA call
    wl = make_workload(args.workload)
    import torch

    from paper_2007_04881_gb300 import build as B
    from paper_2007_04881_gb300 import dg

    ws, rank, local = dist_setup(True)
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    B.build()
    stream = torch.cuda.current_stream()
    ctx = dg.Context(dev, stream.cuda_stream)
    pb = dg.Problem(**wl.problem)
    t0 = time.perf_counter()
    if isinstance(wl, _Batch):
        mesh = dg.Mesh(ctx, None, problem=pb, members=[(w.mesh, w.p, w.a) for w in wl.members])
    else:
        mesh = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    upload_ms = 1e3 * (time.perf_counter() - t0)
    info = mesh.info
    pattern_ms = None
    pattern = None
    if not isinstance(wl, _Batch):
        t0 = time.perf_counter()
        dg.dg_mesh_check(wl.mesh, wl.p, wl.a, pb)
        pattern_ms = 1e3 * (time.perf_counter() - t0)
        # the same pattern built on the device (dg_set_pattern_device); the
        # second upload is timed (the first loads the pattern kernels)
        ctx.dg_set_pattern_device(True)
        for _ in range(2):
            md = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
            td = md.dg_mesh_timings()
            md.close()
        ctx.dg_set_pattern_device(False)
        th = mesh.dg_mesh_timings()
        pattern = {"host_plan_ms": th["pattern_ms"], "host_upload_ms": th["upload_ms"],
                   "device_pattern_ms": td["pattern_ms"], "device_upload_ms": td["upload_ms"],
                   "note": "pattern = faces, interfaces, block rows and offsets, half-face lists, work lists; "
                           "host: the C++ plan on the host cores; device: the kernels of dg_set_pattern_device "
                           "with their host copies; both include the host checks of the descriptor"}

    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    prec = getattr(dg, PRECS[args.prec])
    v32 = torch.empty(mesh.nvals, dtype=torch.float32, device="cuda")
    r32 = torch.empty(mesh.ndofs, dtype=torch.float32, device="cuda")

    for _ in range(args.warmup):
        mesh.dg_assemble_step(prec, v32, r32)
    torch.cuda.synchronize()
    # one recorded pass (CUDA graph), launch shape picked by the autotuner;
    # per-launch timing events are recorded inside the graph
    ctx.dg_set_timing(True)
    g32 = mesh.dg_graph_create(prec, v32, r32, autotune=True)
    ginfo = g32.dg_graph_info()
    for _ in range(args.warmup):
        g32.dg_graph_launch()
    torch.cuda.synchronize()
    launches_per_step = ctx.launches()

    # ---- timed region (FP32 form, headline)
    sampler = ClockSampler(dev)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    kstats_src = "per-launch events recorded inside the graph"
    try:
        times, kstats = time_steps(torch, stream, g32.dg_graph_launch, flush, args.steps, ctx)
    except dg.DGError:
        # in-graph events not timeable here: time the graph alone, then the
        # same launches issued directly with per-launch events
        times, _ = time_steps(torch, stream, g32.dg_graph_launch, flush, args.steps, None)
        _, kstats = time_steps(torch, stream, lambda: mesh.dg_assemble_step(prec, v32, r32), flush,
                               args.steps, ctx)
        kstats_src = "per-launch events of the same launches issued directly (second timed loop)"
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ms_step = max_over_ranks(sum(times) / len(times), ws)
    value = ws * info.ne / (ms_step * 1e-3)

    # ---- FP64 form (same workload), for the reduced-vs-FP64 comparison
    v64 = torch.empty(mesh.nvals, dtype=torch.float64, device="cuda")
    r64 = torch.empty(mesh.ndofs, dtype=torch.float64, device="cuda")
    g64 = mesh.dg_graph_create(dg.DG_PREC_FP64, v64, r64, autotune=False)
    g64.dg_graph_launch()
    torch.cuda.synchronize()
    k64 = max(3, min(args.steps // 10, 20 if info.ne < 200000 and mesh.dim == 2 else 3))
    try:
        t64, kstats64 = time_steps(torch, stream, g64.dg_graph_launch, flush, k64, ctx)
    except dg.DGError:
        t64, _ = time_steps(torch, stream, g64.dg_graph_launch, flush, k64, None)
        _, kstats64 = time_steps(torch, stream, lambda: mesh.dg_assemble_step(dg.DG_PREC_FP64, v64, r64), flush,
                                 k64, ctx)
    ctx.dg_set_timing(False)
    ms64 = max_over_ranks(sum(t64) / len(t64), ws)
    # error of the reduced form against the FP64 form (same device inputs)
    g32.dg_graph_launch()
    g64.dg_graph_launch()
    torch.cuda.synchronize()
    d = (v32.double() - v64)
    err_fro = float(torch.linalg.vector_norm(d) / torch.linalg.vector_norm(v64))
    err_max = float(d.abs().max() / v64.abs().max())
    err_rhs = float(torch.linalg.vector_norm(r32.double() - r64) / torch.linalg.vector_norm(r64))
    del d

    # ---- the other reduced forms (FP32 ALU and tensor-core contractions), same inputs
    forms = {}
    kf = max(3, min(args.steps // 4, 50 if info.ne < 200000 and mesh.dim == 2 else 5))
    variants = [(k, getattr(dg, v), 1) for k, v in PRECS.items() if getattr(dg, v) != prec]
    if prec != dg.DG_PREC_FP64:
        # the same form with the geometry recomputed by the FP64 kernels each
        # pass (FP64 maps, Jacobians, normals and penalties, rounded to FP32)
        variants.append((args.prec + "_fp64_geometry", prec | dg.DG_GEOM_FP64, 1))
    if prec in (dg.DG_PREC_FP32, dg.DG_PREC_FP64):
        variants.append((args.prec + "_pointwise_volume", prec, 0))
        if mesh.dim == 2:  # volume moments exact, from the element's edges
            variants.append((args.prec + "_exact_moments", prec, 2))
    for fname, fprec, vpath in variants:
        ctx.dg_set_volume_path(vpath)
        dtf = torch.float64 if fprec == dg.DG_PREC_FP64 else torch.float32  # the form's output type
        vf = torch.empty(mesh.nvals, dtype=dtf, device="cuda")
        rf = torch.empty(mesh.ndofs, dtype=dtf, device="cuda")
        ctx.dg_set_timing(False)
        gf = mesh.dg_graph_create(fprec, vf, rf, autotune=True)
        for _ in range(2):
            gf.dg_graph_launch()
        torch.cuda.synchronize()
        tf, _ = time_steps(torch, stream, gf.dg_graph_launch, flush, kf, None)
        ctx.dg_set_timing(True)
        _, ksf = time_steps(torch, stream, lambda: mesh.dg_assemble_step(fprec, vf, rf), flush, 3, ctx)
        ctx.dg_set_timing(False)
        df = vf.double() - v64
        msf = max_over_ranks(sum(tf) / len(tf), ws)
        rp = ksf.get("row_pass")
        forms[fname] = {
            "ms_per_step": msf, "value": ws * info.ne / (msf * 1e-3), "steps": kf,
            "row_pass_ms_direct_launch": rp[0] / rp[1] if rp else None,
            "row_pass_tflops_direct_launch": rp[2] / (rp[0] / rp[1] * 1e-3) / 1e12 if rp else None,
            "matrix_rel_fro": float(torch.linalg.vector_norm(df) / torch.linalg.vector_norm(v64)),
            "matrix_rel_max": float(df.abs().max() / v64.abs().max()),
            "rhs_rel_fro": float(torch.linalg.vector_norm(rf.double() - r64) / torch.linalg.vector_norm(r64)),
            "kernels_ms_direct_launch": {k: v[0] / v[1] for k, v in sorted(ksf.items())},
            "graph": gf.dg_graph_info(),
        }
        del vf, rf, gf, df
    ctx.dg_set_volume_path(1)
    del v64, r64, g64
    torch.cuda.empty_cache()

    # ---- end to end through the host-memory entry point
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
    hx, hy, ha = pin(wl.mesh.x, np.float64), pin(wl.mesh.y, np.float64), pin(wl.a, np.float64)
    hz = pin(wl.mesh.z, np.float64) if wl.dim == 3 else None
    hv = torch.empty(mesh.nvals, dtype=torch.float32).pin_memory()
    hr = torch.empty(mesh.ndofs, dtype=torch.float32).pin_memory()
    e2e_steps = max(3, min(args.steps, 50 if info.ne < 200000 and wl.dim == 2 else 5))
    for _ in range(2):
        mesh.dg_assemble_host(prec, hv, hr, x=hx, y=hy, z=hz, a=ha)
    barrier(ws)
    t = time.perf_counter()
    for _ in range(e2e_steps):
        mesh.dg_assemble_host(prec, hv, hr, x=hx, y=hy, z=hz, a=ha)
    e2e_sync_s = max_over_ranks((time.perf_counter() - t) / e2e_steps, ws)
    # the same steps pipelined: step k's copy back runs beside step k + 1's
    # pass (dg_assemble_host_submit / _wait, two output buffer pairs); every
    # step still copies its inputs in and its whole system back
    hv2 = [hv, torch.empty(mesh.nvals, dtype=torch.float32).pin_memory()]
    hr2 = [hr, torch.empty(mesh.ndofs, dtype=torch.float32).pin_memory()]
    for k in range(2):
        mesh.dg_assemble_host_wait(mesh.dg_assemble_host_submit(prec, hv2[k], hr2[k], x=hx, y=hy, z=hz, a=ha))
    barrier(ws)
    t = time.perf_counter()
    prev = None
    for k in range(e2e_steps):
        tk = mesh.dg_assemble_host_submit(prec, hv2[k % 2], hr2[k % 2], x=hx, y=hy, z=hz, a=ha)
        if prev is not None:
            mesh.dg_assemble_host_wait(prev)
        prev = tk
    mesh.dg_assemble_host_wait(prev)
    e2e_s = max_over_ranks((time.perf_counter() - t) / e2e_steps, ws)
    h2d = (hx.numel() + hy.numel() + ha.numel() + (hz.numel() if hz is not None else 0)) * 8
    d2h = hv.numel() * 4 + hr.numel() * 4

    if rank != 0:
        return 0

    # ---- roofline of the dominant kernel
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = device_sms()
    alu_peak = fp32_alu_peak_tflops(sm_max, sms)
    # the dominant unit: the pass of row kernels (per-degree launches, which
    # the recorded graph may run concurrently), else the longest launch
    if "row_pass" in kstats:
        dom = ("row_pass", kstats["row_pass"])
    else:
        dom = max(kstats.items(), key=lambda kv: kv[1][0])
    name, (tot_ms, cnt, fl, by) = dom
    avg_ms = tot_ms / cnt
    achieved = fl / (avg_ms * 1e-3) / 1e12
    step_flops = sum(s[2] for k, s in kstats.items() if not k.startswith("row_pass"))
    step_bytes = sum(s[3] for k, s in kstats.items() if not k.startswith("row_pass"))
    xrec = kstats.get("row_pass_executed")
    executed = xrec[2] / (xrec[0] / xrec[1] * 1e-3) / 1e12 if xrec else achieved
    kern = {k: {"avg_ms": v[0] / v[1], "launches": v[1], "tflops": v[2] / (v[0] / v[1] * 1e-3) / 1e12,
                "gbs": v[3] / (v[0] / v[1] * 1e-3) / 1e9} for k, v in sorted(kstats.items())}
    dom64 = ("row_pass", kstats64["row_pass"]) if "row_pass" in kstats64 else max(kstats64.items(), key=lambda kv: kv[1][0])
    n64, (tm64, c64, fl64, _) = dom64
    ach64 = fl64 / (tm64 / c64 * 1e-3) / 1e12
    traffic = _traffic_entry(args.workload, name) if name in TRAFFIC_GROUPS else None

    line = {
        "metric": METRIC,
        "value": value,
        "unit": "elements/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": DTYPES[args.prec],
        "data": "synthetic",
        "config": workload_config(wl, info, args.workload),
        "matrix_gbs": (info.nvals + info.ndofs) * 4 / (ms_step * 1e-3) / 1e9,
        "roofline": {
            "bound": "alu",
            "kernel": name,
            "achieved": achieved,
            "peak": alu_peak,
            "unit": "TFLOP/s",
            "frac": achieved / alu_peak,
            "traffic": traffic,
            "peak_note": f"FP32 FMA peak = {sms} SMs (device attribute) x 128 lanes x 2 flops x {sm_max:.0f} MHz "
                         f"(sm_max from MEASURED_PEAKS.json, {peak_src})",
            "unit_note": "row_pass = all row-kernel launches of one recorded pass (per degree group: the "
                         "moment volume launch and the row kernel), first start to last end; achieved = their "
                         "algorithmic flops (the quadrature formulation's count) / that span",
            "executed_tflops": executed,
            "frac_executed": executed / alu_peak,
            "executed_note": "the flops the launches executed over the same span, against the same peak: the FP32 "
                             "pipe's actual use; the moment form of the volume terms executes fewer operations than "
                             "the quadrature sums it forms, so frac (credited) exceeds frac_executed",
        },
        "step_algorithmic": {"tflops": step_flops / (ms_step * 1e-3) / 1e12,
                             "gbs": step_bytes / (ms_step * 1e-3) / 1e9},
        "kernels": kern,
        "kernel_timing": kstats_src,
        "graph": ginfo,
        "fp64_form": {
            "value": ws * info.ne / (ms64 * 1e-3),
            "ms_per_step": ms64,
            "steps": k64,
            "speedup_fp32_over_fp64": ms64 / ms_step,
            "roofline": {"bound": "alu", "kernel": n64, "achieved": ach64, "peak": FP64_PEAK_TFLOPS,
                         "unit": "TFLOP/s", "frac": ach64 / FP64_PEAK_TFLOPS},
        },
        "form": args.prec,
        "reduced_vs_fp64_error": {"matrix_rel_fro": err_fro, "matrix_rel_max": err_max, "rhs_rel_fro": err_rhs},
        "other_forms": forms,
        "upload_ms": upload_ms,
        "pattern_ms": pattern_ms,
        "pattern": pattern,
        "e2e": {"value": ws * info.ne / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": h2d,
                "d2h_bytes_per_step": d2h, "ms_per_step": 1e3 * e2e_s,
                "mode": "dg_assemble_host_submit / _wait, two steps in flight (step k's copy back beside "
                        "step k+1's pass); every step copies its inputs in and its system back",
                "sync_ms_per_step": 1e3 * e2e_sync_s,
                "sync_value": ws * info.ne / e2e_sync_s},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "timed_wall_s": t_wall,
    }
    if ws == 1 and not args.no_cpu_baseline and not isinstance(wl, _Batch):
        line["cpu_baseline"], (om, ob) = cpu_baseline_sample(wl)
        # the headline form's result against the oracle on the same sample
        g32.dg_graph_launch()
        torch.cuda.synchronize()
        line["error_vs_oracle"] = oracle_error(mesh, v32.double().cpu().numpy(), r32.double().cpu().numpy(), om, ob)
    elif ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"], _ = cpu_baseline_sample(wl.members[0])
        line["cpu_baseline"]["sample"] = "batch member 0: " + line["cpu_baseline"]["sample"]
    emit(line)
    return 0


def slab_cpu_sample(space_name: str, n_sites: int = 40):
    """The slab oracle (oracle/spacetime.py) as it stands on a bounded sample:
    one slab over a 40-cell mesh of the adr2d recipe (p~U{1..4}, a=10^U(-2,2),
    b=(1,0.5), c=1, sin-product data).  Its source takes no element, so f is
    evaluated with the first element's a (the cost is the same)."""
    import oracle as O
    from oracle import spacetime as S
    from paper_2007_04881_gb300 import configs

    wl = configs.small2d(n_sites, 1, 1, 4, b=(1.0, 0.5), c=1.0)
    om = O.Mesh(wl.mesh)
    pb = O.make_problem(2, **wl.problem)
    a0 = float(wl.a[0])
    sl = S.Slab(om, wl.p.astype(np.int32), wl.a, (1.0, 0.5), 1.0, space_name, 0.0, 0.01)
    t = time.perf_counter()
    sl.assemble(lambda tt, x: O.source_f(pb, a0, x), lambda tt, x: O.exact_u(pb, x), lambda e, x: 0.0)
    dt = time.perf_counter() - t
    return {"value": om.ne / dt, "unit": "elements/s", "cores": 1, "kind": "oracle",
            "sample": f"one {space_name} slab over a {om.ne}-cell mesh of the same recipe, FP64, plain numpy "
                      f"(one thread), {dt:.1f} s"}


def varcoef_flops(mesh, p, dim: int) -> float:
    """Contraction flops of the variable-coefficient kernels over one pass:
    2 N^2 per volume point and per own-face point of each element, 2 N N_k
    per interface point of each off-diagonal block (the kernel contracts
    every point; outflow points carry zero rows), and 2 N per point of the
    load vector."""
    from math import comb

    ne = mesh.ne
    p = np.asarray(p, dtype=np.int64)
    nb = np.array([comb(int(q) + dim, dim) for q in p], dtype=np.float64)
    sub = np.bincount(mesh.dg_mesh_array("sub_elem"), minlength=ne).astype(np.float64)
    nvol = sub * (p + 2.0) ** dim
    nqf = mesh.dg_mesh_array("e_nqf").astype(np.float64)
    hf_ptr = mesh.dg_mesh_array("hf_ptr")
    hf_qoff = mesh.dg_mesh_array("hf_qoff").astype(np.int64)
    nhf = int(hf_ptr[-1])
    owner = np.repeat(np.arange(ne), np.diff(hf_ptr))
    nxt = np.append(hf_qoff[1:], 0)
    last = np.zeros(nhf, dtype=bool)
    last[hf_ptr[1:][np.diff(hf_ptr) > 0] - 1] = True
    pts = np.where(last, nqf[owner].astype(np.int64), nxt) - hf_qoff
    rec = mesh.dg_mesh_array("blk_rec").reshape(-1, 4)
    row_ptr = mesh.dg_mesh_array("row_ptr")
    rows = np.repeat(np.arange(ne), np.diff(row_ptr))
    off = rec[:, 0] >= 0
    cs = np.concatenate([[0], np.cumsum(pts)])
    bpts = cs[rec[off, 1] + rec[off, 2]] - cs[rec[off, 1]]
    nk = np.array([comb(int(q) + dim, dim) for q in rec[off, 3]], dtype=np.float64)
    fl = float(np.sum((nvol + nqf) * 2.0 * nb * nb) + np.sum(bpts * 2.0 * nb[rows[off]] * nk) +
               np.sum((nvol + nqf) * 2.0 * nb))
    return fl


def run_varcoef(args):
    """The 3D test problem of Sec. 4.2 through dg_assemble_varcoef_form."""
    wl = make_workload(args.workload)
    import torch

    from paper_2007_04881_gb300 import build as B
    from paper_2007_04881_gb300 import dg

    ws, rank, local = dist_setup(True)
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    B.build()
    stream = torch.cuda.current_stream()
    ctx = dg.Context(dev, stream.cuda_stream)
    mesh = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(**wl.problem))
    info = mesh.info
    prec = dg.DG_PREC_FP32
    vals = torch.empty(info.nvals, dtype=torch.float32, device="cuda")
    rhs = torch.empty(info.ndofs, dtype=torch.float32, device="cuda")
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    step = lambda: mesh.dg_assemble_varcoef(vals, rhs, prec=prec)  # noqa: E731
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    ctx.dg_set_timing(True)
    step()
    torch.cuda.synchronize()
    launches_per_step = ctx.launches()
    sampler = ClockSampler(dev)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    times, kstats = time_steps(torch, stream, step, flush, args.steps, ctx)
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ctx.dg_set_timing(False)
    ms_step = max_over_ranks(sum(times) / len(times), ws)
    value = ws * info.ne / (ms_step * 1e-3)

    # the FP64 form (few steps: FP64 runs at 1/64 of the FP32 rate on this part)
    v64 = torch.empty(info.nvals, dtype=torch.float64, device="cuda")
    r64 = torch.empty(info.ndofs, dtype=torch.float64, device="cuda")
    mesh.dg_assemble_varcoef(v64, r64, prec=dg.DG_PREC_FP64)
    torch.cuda.synchronize()
    t64 = []
    for _ in range(3):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        flush.zero_()
        e0.record(stream)
        mesh.dg_assemble_varcoef(v64, r64, prec=dg.DG_PREC_FP64)
        e1.record(stream)
        torch.cuda.synchronize()
        t64.append(e0.elapsed_time(e1))
    err = {"matrix_rel_fro": float(torch.linalg.norm(vals.double() - v64) / torch.linalg.norm(v64)),
           "rhs_rel_fro": float(torch.linalg.norm(rhs.double() - r64) / torch.linalg.norm(r64))}

    # end to end through the public calls: the field table from the host, the
    # system back to pinned host memory
    hv = torch.empty(info.nvals, dtype=torch.float32).pin_memory()
    hr = torch.empty(info.ndofs, dtype=torch.float32).pin_memory()

    def e2e_step():
        mesh.dg_mesh_set_fields((1.0, 1.0, 1.0), np.eye(3), [3.0] + [0.0] * 14 + [1.0])
        mesh.dg_assemble_varcoef(vals, rhs, prec=prec)
        hv.copy_(vals, non_blocking=True)
        hr.copy_(rhs, non_blocking=True)
        torch.cuda.synchronize()

    e2e_steps = max(3, min(args.steps, 10))
    e2e_step()
    barrier(ws)
    t = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = max_over_ranks((time.perf_counter() - t) / e2e_steps, ws)
    if rank != 0:
        return 0

    kname = "varcoef_terms_f32"
    kt = kstats.get(kname)
    avg_ms = kt[0] / kt[1] if kt else float("nan")
    flops = varcoef_flops(mesh, wl.p, wl.dim)
    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    sms = device_sms()
    alu_peak = fp32_alu_peak_tflops(sm_max, sms)
    achieved = flops / (avg_ms * 1e-3) / 1e12
    kern = {k: {"avg_ms": v[0] / v[1], "launches": v[1]} for k, v in sorted(kstats.items())}
    cfg = workload_config(wl, info, args.workload)
    cfg["fields"] = "b = (1+x, 1+y, 1+z), c = 3 + xyz (Sec. 4.2), A = 0.01 I"
    cfg["l2"] = "system larger than L2; L2 flushed between timed steps (256 MiB write, outside the timed region)"
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "elements/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": cfg,
        "matrix_gbs": (info.nvals + info.ndofs) * 4 / (ms_step * 1e-3) / 1e9,
        "roofline": {
            "bound": "alu", "kernel": kname, "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
            "frac": achieved / alu_peak, "traffic": None,
            "peak_note": f"FP32 FMA peak = {sms} SMs x 128 lanes x 2 flops x {sm_max:.0f} MHz (sm_max from "
                         f"MEASURED_PEAKS.json, {peak_src})",
            "unit_note": f"{flops:.4g} contraction flops per launch group (2 N^2 per volume and own-face point, "
                         "2 N N_k per interface point, 2 N per load point) / the launch group's event time",
        },
        "kernels": kern,
        "fp64_form": {"ms_per_step": sum(t64) / len(t64), "value": info.ne / (sum(t64) / len(t64) * 1e-3)},
        "fp32_vs_fp64": err,
        "e2e": {"value": ws * info.ne / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": 8 * 32,
                "d2h_bytes_per_step": (info.nvals + info.ndofs) * 4, "ms_per_step": 1e3 * e2e_s},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "timed_wall_s": t_wall,
    }
    if ws == 1 and not args.no_cpu_baseline:
        import copy

        wo = copy.copy(wl)
        wo.problem = dict(wl.problem, coef=1)
        cb, (om, ob) = cpu_baseline_sample(wo, seconds_target=8.0)
        line["cpu_baseline"] = cb
        line["error_vs_oracle"] = oracle_error(mesh, vals.double().cpu().numpy(), rhs.double().cpu().numpy(), om, ob)
    emit(line)
    return 0


def run_slab(args):
    """One space-time slab step (dg_assemble_slab) over the adr2d_65k mesh."""
    wl = make_workload(args.workload)
    import torch

    from paper_2007_04881_gb300 import build as B
    from paper_2007_04881_gb300 import dg

    ws, rank, local = dist_setup(True)
    dev = local if ws > 1 else 0
    torch.cuda.set_device(dev)
    B.build()
    stream = torch.cuda.current_stream()
    ctx = dg.Context(dev, stream.cuda_stream)
    mesh = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, dg.Problem(**wl.problem))
    info = mesh.info
    space = dg.DG_SPACE_PQ if args.workload.endswith("_pq") else dg.DG_SPACE_P
    prec = dg.DG_PREC_FP32
    t0, t1 = 0.0, 0.01
    nv, nd = mesh.dg_slab_layout(space)
    vals = torch.empty(nv, dtype=torch.float32, device="cuda")
    rhs = torch.empty(nd, dtype=torch.float32, device="cuda")
    u_prev = torch.randn(mesh.ndofs, dtype=torch.float32, device="cuda", generator=torch.Generator("cuda").manual_seed(3))
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    direct = lambda: mesh.dg_assemble_slab(prec, space, t0, t1, vals, rhs, u_prev)  # noqa: E731
    for _ in range(args.warmup):
        direct()
    torch.cuda.synchronize()
    # the slab step recorded as one CUDA graph (per-launch timing events inside)
    ctx.dg_set_timing(True)
    graph = mesh.dg_slab_graph_create(prec, space, t0, t1, vals, rhs, u_prev)
    step = graph.dg_graph_launch
    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    launches_per_step = ctx.launches()
    sampler = ClockSampler(dev)
    barrier(ws)
    torch.cuda.synchronize()
    sampler.start()
    t_wall = time.perf_counter()
    times, kstats = time_steps(torch, stream, step, flush, args.steps, ctx)
    t_wall = time.perf_counter() - t_wall
    torch.cuda.synchronize()
    barrier(ws)
    clocks = sampler.stop()
    ctx.dg_set_timing(False)
    ms_step = max_over_ranks(sum(times) / len(times), ws)
    value = ws * info.ne / (ms_step * 1e-3)

    # end to end: u_prev from pinned host memory, the slab system back to it
    hu = u_prev.cpu().pin_memory()
    hv = torch.empty(nv, dtype=torch.float32).pin_memory()
    hr = torch.empty(nd, dtype=torch.float32).pin_memory()
    du = torch.empty_like(u_prev)

    def e2e_step():
        du.copy_(hu, non_blocking=True)
        mesh.dg_assemble_slab(prec, space, t0, t1, vals, rhs, du)  # the public call, not the recording
        hv.copy_(vals, non_blocking=True)
        hr.copy_(rhs, non_blocking=True)
        torch.cuda.synchronize()

    e2e_steps = max(3, min(args.steps, 10))
    e2e_step()
    barrier(ws)
    t = time.perf_counter()
    for _ in range(e2e_steps):
        e2e_step()
    e2e_s = max_over_ranks((time.perf_counter() - t) / e2e_steps, ws)
    if rank != 0:
        return 0

    # roofline of the expansion kernel: it writes the slab matrix once and
    # reads every spatial block and every diagonal block of the mass matrix once
    row_ptr, col, blk_off, _ = mesh.dg_bsr_pattern()
    rows = np.repeat(np.arange(info.ne), np.diff(row_ptr))
    diag_entries = int(np.diff(blk_off)[col == rows].sum())
    alg_bytes = 4 * (nv + int(info.nvals) + diag_entries)
    kname = "slab_matrix_f32"
    kt = kstats.get(kname)
    avg_ms = kt[0] / kt[1] if kt else float("nan")
    achieved = alg_bytes / (avg_ms * 1e-3) / 1e9
    peaks, peak_src = _peaks()
    peak = float(peaks.get("hbm_gbs", 6800.0))
    kern = {k: {"avg_ms": v[0] / v[1], "launches": v[1]} for k, v in sorted(kstats.items())}
    cfg = workload_config(wl, info, args.workload)
    cfg.update({"slab_matrix_entries": int(nv), "slab_dofs": int(nd), "space": "PQ" if space else "P",
                "slab": [t0, t1]})
    line = {
        "metric": METRIC,
        "value": value,
        "unit": "elements/s",
        "n_gpus": ws,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": ms_step,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": cfg,
        "matrix_gbs": (nv + nd) * 4 / (ms_step * 1e-3) / 1e9,
        "roofline": {
            "bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "unit": "GB/s",
            "frac": achieved / peak, "traffic": _traffic_entry(args.workload, "slab_matrix"),
            "unit_note": f"algorithmic bytes per launch = 4 x (slab entries written {nv} + spatial entries read "
                         f"{int(info.nvals)} + mass-matrix entries read {diag_entries}); peak hbm_gbs of "
                         f"MEASURED_PEAKS.json ({peak_src})",
        },
        "kernels": kern,
        "e2e": {"value": ws * info.ne / e2e_s, "unit": "elements/s", "h2d_bytes_per_step": hu.numel() * 4,
                "d2h_bytes_per_step": (nv + nd) * 4, "ms_per_step": 1e3 * e2e_s},
        "gpu_launches": launches_per_step * args.steps,
        "clocks": clocks,
        "timed_wall_s": t_wall,
    }
    if ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = slab_cpu_sample("PQ" if space else "P")
    emit(line)
    return 0


# kernel groups whose DRAM traffic --record-traffic stores: the ncu kernel
# names they match, and the sources they are compiled from (translation
# units by name prefix, and the headers they include)
TRAFFIC_GROUPS = {
    "row_pass": {"units": ("dg_row",), "headers": ("dg_device.cuh", "dg_moment.cuh", "dg_launch.cuh",
                                                   "dg_iface.cuh", "dg_internal.h"),
                 "match": ("row_lane_kernel", "row_kernel", "vol_moment_kernel", "iface_kernel")},
    "slab_matrix": {"units": ("dg_slab",), "headers": ("dg_slab.cuh", "dg_internal.h"),
                    "match": ("slab_matrix_kernel",)},
}


def _kernel_source_sha(group="row_pass") -> str:
    """Hash of the sources a kernel group is compiled from: its translation
    units, its headers and the library header."""
    import hashlib

    g = TRAFFIC_GROUPS[group]
    h = hashlib.sha1()
    csrc = os.path.join(ROOT, "paper_2007_04881_gb300", "csrc")
    for fn in sorted(os.listdir(csrc)):
        if fn in g["headers"] or (fn.startswith(g["units"]) and fn.endswith(".cu")):
            h.update(open(os.path.join(csrc, fn), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "dg.h"), "rb").read())
    return h.hexdigest()[:16]


def _traffic_entry(workload: str, group: str):
    """Bytes per launch of a kernel group from profiles/traffic.json, or
    None when absent or taken on other sources."""
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        ent = json.load(open(tfile)).get(workload, {}).get(group)
        if ent and ent.get("source_sha") == _kernel_source_sha(group):
            return ent.get("bytes_per_launch")
    except Exception:
        pass
    return None


def record_traffic(csv_path: str, workload: str, group: str, launches: int) -> int:
    """Store in profiles/traffic.json the DRAM bytes (read + write) of one
    launch group from an ncu CSV log (--metrics dram__bytes_read.sum,
    dram__bytes_write.sum --csv --log-file): the first ``launches`` captured
    launches of the group's kernels, summed, per kernel name as well, with the
    hash of the sources they were built from."""
    import csv

    rows = {}
    with open(csv_path) as f:
        lines = [ln for ln in f if ln.startswith('"')]
    for r in csv.DictReader(lines):
        name = r.get("Kernel Name", "")
        if not any(name.startswith(k) or (k + "<") in name for k in TRAFFIC_GROUPS[group]["match"]):
            continue
        lid = r.get("ID")
        ent = rows.setdefault(lid, {"kernel": name, "bytes": 0.0})
        if r.get("Metric Name") in ("dram__bytes_read.sum", "dram__bytes_write.sum"):
            scale = {"byte": 1, "Kbyte": 1e3, "Mbyte": 1e6, "Gbyte": 1e9, "KB": 1024, "MB": 1024 ** 2,
                     "GB": 1024 ** 3}.get(r.get("Metric Unit", "byte"), 1)
            ent["bytes"] += float(r["Metric Value"].replace(",", "")) * scale
    ids = sorted(rows, key=lambda k: int(k))[:launches]
    if len(ids) < launches:
        print(f"record-traffic: {len(ids)} launches of {group} in {csv_path}, expected {launches}")
        return 1
    per = {}
    for k in ids:
        per[rows[k]["kernel"]] = per.get(rows[k]["kernel"], 0) + int(rows[k]["bytes"])
    tfile = os.path.join(ROOT, "profiles", "traffic.json")
    tj = json.load(open(tfile)) if os.path.exists(tfile) else {}
    tj.setdefault(workload, {})[group] = {
        "bytes_per_launch": int(sum(per.values())),
        "source_sha": _kernel_source_sha(group),
        "launches": launches,
        "per_kernel": per,
        "note": "dram__bytes_read.sum + dram__bytes_write.sum of the group's captured launches of one pass, "
                "summed; ncu flushes the caches before each captured launch",
    }
    json.dump(tj, open(tfile, "w"), indent=1)
    print(json.dumps(tj[workload][group]))
    return 0


def run_learned(args):
    """The learned-quadrature workload: train the proposal network on the
    method's own converged rules, then measure on the 262,144-cell mesh."""
    from paper_2007_04881_gb300 import configs

    train = configs.learned_training_meshes()  # process pool before any CUDA call
    wl = configs.learned2d()
    import torch

    from paper_2007_04881_gb300 import build as B
    from paper_2007_04881_gb300 import dg

    torch.cuda.set_device(0)
    B.build()
    stream = torch.cuda.current_stream()
    ctx = dg.Context(0, stream.cuda_stream)
    t0 = time.perf_counter()
    feats, tgts = [], []
    for w in train:
        m = dg.Mesh(ctx, w.mesh, w.p, w.a, dg.Problem(**w.problem))
        m.dg_quad_prepare()
        m.dg_quad_fit(None, iters=10, install=False)
        t = torch.zeros(m.ne, 84, dtype=torch.float32, device="cuda")
        m.dg_quad_targets(t)
        b = m.dg_quad_buffers()
        ok = dg.device_view(b["ok"], (m.ne,), "i4").clone().bool()
        feats.append(dg.device_view(b["feat"], (m.ne, 24), "bf16").clone()[ok])
        tgts.append(t[ok])
        m.close()
    X = torch.cat(feats)
    T = torch.cat(tgts)
    torch.cuda.synchronize()
    targets_s = time.perf_counter() - t0
    net = dg.MLP(ctx, seed=0)
    g = torch.Generator(device="cuda")
    g.manual_seed(0)
    bs, epochs = 1024, args.epochs
    loss = torch.zeros(1, device="cuda")
    t0 = time.perf_counter()
    nstep = 0
    for ep in range(epochs):
        perm = torch.randperm(X.shape[0], device="cuda", generator=g)
        lr = 2e-3 * 0.5 * (1 + math.cos(math.pi * ep / epochs))
        for i in range(0, X.shape[0] - bs + 1, bs):
            idx = perm[i:i + bs]
            net.train_step(X[idx].contiguous(), T[idx].contiguous(), bs, lr, loss)
            nstep += 1
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t0
    final_loss = float(loss.item())

    pb = dg.Problem(**wl.problem)
    mesh = dg.Mesh(ctx, wl.mesh, wl.p, wl.a, pb)
    info = mesh.info
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device="cuda")
    v32 = torch.empty(mesh.nvals, dtype=torch.float32, device="cuda")
    r32 = torch.empty(mesh.ndofs, dtype=torch.float32, device="cuda")
    v64 = torch.empty(mesh.nvals, dtype=torch.float64, device="cuda")
    r64 = torch.empty(mesh.ndofs, dtype=torch.float64, device="cuda")

    def timed_graph(prec, vals, rhs, steps, timing):
        ctx.dg_set_timing(timing)
        gr = mesh.dg_graph_create(prec, vals, rhs, autotune=(prec == dg.DG_PREC_FP32))
        for _ in range(3):
            gr.dg_graph_launch()
        torch.cuda.synchronize()
        ts, ks = time_steps(torch, stream, gr.dg_graph_launch, flush, steps, ctx if timing else None)
        ctx.dg_set_timing(False)
        return sum(ts) / len(ts), ks, gr

    # sub-triangle rules: FP32 and FP64 forms
    fan32_ms, _, _ = timed_graph(dg.DG_PREC_FP32, v32, r32, args.steps, False)
    fan64_ms, _, g64 = timed_graph(dg.DG_PREC_FP64, v64, r64, 3, False)
    g64.dg_graph_launch()
    torch.cuda.synchronize()
    ref64 = v64.clone()
    # learned rules: one-shot cost (moments + network + 3 Gauss-Newton steps + install)
    out = torch.zeros(info.ne, 84, dtype=torch.float32, device="cuda")
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    mesh.dg_quad_prepare()
    b = mesh.dg_quad_buffers()
    net.forward(b["feat"], info.ne, out)
    st = mesh.dg_quad_fit(out, iters=3, install=True)
    torch.cuda.synchronize()
    oneshot_ms = 1e3 * (time.perf_counter() - t0)
    fixed3 = None
    # amortised: assembly with the cached rules
    sampler = ClockSampler(0)
    sampler.start()
    lrn32_ms, kstats, _ = timed_graph(dg.DG_PREC_FP32, v32, r32, args.steps, True)
    clocks = sampler.stop()
    lrn64_ms, _, gl64 = timed_graph(dg.DG_PREC_FP64, v64, r64, 3, False)
    gl64.dg_graph_launch()
    torch.cuda.synchronize()
    e64 = float(torch.linalg.vector_norm(v64 - ref64) / torch.linalg.vector_norm(ref64))
    e32 = float(torch.linalg.vector_norm(v32.double() - ref64) / torch.linalg.vector_norm(ref64))
    e32max = float((v32.double() - ref64).abs().max() / ref64.abs().max())
    resid = dg.device_view(b["resid"], (info.ne,), "f4").cpu().numpy()
    okv = dg.device_view(b["ok"], (info.ne,), "i4").cpu().numpy().astype(bool)
    # end to end through the host-memory entry point, learned rules installed
    pin = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a, dtype=dt)).pin_memory()  # noqa: E731
    hx, hy, ha = pin(wl.mesh.x, np.float64), pin(wl.mesh.y, np.float64), pin(wl.a, np.float64)
    hv = torch.empty(mesh.nvals, dtype=torch.float32).pin_memory()
    hr = torch.empty(mesh.ndofs, dtype=torch.float32).pin_memory()
    for _ in range(2):
        mesh.dg_assemble_host(dg.DG_PREC_FP32, hv, hr, x=hx, y=hy, a=ha)
    e2e_steps = max(3, min(args.steps, 20))
    t = time.perf_counter()
    for _ in range(e2e_steps):
        mesh.dg_assemble_host(dg.DG_PREC_FP32, hv, hr, x=hx, y=hy, a=ha)
    e2e_s = (time.perf_counter() - t) / e2e_steps
    e2e = {"value": info.ne / e2e_s, "unit": "elements/s",
           "h2d_bytes_per_step": (hx.numel() + hy.numel() + ha.numel()) * 8,
           "d2h_bytes_per_step": (hv.numel() + hr.numel()) * 4, "ms_per_step": 1e3 * e2e_s}
    # the same budget from the fixed start (no network)
    mesh.dg_quad_clear()
    fixed3 = mesh.dg_quad_fit(None, iters=3, install=False)
    fixed4 = mesh.dg_quad_fit(None, iters=4, install=False)
    learned4 = mesh.dg_quad_fit(out, iters=4, install=False)

    peaks, peak_src = _peaks()
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    alu_peak = fp32_alu_peak_tflops(sm_max, device_sms())
    unit = kstats.get("row_pass") or max(kstats.values(), key=lambda v: v[0])
    achieved = unit[2] / (unit[0] / unit[1] * 1e-3) / 1e12
    ne = info.ne
    amort = {f"K={k}": ne / ((oneshot_ms + k * lrn32_ms) * 1e-3 / k) for k in (1, 10, 100)}
    line = {
        "metric": METRIC,
        "value": ne / (lrn32_ms * 1e-3),
        "unit": "elements/s",
        "n_gpus": 1,
        "steps": args.steps,
        "warmup": args.warmup,
        "ms_per_step": lrn32_ms,
        "higher_is_better": True,
        "scaling": "weak",
        "vs_baseline": None,
        "dtype": "f32",
        "data": "synthetic",
        "config": workload_config(wl, info, "learned2d_262k"),
        "roofline": {"bound": "alu", "kernel": "row_pass", "achieved": achieved, "peak": alu_peak, "unit": "TFLOP/s",
                     "frac": achieved / alu_peak, "traffic": None},
        "learned": {
            "accepted": st["accepted"], "eligible": st["eligible"], "fallback": ne - st["accepted"],
            "max_accepted_moment_residual": float(resid[okv].max()) if okv.any() else None,
            "accepted_at_3_steps_fixed_start": fixed3["accepted"], "accepted_at_4_steps_fixed_start": fixed4["accepted"],
            "accepted_at_4_steps_learned": learned4["accepted"],
            "oneshot_ms": oneshot_ms, "assembly_fp32_ms": lrn32_ms, "assembly_fp64_ms": lrn64_ms,
            "subtriangle_fp32_ms": fan32_ms, "subtriangle_fp64_ms": fan64_ms,
            "amortised_elements_per_s": amort,
            "matrix_rel_fro_vs_subtriangle_fp64": {"learned_fp32": e32, "learned_fp64": e64},
            "matrix_rel_max_learned_fp32": e32max,
            "training": {"polygons": int(X.shape[0]), "epochs": epochs, "steps": nstep, "batch": bs,
                         "targets_s": targets_s, "train_s": train_s, "final_loss": final_loss},
        },
        "e2e": e2e,
        "gpu_launches": mesh.ctx.launches() * args.steps,
        "clocks": clocks,
    }
    emit(line)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="adr2d_65k", choices=sorted(WORKLOADS))
    ap.add_argument("--ref-sample", type=int, default=512, help="oracle elements per reference step")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--prec", default="fp32", choices=sorted(PRECS),
                    help="form of the timed pass: FP32 contractions, or split-BF16 / 3xTF32 tensor-core contractions")
    ap.add_argument("--epochs", type=int, default=40, help="training epochs of the learned-rule workload")
    ap.add_argument("--jsonl", metavar="FILE", help="also append each bench line to this JSONL run log")
    ap.add_argument("--record-traffic", metavar="CSV", help="store the DRAM traffic of --traffic-group from an ncu "
                    "CSV log in profiles/traffic.json for --workload, and exit")
    ap.add_argument("--traffic-group", default="row_pass", choices=sorted(TRAFFIC_GROUPS))
    ap.add_argument("--traffic-launches", type=int, default=6, help="captured launches that make one pass")
    args = ap.parse_args()
    emit.jsonl = args.jsonl
    if args.record_traffic:
        return record_traffic(args.record_traffic, args.workload, args.traffic_group, args.traffic_launches)
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "learned2d_262k":
        return run_learned(args)
    if args.workload.startswith("slab2d"):
        return run_slab(args)
    if args.workload.startswith("adr3d_varcoef"):
        return run_varcoef(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
