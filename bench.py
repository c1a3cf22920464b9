"""Benchmark: assembly of all unique blocks of the block-Hessenberg system,
then block-Hessenberg matvecs with the assembled matrix.

One step = one tdbem_assemble_all call (psi tables, element-pair bounds,
vertex-pair windows, far and near quadrature, per-block CSR) on a mesh and
time grid already resident on the device, followed by --matvecs (default
20) tdbem_hessenberg_apply calls on seeded N(0,1) vectors already resident
on the device. value = structural nonzeros assembled per second of the whole
step. e2e: the same step through the public API from host data: mesh, time
grid and the right-hand sides copied in (vectors from pinned memory), every
matvec result copied back to pinned host memory. Prints one JSON line.

On one GPU the line carries two sub-records: "graded", the same measurement
on the graded torus (8192 triangles, 97 grid points, every nonzero block
unique; one warm-up and two timed steps), and "potential", the retarded
double layer potential at 257 x 257 points on a plane and 40 grid times
(tdbem_double_layer; point-times per second).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--config NAME] [--impl ours|reference]

--impl reference times the FP64 CPU oracle (the reference arm of this
project) on a bounded row sample of the same workload on the host cores.
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_1503_07221_gb300 import inputs  # noqa: E402

CONFIGS = {
    # name: (workload builder, precision label)
    "sphere20480": "icosphere 20480 triangles / 10242 vertices, N=129 points, dt=0.05 on [0,6.4], c=1, p=0",
    "sphere5120j": "icosphere 5120 / 2562 jittered +-1% h (seed 0), N=65 points, dt=0.0625 on [0,4], c=1, p=0",
    "sphere320": "icosphere 320 / 162, N=17 points, dt=0.25 on [0,4], c=1, p=0",
    "sphere5120p": "icosphere 5120 / 2562, N=65 points, dt=0.07 on [0,4.48], c=1, p=0 (far-kernel profiling case)",
    "torus8192g": "torus R=1 r=0.4, 128x32 quads (8192 triangles / 4096 vertices), graded grid of 96 steps "
                  "with ratio 1.02 on [0,6] (N=97 points), c=1, p=0; every nonzero block assembled",
    "torus2048g": "torus R=1 r=0.4, 64x16 quads (2048 triangles / 1024 vertices), the same graded grid",
}


def workload(name):
    w = inputs.workload(name)
    return w.verts, w.tris, w.t


def is_graded(name):
    return not inputs.workload(name).equidistant


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu=0):
        self.gpu = gpu
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except OSError:
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx.append(float(f[2]))
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unavailable"], "samples": 0}
        return {"sm_mhz": float(np.median(sm)), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def cpu_sample(V, F, t, rows_n, seed=0, equidistant=True, blocks_n=None, psi_mode="interp"):
    """Time the FP64 oracle on a fixed row sample (all unique blocks, or a
    seeded sample of blocks_n of them)."""
    from oracle.oracle import Oracle, num_threads
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(V.shape[0], size=rows_n, replace=False))
    t0 = time.perf_counter()
    o = Oracle(V, F, t, equidistant=equidistant, psi_mode=psi_mode)
    t1 = time.perf_counter()
    nb = o.num_blocks()
    blks = np.arange(nb) if blocks_n is None else np.sort(rng.choice(nb, size=min(blocks_n, nb), replace=False))
    res = o.assemble_rows(rows, blks)
    t2 = time.perf_counter()
    nnz = sum(len(c) for b in res.values() for (c, f, n) in b)
    return {"nnz": nnz, "seconds": t2 - t0, "setup_s": t1 - t0, "rows": int(rows_n), "cores": num_threads(),
            "blocks": int(blks.size)}


def cpu_sample_args(args):
    # graded grids: every nonzero block is unique (thousands); the oracle then
    # takes 2 rows x a seeded sample of 60 blocks to stay within ~30 s
    if is_graded(args.config):
        return {"rows_n": min(args.cpu_rows, 2), "equidistant": False, "blocks_n": 60}
    return {"rows_n": args.cpu_rows, "equidistant": True, "blocks_n": None}


def config_dict(name, precision, world):
    return {"workload": name, "desc": CONFIGS[name], "precision": precision,
            "parallelism": "replicas" if world > 1 else "single GPU",
            "l2": "working set (element-pair records, lag windows, CSR) far larger than L2"}


def reference_rows(args):
    # each step of the reference arm is a bounded sample: with K steps the
    # whole run stays near three minutes on 16 cores (~1.2 s per row)
    return max(2, min(args.cpu_rows, int(160 // max(args.steps, 1))))


def run_reference(args):
    V, F, t = workload(args.config)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ca = cpu_sample_args(args)
    if not is_graded(args.config):
        ca["rows_n"] = reference_rows(args)
    rows_n = ca["rows_n"]
    rates, secs = [], []
    for _ in range(args.steps):
        s = cpu_sample(V, F, t, **ca)
        rates.append(s["nnz"] / s["seconds"])
        secs.append(s["seconds"])
    v = float(np.median(rates))
    sample = "%d random rows (seed 0) x %d unique blocks of %s per step" % (rows_n, s["blocks"], args.config)
    line = {
        "impl": "reference", "metric": "assembled nonzeros/s", "value": v, "unit": "nonzeros/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.median(secs)) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": config_dict(args.config, args.precision, args.gpus),
        "cpu_baseline": {"value": v, "unit": "nonzeros/s", "cores": s["cores"], "kind": "oracle",
                         "sample": sample},
        "e2e": {"value": v, "unit": "nonzeros/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))


def max_over_ranks(x, dist, device):
    """The largest of every rank's x (the job takes as long as its slowest
    replica); x unchanged without a process group."""
    if dist is None:
        return float(x)
    import torch
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank, world, ms):
    """Whole-job rate: the units every replica processed over the slowest time."""
    return units_per_rank * world / (ms * 1e-3)


# DRAM bytes (read + written) of one far phase, all colour launches of one
# assembly, from one single-pass ncu capture of the current far kernel on
# that workload (summary under profiles/); None where no capture exists.
# An entry goes when the kernel changes.
FAR_TRAFFIC = {"sphere20480": 202.30e9 + 132.86e9}


def far_flops(st):
    # algorithmic FP32 work of the far kernel per far point pair: distance
    # and Chebyshev argument (~14 FMA-equivalents), T_n recurrence (31 FMA),
    # 8 evaluated panels x (psi, psi~) x 33 coefficients (528 FMA; the other
    # two C2 panels follow from the antisymmetry of Eq. symmetryXi, 4 FMA-
    # equivalents), weights (4 FMA), accumulation 10 panels x 4 (40 FMA):
    # 621 FMA = 1242 FLOP. Compensation terms are not counted.
    return 1242.0 * st["far_pairs"] * 49


def gfar_flops(st):
    # graded grids (gfar_kernel): per far point pair and kept block, the T_n
    # recurrence (31 FMA) and the sums over 33 coefficients of psi and psi~
    # (66 FMA): 194 FLOP; 1/r scaling (2) and the four weighted sums (8):
    # 204 FLOP; per far point pair the distance and its FP64-anchored
    # correction, ~28 FLOP. Compensation terms are not counted.
    return 204.0 * st["quad_points_far"] + 28.0 * st["far_pairs"] * 49


def matvec_work(asm, N, graded):
    # every stored entry times the number of block positions that reuse its block
    w = 0
    for b in range(asm.num_blocks()):
        bi = asm.block_info(b)
        k, i = bi["k"], bi["i"]
        reuse = (N - 1 - k) if (i == 1 and 1 <= k <= N - 2) else ((N - 3) if (k == 1 and i == 2) else 1)
        if graded:
            reuse = 1
        w += (bi["nnz_far"] + bi["nnz_near"]) * reuse
    return w


def measure_assembly(name, precision, steps, warmup, matvecs, *, world=1, rank=0, local=0, dist=None,
                     do_e2e=True, fp64_compare=True, do_cpu=True, cpu_rows=16, staging_mb=0):
    """One record of the assembly bench on workload `name`: `warmup` untimed
    and `steps` timed steps (assembly + `matvecs` products), CUDA events on
    the launching stream, clocks sampled during the timed steps."""
    import torch
    from paper_1503_07221_gb300 import tdbem

    V, F, t = workload(name)
    graded = is_graded(name)
    prec = tdbem.PREC_MIXED if precision == "mixed" else tdbem.PREC_FP64
    mesh, grid = tdbem.Mesh(V, F), tdbem.TimeGrid(t)
    asm = tdbem.Assembler(mesh, grid, precision=prec, staging_mb=staging_mb)
    stream = torch.cuda.current_stream()
    N, M = t.size, V.shape[0]
    # matvec inputs: x_r ~ N(0, 1) from a CPU generator with seed r, copied once
    X = torch.empty((max(matvecs, 1), N, M), dtype=torch.float64, device="cuda")
    for r in range(X.shape[0]):
        gen = torch.Generator()
        gen.manual_seed(r)
        X[r].copy_(torch.randn((N, M), dtype=torch.float64, generator=gen))
    Y = torch.empty((N, M), dtype=torch.float64, device="cuda")

    def step(mv_events=None):
        asm.assemble()
        if mv_events:
            mv_events[0].record(stream)
        for r in range(matvecs):
            asm.hessenberg_apply(X[r], Y)
        if mv_events:
            mv_events[1].record(stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    far_ms, asm_ms, mv_ev = [], [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            step(e)
            mv_ev.append(e)
            far_ms.append(asm.stats()["ms_far"])
            asm_ms.append(asm.stats()["ms_total"])
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    mv_ms = float(np.mean([a.elapsed_time(b) for a, b in mv_ev])) / max(matvecs, 1)
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    st = asm.stats()
    nnz = st["nnz"]
    value = job_throughput(nnz, world, ms)
    qps = job_throughput(st["quad_points"], world, ms)
    nb = st["n_blocks"]
    launches_per_step = st["kernel_launches"] + 2 * matvecs  # transpose + product per matvec
    mv_work = matvec_work(asm, N, graded)
    # roofline of the dominant kernel (far field): FP32 FMA pipe
    far_avg_ms = float(np.mean(far_ms))
    flops = gfar_flops(st) if graded else far_flops(st)
    achieved = flops / (far_avg_ms * 1e-3) / 1e12
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peak_nominal = sm_count * 128 * 2 * 2.070e9 / 1e12
    # measured right after the timed region, at the clock the GPU runs at now
    peak32, peak64 = tdbem.measure_fma_peaks()
    clocks = clk.summary()
    fp64_cmp = None
    if fp64_compare and prec == tdbem.PREC_MIXED and not graded:
        y_mixed = asm.hessenberg_apply(X[0]).cpu()
    # end to end through the C ABI: host mesh, grid and right-hand sides in,
    # assembly, matvecs, every result back to host
    del asm
    torch.cuda.empty_cache()
    e2e = None
    if do_e2e:
        Xh = X.cpu().pin_memory()
        Yh = torch.empty((max(matvecs, 1), N, M), dtype=torch.float64).pin_memory()
        Xd = torch.empty_like(X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2, g2 = tdbem.Mesh(V, F), tdbem.TimeGrid(t)
        a2 = tdbem.Assembler(m2, g2, precision=prec, staging_mb=staging_mb)
        Xd.copy_(Xh, non_blocking=True)
        a2.assemble()
        for r in range(matvecs):
            a2.hessenberg_apply(Xd[r], Y)
            Yh[r].copy_(Y, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        del a2
        torch.cuda.empty_cache()
        e2e = {"value": nnz / (t1 - t0), "unit": "nonzeros/s", "seconds": t1 - t0,
               "h2d_bytes_per_step": int(V.nbytes + F.nbytes + t.nbytes + Xh[:matvecs].numel() * 8),
               "d2h_bytes_per_step": int(Yh[:matvecs].numel() * 8)}
    if fp64_compare and prec == tdbem.PREC_MIXED and not graded:
        # the plain FP64 path on the same workload, one timed step (the
        # allocations come from the cache the mixed assembler left)
        a64 = tdbem.Assembler(mesh, grid, precision=tdbem.PREC_FP64)
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        a64.assemble()
        e1.record(stream)
        for r in range(matvecs):
            a64.hessenberg_apply(X[r], Y)
        e2.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        mv64 = e1.elapsed_time(e2) / max(matvecs, 1)
        s64 = a64.stats()
        y64 = a64.hessenberg_apply(X[0]).cpu()
        rel = float(torch.linalg.norm(y_mixed - y64) / torch.linalg.norm(y64))
        fp64_cmp = {"value": s64["nnz"] / ((ms64 + matvecs * mv64) * 1e-3), "unit": "nonzeros/s",
                    "ms_step": ms64 + matvecs * mv64, "ms_assembly": ms64, "ms_matvec_each": mv64,
                    "ms_far": s64["ms_far"], "ms_near": s64["ms_near"],
                    "matvec_rel_diff_mixed_vs_fp64": rel}
        del a64
        torch.cuda.empty_cache()
    cpu = None
    if rank == 0 and world == 1 and do_cpu:
        cpu = cpu_baseline_record(name, V, F, t, nb, cpu_rows)
    return {
        "metric": "assembled nonzeros/s", "value": value, "unit": "nonzeros/s", "n_gpus": world,
        "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64" if prec == tdbem.PREC_MIXED else "f64", "data": "synthetic",
        "config": config_dict(name, precision, world),
        "quad_points_per_s": qps,
        "nnz": nnz, "unique_blocks": nb, "quad_points": st["quad_points"],
        "phase_ms": dict({k: st[k] for k in ("ms_pattern", "ms_far", "ms_near", "ms_extract")},
                         ms_assembly=float(np.mean(asm_ms)), ms_matvec_each=mv_ms, matvecs=matvecs),
        "assembly_only_nnz_per_s": nnz * world / (float(np.mean(asm_ms)) * 1e-3),
        "matvec_nnz_reuse_per_s": mv_work * world / (mv_ms * 1e-3) if matvecs else None,
        "roofline": {"bound": "alu", "achieved": achieved, "peak": peak32, "unit": "TFLOP/s",
                     "frac": achieved / peak32, "traffic": None if graded else FAR_TRAFFIC.get(name),
                     "traffic_unit": "bytes per far phase (all colour launches of one assembly)",
                     "kernel": ("gfar_kernel<false>" if graded else "far32_kernel") + " (FP32 FMA pipe)",
                     "peak_basis": "measured: packed FP32 FMA microbenchmark (tdbem_measure_fma_peaks) "
                                   "after the timed region",
                     "peak_nominal": peak_nominal, "frac_of_nominal": achieved / peak_nominal,
                     "nominal_basis": "%d SMs x 128 FP32 FMA/clk x 2 x 2070 MHz max clock" % sm_count,
                     "fp64_fma_peak_measured": peak64},
        "e2e": e2e, "clocks": clocks, "gpu_launches": launches_per_step * steps,
        "fp64_gpu": fp64_cmp, "cpu_baseline": cpu,
    }


def cpu_baseline_record(name, V, F, t, nb, cpu_rows):
    """The FP64 oracle on the host cores: a bounded row sample of the same
    workload with every core, the same kind of sample on one thread, and on
    the 320-triangle sphere the rows assembled with direct 1-D quadrature of
    psi (no interpolant) for comparison."""
    from oracle.oracle import set_threads
    graded = is_graded(name)
    ca = ({"rows_n": min(cpu_rows, 2), "equidistant": False, "blocks_n": 60} if graded
          else {"rows_n": cpu_rows, "equidistant": True, "blocks_n": None})
    s = cpu_sample(V, F, t, **ca)
    cpu = {"value": s["nnz"] / s["seconds"], "unit": "nonzeros/s", "cores": s["cores"], "kind": "oracle",
           "sample": "%d random rows (seed 0) x %d of %d unique blocks, %.1f s incl. %.1f s psi interpolant "
                     "setup" % (s["rows"], s["blocks"], nb, s["seconds"], s["setup_s"])}
    if not graded:
        # one thread, one row: the rate per core (on the graded grid the
        # per-block interpolant set-up alone takes minutes on one thread)
        prev = set_threads(1)
        try:
            s1 = cpu_sample(V, F, t, **dict(ca, rows_n=1))
            cpu["single_thread"] = {"value": s1["nnz"] / s1["seconds"], "unit": "nonzeros/s", "cores": 1,
                                    "sample": "1 random row (seed 0) x %d unique blocks, %.1f s"
                                              % (s1["blocks"], s1["seconds"])}
        finally:
            set_threads(prev)
    if name == "sphere20480":
        # the 320-triangle configuration: psi by interpolant and by direct
        # 1-D Gauss quadrature at every evaluation, one row, 8 seeded blocks
        V0, F0, t0 = workload("sphere320")
        di = {}
        for mode in ("interp", "direct"):
            d = cpu_sample(V0, F0, t0, rows_n=1, blocks_n=8, psi_mode=mode)
            di[mode] = {"value": d["nnz"] / d["seconds"], "seconds": d["seconds"], "nnz": d["nnz"]}
        cpu["sphere320_psi_modes"] = dict(di, unit="nonzeros/s", cores=s["cores"],
                                          sample="1 random row (seed 0) x 8 seeded of the unique blocks of "
                                                 "sphere320")
    return cpu


def measure_potential(name, steps, warmup, *, local=0, do_cpu=True):
    """Retarded double layer potential (tdbem_double_layer) on a named
    evaluation: value = (point, time) pairs per second, density seeded
    N(0, 1), points, times and density resident on the device; e2e with the
    density, points and times copied from pinned host memory and the
    potential copied back, every step."""
    import torch
    from paper_1503_07221_gb300 import inputs, tdbem

    w = inputs.potential_workload(name)
    asm = tdbem.Assembler(tdbem.Mesh(w.verts, w.tris), tdbem.TimeGrid(w.t))
    stream = torch.cuda.current_stream()
    gen = torch.Generator()
    gen.manual_seed(0)
    alpha_h = torch.randn((w.t.size, w.verts.shape[0]), dtype=torch.float64, generator=gen)
    alpha, X = alpha_h.cuda(), torch.from_numpy(w.X).cuda()
    times = torch.from_numpy(w.times).cuda()
    P, nt = w.X.shape[0], w.times.size
    out = torch.empty((P, nt), dtype=torch.float64, device="cuda")
    for _ in range(warmup):
        asm.double_layer(alpha, X, times, n=w.n, out=out)
    torch.cuda.synchronize()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(steps):
            asm.double_layer(alpha, X, times, n=w.n, out=out)
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / steps
    # end to end: host density, points and times in, potential out
    ah, Xh, th = alpha_h.pin_memory(), torch.from_numpy(w.X).pin_memory(), torch.from_numpy(w.times).pin_memory()
    oh = torch.empty((P, nt), dtype=torch.float64).pin_memory()
    ad, Xd, td = torch.empty_like(alpha), torch.empty_like(X), torch.empty_like(times)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(steps):
        ad.copy_(ah, non_blocking=True)
        Xd.copy_(Xh, non_blocking=True)
        td.copy_(th, non_blocking=True)
        asm.double_layer(ad, Xd, td, n=w.n, out=out)
        oh.copy_(out, non_blocking=True)
        torch.cuda.synchronize()
    e2e_s = (time.perf_counter() - t0) / steps
    quad = w.tris.shape[0] * w.n * w.n
    rec = {"metric": "potential point-times/s", "value": P * nt / (ms * 1e-3), "unit": "point-times/s",
           "steps": steps, "warmup": warmup, "ms_per_step": ms, "higher_is_better": True, "dtype": "f64",
           "data": "synthetic",
           "config": {"workload": name, "points": P, "times": nt, "triangles": int(w.tris.shape[0]),
                      "gauss_points_per_triangle": w.n * w.n, "grid_points": int(w.t.size),
                      "density": "seeded N(0, 1) coefficients"},
           "triples_per_s": P * nt * quad / (ms * 1e-3),
           "e2e": {"value": P * nt / e2e_s, "unit": "point-times/s", "seconds": e2e_s,
                   "h2d_bytes_per_step": int(ah.numel() * 8 + Xh.numel() * 8 + th.numel() * 8),
                   "d2h_bytes_per_step": int(oh.numel() * 8)},
           "clocks": clk.summary(), "gpu_launches": 4 * steps, "cpu_baseline": None}
    if do_cpu:
        from oracle.oracle import Oracle, num_threads
        o = Oracle(w.verts, w.tris, w.t, equidistant=True)
        rng = np.random.default_rng(0)
        pts = np.sort(rng.choice(P, size=32, replace=False))
        c0 = time.perf_counter()
        o.double_layer(alpha_h.numpy(), w.X[pts], w.times, n=w.n)
        sec = time.perf_counter() - c0
        rec["cpu_baseline"] = {"value": pts.size * nt / sec, "unit": "point-times/s", "cores": num_threads(),
                               "kind": "oracle", "sample": "32 random points (seed 0) x %d times, %.1f s" % (nt, sec)}
    del asm
    torch.cuda.empty_cache()
    return rec


def run_ours(args):
    import torch
    from paper_1503_07221_gb300 import build, tdbem

    build.build()
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")
    tdbem.use_torch_allocator()
    line = measure_assembly(args.config, args.precision, args.steps, args.warmup, args.matvecs, world=world,
                            rank=rank, local=local, dist=dist, do_e2e=args.e2e, fp64_compare=args.fp64_compare,
                            do_cpu=not args.no_cpu, cpu_rows=args.cpu_rows, staging_mb=args.staging_mb)
    # sub-records on one GPU: the graded torus (every nonzero block unique;
    # one warm-up, two timed steps: a step takes about a minute) and the
    # retarded potential at the paper's point and time counts
    if world == 1 and args.graded and not is_graded(args.config):
        line["graded"] = measure_assembly("torus8192g", "mixed", 2, 1, args.matvecs, local=local,
                                          fp64_compare=False, do_cpu=not args.no_cpu)
    if world == 1 and args.potential:
        line["potential"] = measure_potential("plane66049_sphere320", 2, 1, local=local, do_cpu=not args.no_cpu)
    if rank == 0:
        print(json.dumps(line))
    if dist:
        dist.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--config", default="sphere20480", choices=sorted(CONFIGS))
    ap.add_argument("--precision", default="mixed", choices=["mixed", "fp64"])
    ap.add_argument("--cpu-rows", type=int, default=16)
    ap.add_argument("--matvecs", type=int, default=20)
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--staging-mb", type=int, default=0,
                    help="non-equidistant grids: cap on the staging windows of one batch (MiB, 0 = default)")
    ap.add_argument("--no-e2e", dest="e2e", action="store_false")
    ap.add_argument("--no-fp64-compare", dest="fp64_compare", action="store_false")
    ap.add_argument("--no-graded", dest="graded", action="store_false",
                    help="skip the graded-torus sub-record")
    ap.add_argument("--no-potential", dest="potential", action="store_false",
                    help="skip the retarded-potential sub-record")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
