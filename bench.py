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


def cpu_sample(V, F, t, rows_n, seed=0, equidistant=True, blocks_n=None):
    """Time the FP64 oracle on a fixed row sample (all unique blocks, or a
    seeded sample of blocks_n of them)."""
    from oracle.oracle import Oracle, num_threads
    rng = np.random.default_rng(seed)
    rows = np.sort(rng.choice(V.shape[0], size=rows_n, replace=False))
    t0 = time.perf_counter()
    o = Oracle(V, F, t, equidistant=equidistant, psi_mode="interp")
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


def run_reference(args):
    V, F, t = workload(args.config)
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    ca = cpu_sample_args(args)
    rows_n = ca["rows_n"]
    rates, secs = [], []
    for _ in range(args.steps):
        s = cpu_sample(V, F, t, **ca)
        rates.append(s["nnz"] / s["seconds"])
        secs.append(s["seconds"])
    v = float(np.median(rates))
    line = {
        "impl": "reference", "metric": "assembled nonzeros/s", "value": v, "unit": "nonzeros/s",
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": float(np.median(secs)) * 1e3, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": args.config, "desc": CONFIGS[args.config], "precision": "fp64 oracle",
                   "sample": "%d random rows (seed 0) x %d unique blocks" % (rows_n, s["blocks"])},
        "cpu_baseline": {"value": v, "unit": "nonzeros/s", "cores": s["cores"], "kind": "oracle",
                         "sample": "%d rows x %d unique blocks of %s" % (rows_n, s["blocks"], args.config)},
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
    V, F, t = workload(args.config)
    graded = is_graded(args.config)
    prec = tdbem.PREC_MIXED if args.precision == "mixed" else tdbem.PREC_FP64
    mesh, grid = tdbem.Mesh(V, F), tdbem.TimeGrid(t)
    asm = tdbem.Assembler(mesh, grid, precision=prec, staging_mb=args.staging_mb)
    stream = torch.cuda.current_stream()
    N, M = t.size, V.shape[0]
    # matvec inputs: x_r ~ N(0, 1) from a CPU generator with seed r, copied once
    X = torch.empty((max(args.matvecs, 1), N, M), dtype=torch.float64, device="cuda")
    for r in range(X.shape[0]):
        gen = torch.Generator()
        gen.manual_seed(r)
        X[r].copy_(torch.randn((N, M), dtype=torch.float64, generator=gen))
    Y = torch.empty((N, M), dtype=torch.float64, device="cuda")

    def step(mv_events=None):
        asm.assemble()
        if mv_events:
            mv_events[0].record(stream)
        for r in range(args.matvecs):
            asm.hessenberg_apply(X[r], Y)
        if mv_events:
            mv_events[1].record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    ev0, ev1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    far_ms, asm_ms, mv_ev = [], [], []
    with ClockSampler(local) as clk:
        torch.cuda.synchronize()
        ev0.record(stream)
        for _ in range(args.steps):
            e = (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
            step(e)
            mv_ev.append(e)
            far_ms.append(asm.stats()["ms_far"])
            asm_ms.append(asm.stats()["ms_total"])
        ev1.record(stream)
        torch.cuda.synchronize()
    ms = ev0.elapsed_time(ev1) / args.steps
    mv_ms = float(np.mean([a.elapsed_time(b) for a, b in mv_ev])) / max(args.matvecs, 1)
    if dist:
        ms = max_over_ranks(ms, dist, "cuda")
    st = asm.stats()
    nnz = st["nnz"]
    value = job_throughput(nnz, world, ms)
    qps = job_throughput(st["quad_points"], world, ms)
    nb = st["n_blocks"]
    launches_per_step = st["kernel_launches"] + 2 * args.matvecs  # transpose + product per matvec
    # matvec work: every stored entry times the number of block positions that reuse its block
    mv_work = 0
    for b in range(asm.num_blocks()):
        bi = asm.block_info(b)
        k, i = bi["k"], bi["i"]
        reuse = (N - 1 - k) if (i == 1 and 1 <= k <= N - 2) else ((N - 3) if (k == 1 and i == 2) else 1)
        if graded:
            reuse = 1
        mv_work += (bi["nnz_far"] + bi["nnz_near"]) * reuse
    # end to end through the C ABI: host mesh, grid and right-hand sides in,
    # assembly, matvecs, every result back to host
    e2e = None
    if graded and args.e2e:
        # the graded workload holds ~80 GB of CSR: free it before the second assembler
        del asm
        torch.cuda.empty_cache()
    if args.e2e:
        Xh = X.cpu().pin_memory()
        Yh = torch.empty((max(args.matvecs, 1), N, M), dtype=torch.float64).pin_memory()
        Xd = torch.empty_like(X)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        m2, g2 = tdbem.Mesh(V, F), tdbem.TimeGrid(t)
        a2 = tdbem.Assembler(m2, g2, precision=prec)
        Xd.copy_(Xh, non_blocking=True)
        a2.assemble()
        for r in range(args.matvecs):
            a2.hessenberg_apply(Xd[r], Y)
            Yh[r].copy_(Y, non_blocking=True)
        torch.cuda.synchronize()
        t1 = time.perf_counter()
        del a2
        e2e = {"value": nnz / (t1 - t0), "unit": "nonzeros/s", "seconds": t1 - t0,
               "h2d_bytes_per_step": int(V.nbytes + F.nbytes + t.nbytes + Xh[:args.matvecs].numel() * 8),
               "d2h_bytes_per_step": int(Yh[:args.matvecs].numel() * 8)}
    # roofline of the dominant kernel (far field): FP32 FMA pipe
    far_avg_ms = float(np.mean(far_ms))
    flops = gfar_flops(st) if graded else far_flops(st)
    achieved = flops / (far_avg_ms * 1e-3) / 1e12
    sm_count = torch.cuda.get_device_properties(local).multi_processor_count
    peak_nominal = sm_count * 128 * 2 * 2.070e9 / 1e12
    # measured right after the timed region, at the clock the GPU runs at now
    peak32, peak64 = tdbem.measure_fma_peaks()
    peak = peak32
    clocks = clk.summary()
    fp64_cmp = None
    if args.fp64_compare and prec == tdbem.PREC_MIXED and not graded:
        y_mixed = asm.hessenberg_apply(X[0]).cpu()
        del asm
        torch.cuda.empty_cache()
        a64 = tdbem.Assembler(mesh, grid, precision=tdbem.PREC_FP64)
        a64.assemble()
        a64.hessenberg_apply(X[0], Y)  # first product tunes the launch shape, untimed
        torch.cuda.synchronize()
        e0, e1, e2 = (torch.cuda.Event(enable_timing=True) for _ in range(3))
        e0.record(stream)
        a64.assemble()
        e1.record(stream)
        for r in range(args.matvecs):
            a64.hessenberg_apply(X[r], Y)
        e2.record(stream)
        torch.cuda.synchronize()
        ms64 = e0.elapsed_time(e1)
        mv64 = e1.elapsed_time(e2) / max(args.matvecs, 1)
        s64 = a64.stats()
        y64 = a64.hessenberg_apply(X[0]).cpu()
        rel = float(torch.linalg.norm(y_mixed - y64) / torch.linalg.norm(y64))
        fp64_cmp = {"value": s64["nnz"] / ((ms64 + args.matvecs * mv64) * 1e-3), "unit": "nonzeros/s",
                    "ms_step": ms64 + args.matvecs * mv64, "ms_assembly": ms64, "ms_matvec_each": mv64,
                    "ms_far": s64["ms_far"], "ms_near": s64["ms_near"],
                    "matvec_rel_diff_mixed_vs_fp64": rel}
        del a64
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        s = cpu_sample(V, F, t, **cpu_sample_args(args))
        cpu = {"value": s["nnz"] / s["seconds"], "unit": "nonzeros/s", "cores": s["cores"], "kind": "oracle",
               "sample": "%d random rows (seed 0) x %d of %d unique blocks, %.1f s incl. %.1f s psi interpolant "
                         "setup" % (s["rows"], s["blocks"], nb, s["seconds"], s["setup_s"])}
    if rank == 0:
        line = {
            "metric": "assembled nonzeros/s", "value": value, "unit": "nonzeros/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if prec == tdbem.PREC_MIXED else "f64", "data": "synthetic",
            "config": {"workload": args.config, "desc": CONFIGS[args.config], "precision": args.precision,
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "l2": "working set (element-pair records, lag windows, CSR) far larger than L2"},
            "quad_points_per_s": qps,
            "nnz": nnz, "unique_blocks": nb, "quad_points": st["quad_points"],
            "phase_ms": dict({k: st[k] for k in ("ms_pattern", "ms_far", "ms_near", "ms_extract")},
                             ms_assembly=float(np.mean(asm_ms)), ms_matvec_each=mv_ms, matvecs=args.matvecs),
            "assembly_only_nnz_per_s": nnz * world / (float(np.mean(asm_ms)) * 1e-3),
            "matvec_nnz_reuse_per_s": mv_work * world / (mv_ms * 1e-3) if args.matvecs else None,
            "roofline": {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": ("gfar_kernel<false>" if graded else "far32_kernel") + " (FP32 FMA pipe)",
                         "peak_basis": "measured: packed FP32 FMA microbenchmark (tdbem_measure_fma_peaks) "
                                       "after the timed region",
                         "peak_nominal": peak_nominal, "frac_of_nominal": achieved / peak_nominal,
                         "nominal_basis": "%d SMs x 128 FP32 FMA/clk x 2 x 2070 MHz max clock" % sm_count,
                         "fp64_fma_peak_measured": peak64},
            "e2e": e2e, "clocks": clocks, "gpu_launches": launches_per_step * args.steps,
            "fp64_gpu": fp64_cmp, "cpu_baseline": cpu,
        }
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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
