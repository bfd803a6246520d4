#!/usr/bin/env python3
"""Benchmark of the pixel-basis Gram-filter reconstruction path on GB300.

Workload: N = 2048 unit-pixel grid, 1800 views uniform in [0, pi), 2900 detector bins at
lambda_y = 1, detector blur zeta = 1, seeded 40-ellipse phantom (4096 x 4096
zero-padded FFT grids).  A step is one Gram apply y = G x on a resident 2048^2 image
(the unit of the headline Gram-apply/s); L2 is flushed (256 MiB write) before every
timed step, outside the timed events.  Alongside: CG iterations/s, one full pass of
the hot path (Gram build + back projection + 100 CG iterations), plain-CG time to a
1e-4 relative residual, the end-to-end rate through the C ABI with host buffers, the
roofline of the dominant kernel and the FP64 CPU oracle timed on the host cores.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
import argparse
import hashlib
import json
import os
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Gram-apply/s and CG iters/s at N=2048; time-to-1e-4 residual, learned vs plain"
UNIT = "Gram-apply/s"
WORKLOAD = "fp32_n2048"
FALLBACK_HBM_GBS = 6800.0


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=50)
    p.add_argument("--warmup", type=int, default=5)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--cg-iters", type=int, default=100)
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--quick", action="store_true", help="skip the hot-path pass, batch and time-to-1e-4 extras")
    p.add_argument("--no-batch", action="store_true")
    p.add_argument("--batch-slices", type=int, default=256)
    p.add_argument("--learned-pairs", type=int, default=10000,
                   help="training pairs for the learned warm start (0 = skip; 10000 = the configured set)")
    p.add_argument("--learned-loss", choices=["gnorm", "mse"], default="gnorm",
                   help="training loss: relative G-norm error (the norm CG minimises) or mean squared error")
    p.add_argument("--workload", default=WORKLOAD, help="named workload of the timed steps (profiling runs use smaller ones)")
    p.add_argument("--learned-epochs", type=int, default=2)
    p.add_argument("--no-tune", action="store_true", help="keep the built-in FFT launch shapes (no autotuner)")
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", "0")), int(os.environ.get("WORLD_SIZE", "1")), int(os.environ.get("LOCAL_RANK", "0"))


def measured_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            pk = json.load(f)
        return float(pk["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM_GBS, "fallback"


def measured_bf16_tflops():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return float(json.load(f)["bf16_tflops"]), "measured"
    except Exception:
        return 1900.0, "fallback"


def kernel_source_hash():
    h = hashlib.sha256()
    for name in ("gram_fft.cu", "bsct_fft.cuh", "bsct_fft2.cuh", "bsct_common.cuh"):
        with open(os.path.join(ROOT, "paper_2005_13471_gb300", "csrc", name), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def profiled_traffic(kernel, n):
    """DRAM bytes per launch of `kernel` from the committed ncu summary, if the kernel source is unchanged."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            rec = json.load(f)
        e = rec[kernel]
        if e.get("source_hash") != kernel_source_hash() or int(e.get("N", -1)) != n:
            return None
        return float(e["dram_bytes_per_launch"])
    except Exception:
        return None


class ClockSampler:
    """nvidia-smi clocks / throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bsct_clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=self.f, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()
            self.f.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = []
        try:
            for line in open(self.path):
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        except Exception:
            pass
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        import statistics

        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower() == "active"})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "reasons": reasons, "samples": len(rows)}


def cpu_oracle_apply_rate(n_applies):
    """The FP64 oracle's FFT Gram apply at N = 2048 on the host (as it stands)."""
    import numpy as np

    from oracle import gram as ogram

    N = 2048
    angles = np.arange(12) / 12  # the apply cost does not depend on the number of views
    G = ogram.gram_taps(N, angles, 1.0)
    x = np.random.default_rng(0).standard_normal((N, N))
    t0 = time.perf_counter()
    for _ in range(n_applies):
        ogram.gram_apply_fft(G, x)
    dt = time.perf_counter() - t0
    return n_applies / dt, dt


# ---------------------------------------------------------------- host-core baselines of the oracle
# Workers of a "spawn" process pool (module level so that they pickle); every one calls
# the oracle as it stands on its own unit of work.
def _w_apply(args):
    import numpy as np

    from oracle import gram as ogram

    seed, reps = args
    N = 2048
    rng = np.random.default_rng(seed)
    G = rng.random((2 * N - 1, 2 * N - 1))  # the apply's cost does not depend on the tap values
    x = rng.standard_normal((N, N))
    t0 = time.perf_counter()
    for _ in range(reps):
        ogram.gram_apply_fft(G, x)
    return time.perf_counter() - t0


def _w_taps(args):
    import numpy as np

    from oracle import gram as ogram

    N, views, zeta = args
    t0 = time.perf_counter()
    G = ogram.gram_taps(N, np.asarray(views), zeta)
    return time.perf_counter() - t0, G


def _w_bp(args):
    import numpy as np

    from oracle import backproject as obp

    N, views, M, pts, seed = args
    sino = np.random.default_rng(seed).standard_normal((len(views), M))
    t0 = time.perf_counter()
    obp.backproject_sampled(sino, N, np.asarray(views), 1.0, 1.0, pts)
    return time.perf_counter() - t0


def cpu_suite(cores):
    """The FP64 oracle on the host cores, per workload of the bench (bounded samples).

    Single-threaded figures call the oracle directly; the multi-core figures run independent
    units (applies, view subsets, pixel samples) in a spawn process pool of `cores` workers
    and divide the work done by the wall time.  Gram build and back projection are sampled
    (a subset of views / pixels) and scaled to the full workload by the work they cover.
    """
    import concurrent.futures as cf
    import multiprocessing as mp

    import numpy as np

    from oracle import cg as ocg
    from oracle import gram as ogram
    from workloads import ellipse_image, ellipse_params, get_config

    out = {"cores": cores}
    # spawn: the pool starts no child from a process that holds a CUDA context; a worker that
    # dies raises BrokenProcessPool instead of leaving the map waiting
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_w_apply, [(k, 1) for k in range(cores)]))  # start-up, imports, first touch: untimed
        # Gram apply at N = 2048: two per worker, all workers at once
        t0 = time.perf_counter()
        list(pool.map(_w_apply, [(100 + k, 2) for k in range(cores)]))
        dt = time.perf_counter() - t0
        out["gram_apply_n2048"] = {"applies_per_s_1core": None, "applies_per_s_all": 2 * cores / dt,
                                   "sample": f"{2 * cores} applies, two per worker ({dt:.1f} s)"}
        # Gram build at N = 2048, 1800 views, zeta = 1: a sample of views per worker
        cfg = get_config("fp32_n2048")
        N, na = cfg["N"], cfg["n_angles"]
        views = np.arange(na) / na
        per = 2
        sample = [(N, views[(k * 97 + np.arange(per)) % na].tolist(), cfg["zeta"]) for k in range(cores)]
        t1 = time.perf_counter()
        res = list(pool.map(_w_taps, sample))
        dt = time.perf_counter() - t1
        t_view = float(np.mean([r[0] for r in res])) / per
        out["gram_build_n2048"] = {"ms_1core": 1e3 * t_view * na, "ms_all": 1e3 * dt * na / (per * cores),
                                   "sample": f"{per * cores} of {na} views ({per} per worker), scaled by views"}
        # back projection at N = 2048, 1800 views: sampled pixels x views per worker
        npx, nv = 250, 24
        rng = np.random.default_rng(0)
        jobs = [(N, views[(k * 53 + np.arange(nv) * 75) % na].tolist(), cfg["n_bins"],
                 [tuple(int(v) for v in p) for p in rng.integers(0, N, size=(npx, 2))], k) for k in range(cores)]
        t2 = time.perf_counter()
        times = list(pool.map(_w_bp, jobs))
        dt = time.perf_counter() - t2
        pairs = npx * nv
        out["backproject_n2048"] = {"pairs_per_s_1core": pairs / float(np.mean(times)),
                                    "pairs_per_s_all": pairs * cores / dt,
                                    "sample": f"{npx} pixels x {nv} views per worker (pixel-view pairs / s)"}
        # time to a 1e-4 relative residual (N = 512, 720 views, zeta = 1): taps over the pool,
        # then the oracle's CG on one core; right-hand side G x of a 40-ellipse phantom (the
        # back projection is measured on its own above)
        c5 = get_config("learned_eval_n512")
        N5, na5 = c5["N"], c5["n_angles"]
        v5 = np.arange(na5) / na5
        chunks = [(N5, v5[k::cores].tolist(), c5["zeta"]) for k in range(cores)]
        t3 = time.perf_counter()
        parts = list(pool.map(_w_taps, chunks))
        t_taps = time.perf_counter() - t3
    G5 = sum(p[1] for p in parts)
    x5 = ellipse_image(ellipse_params(N5, 40, seed=7), N5, supersample=1)
    apply5 = lambda v: ogram.gram_apply_fft(G5, v)
    b5 = apply5(x5)
    t4 = time.perf_counter()
    _, hist, _ = ocg.cg(apply5, b5, iters=2000, tol=1e-4)
    t_cg = time.perf_counter() - t4
    out["time_to_1e-4_n512"] = {"cg_s_1core": t_cg, "cg_iters": len(hist) - 1, "gram_build_s_all": t_taps,
                                "rhs": "G x of a 40-ellipse phantom (FP64 oracle)"}
    # the single-core apply rate (the reference arm's unit)
    rate, dt = cpu_oracle_apply_rate(2)
    out["gram_apply_n2048"]["applies_per_s_1core"] = rate
    return out


def reduce_max(v, device):
    """Maximum of v over the ranks of the default process group (v itself without one)."""
    import torch
    import torch.distributed as dist

    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return v
    t = torch.tensor([v], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(world, steps, step_ms):
    """Units of all ranks per second: each rank ran `steps` units; step_ms is the max over ranks."""
    return world * steps / (step_ms * 1e-3)


def run_reference(args):
    """The oracle as it stands on all host cores: every step runs one FP64 Gram apply at
    N = 2048 on each core at once (independent units in a spawn process pool) and is timed
    by wall clock; value = applies / time."""
    import concurrent.futures as cf
    import multiprocessing as mp

    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    cores = len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity") else (os.cpu_count() or 1)
    with cf.ProcessPoolExecutor(max_workers=cores, mp_context=mp.get_context("spawn")) as pool:
        list(pool.map(_w_apply, [(k, 1) for k in range(cores)]))  # start-up, imports, first touch
        for w in range(args.warmup):
            list(pool.map(_w_apply, [(1000 + 97 * w + k, 1) for k in range(cores)]))
        t0 = time.perf_counter()
        for st in range(args.steps):
            list(pool.map(_w_apply, [(5000 + 97 * st + k, 1) for k in range(cores)]))
        dt = time.perf_counter() - t0
    rate = cores * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": rate, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": f"{WORKLOAD}: N=2048 Gram apply (4096^2 zero-padded FFT convolution)",
                   "N": 2048, "fft_grid": 4096},
        "cpu_baseline": {"value": rate, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} steps of {cores} concurrent applies (one per host core) of the "
                                   "numpy FP64 oracle gram_apply_fft at N=2048 (random taps: the apply's cost does "
                                   "not depend on their values)"},
        "e2e": {"value": rate, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line))
    return 0


def run_ours(args):
    import numpy as np
    import torch

    import paper_2005_13471_gb300 as bsct
    from workloads import get_config, make_problem

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=dev)
    bsct.lib()

    def barrier():
        if world > 1:
            import torch.distributed as dist

            dist.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v):
        return reduce_max(v, dev)

    cfg = get_config(args.workload)
    N = cfg["N"]
    angles, sino_np, _ = make_problem(cfg, slice_id=rank)
    geom = bsct.Geometry(N, angles, cfg["n_bins"], cfg["lambda_y"], cfg["zeta"])
    sino = torch.tensor(sino_np, dtype=torch.float32, device=dev)
    g = bsct.gram_build(geom, bsct.F32)
    b = bsct.backproject(geom, sino, bsct.F32)
    x = b.clone()
    y = torch.empty_like(x)
    flush = torch.empty(256 * 1024 * 1024, dtype=torch.uint8, device=dev)
    stream = torch.cuda.current_stream()

    # ---------------------------------------------------------------- launch shape (autotuner)
    tune = None
    if not args.no_tune:
        # the timed step flushes L2 first, so the shapes are timed on a cold L2 as well
        shape, tune_us, all_us = bsct.fft_autotune(N, bsct.F32, reps=20, flush_bytes=256 << 20)
        tune = {"N": N, "shape": {"rows_fwd": shape[0], "rows_inv": shape[1], "cols_one_per_sm": shape[2]},
                "us_per_apply": tune_us, "candidates_us": [round(t, 2) for t in all_us if t >= 0],
                "how": "bsct_fft_autotune_flushed: 20 applies of every valid launch shape, each after a "
                       "256 MiB write that evicts L2, fastest kept"}

    # ---------------------------------------------------------------- timed steps
    for _ in range(args.warmup):
        flush.zero_()
        g.apply(x, y)
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with ClockSampler(local) as clk:
        # keep the GPU busy for ~1.5 s first so that the clock samples see it under load
        t_load = time.perf_counter()
        while time.perf_counter() - t_load < 1.5:
            for _ in range(50):
                g.apply(x, y)
            torch.cuda.synchronize()
        launches0 = bsct.launch_count()
        wall0 = time.perf_counter()
        for i in range(args.steps):
            flush.zero_()
            ev[i][0].record(stream)
            g.apply(x, y)
            ev[i][1].record(stream)
        barrier()
        wall = time.perf_counter() - wall0
        launches = bsct.launch_count() - launches0
        # per-kernel durations: the same K steps again with CUDA events recorded on the
        # launching stream between the three kernels.  The events serialise the kernels
        # (no launch overlap), so this pass is kept out of the headline loop above.
        bsct.set_kernel_timing(True)
        ktimes = np.zeros(3)
        for i in range(args.steps):
            flush.zero_()
            g.apply(x, y)
            ktimes += np.array(bsct.kernel_times())
        bsct.set_kernel_timing(False)
    step_ms = sum(a.elapsed_time(b_) for a, b_ in ev)
    step_ms = max_over_ranks(step_ms)
    value = whole_job_rate(world, args.steps, step_ms)
    kt = ktimes / args.steps  # ms per launch: row R2C, column conv, row C2R

    # ---------------------------------------------------------------- roofline (dominant kernel)
    hbm, peak_kind = measured_peaks()
    # the FP32 apply's three kernels (paired-FFT forms): algorithmic bytes per launch
    kernel_bytes = {
        "k2_rows_r2c": 4 * N * N + 8 * N * N,
        "k2_cols_conv": 8 * N * N + 8 * N * (N + 1) + 8 * N * N,
        "k2_rows_c2r": 8 * N * N + 4 * N * N,
    }
    names = list(kernel_bytes)
    dom = int(np.argmax(kt))
    dname = names[dom]
    achieved = kernel_bytes[dname] / (kt[dom] * 1e-3) / 1e9
    apply_bytes = 8 * N * N + 40 * N * (N + 1)
    roofline = {"bound": "hbm", "kernel": dname, "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "frac": achieved / hbm, "peak_source": f"{peak_kind} hbm_gbs",
                "algorithmic_bytes_per_launch": kernel_bytes[dname],
                "traffic": profiled_traffic(dname, N),
                "kernel_ms": {n: float(t) for n, t in zip(names, kt)},
                "kernel_timing": "CUDA events between the kernels in a second pass of the K steps, after the "
                                 "headline loop (the events serialise the kernels)",
                "whole_apply": {"algorithmic_bytes": apply_bytes,
                                "achieved_GBs": apply_bytes / (step_ms / args.steps * 1e-3) / 1e9 / world * world,
                                "frac": apply_bytes / (step_ms / args.steps * 1e-3) / 1e9 / hbm}}

    # ---------------------------------------------------------------- CG iterations/s
    n_cg = args.cg_iters
    g.cg_begin(b, x, x0_is_zero=True)
    g.cg_iterate(x, 3)
    flush.zero_()
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    g.cg_iterate(x, n_cg)
    e1.record(stream)
    barrier()
    cg_ms = max_over_ranks(e0.elapsed_time(e1))
    cg_rate = world * n_cg / (cg_ms * 1e-3)
    cg_bytes = apply_bytes + 36 * N * N
    pcg_info = None
    if not args.quick:
        # preconditioned CG: two applies (G, M^-1) and one vector update per iteration
        g.pcg_solve(b, max_iter=3)
        barrier()
        e0.record(stream)
        g.pcg_solve(b, max_iter=n_cg)
        e1.record(stream)
        barrier()
        pcg_ms = max_over_ranks(e0.elapsed_time(e1))
        pcg_info = {"iters": n_cg, "ms_per_iter": pcg_ms / n_cg, "eps": bsct.PRECOND_EPS,
                    "timed": "one bsct_pcg_solve call from x = 0 (its start-up M^-1 apply included)"}

    # ---------------------------------------------------------------- forward projection S H c
    fwork = torch.empty(bsct.forward_project_workspace(geom, bsct.F32), dtype=torch.uint8, device=dev)
    sino_f = torch.empty_like(sino)
    bsct.forward_project(geom, x, bsct.F32, out=sino_f, work=fwork)
    barrier()
    e0.record(stream)
    bsct.forward_project(geom, x, bsct.F32, out=sino_f, work=fwork)
    e1.record(stream)
    barrier()
    fp_ms = max_over_ranks(e0.elapsed_time(e1))
    forward_info = {"ms": fp_ms, "Gpairs_per_s": N * N * cfg["n_angles"] / (fp_ms * 1e-3) / 1e9,
                    "pairs": "pixel-view pairs N^2 x views, as for the back projection",
                    "launches": 3, "includes": "per-view tables, image transpose, gather"}

    # ---------------------------------------------------------------- end to end (host buffers)
    # bsct_gram_apply_host: K images in pinned host memory; every step copies its image in,
    # applies G and copies the result out, the copies overlapped with the neighbouring
    # steps' applies on the library's three streams
    K = args.steps
    xh = torch.empty((K, N, N), dtype=torch.float32, pin_memory=True)
    xh.copy_(x.cpu().unsqueeze(0).expand(K, N, N))
    yh = torch.empty((K, N, N), dtype=torch.float32, pin_memory=True)
    # untimed warm-up over the same buffers: creates the pipeline's streams and device images
    # and has every pinned page written once by the copy engines before the timed pass (one
    # run that skipped this saw the overlapped pass take 7x its usual time)
    g.apply_host(xh, yh)
    torch.cuda.synchronize()
    barrier()
    e0.record(stream)
    g.apply_host(xh, yh)
    e1.record(stream)
    barrier()
    e2e_ms = max_over_ranks(e0.elapsed_time(e1))
    e2e_exact = bool(torch.equal(yh[K - 1], g.apply(x).cpu()))
    e2e = {"value": world * K / (e2e_ms * 1e-3), "unit": UNIT, "h2d_bytes_per_step": 4 * N * N,
           "d2h_bytes_per_step": 4 * N * N, "api": "bsct_gram_apply_host (pinned host buffers)",
           "result_equals_device_apply": e2e_exact}
    # the same steps one after another on one stream (no overlap), for comparison
    xd = torch.empty_like(x)
    barrier()
    e0.record(stream)
    for k in range(K):
        xd.copy_(xh[k], non_blocking=True)
        g.apply(xd, y)
        yh[k].copy_(y, non_blocking=True)
    e1.record(stream)
    barrier()
    e2e["serial_value"] = world * K / (max_over_ranks(e0.elapsed_time(e1)) * 1e-3)

    # ---------------------------------------------------------------- whole hot path, time to 1e-4
    extras = {}
    if not args.quick:
        barrier()
        t = {}
        e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        e[0].record(stream)
        g2 = bsct.gram_build(geom, bsct.F32)
        e[1].record(stream)
        b2 = bsct.backproject(geom, sino, bsct.F32)
        e[2].record(stream)
        x2, _ = g2.cg_solve(b2, max_iter=100)
        e[3].record(stream)
        barrier()
        t = {"gram_build_ms": e[0].elapsed_time(e[1]), "backproject_ms": e[1].elapsed_time(e[2]),
             "cg100_ms": e[2].elapsed_time(e[3])}
        t["total_ms"] = sum(t.values())
        t["backproject_Gpairs_per_s"] = N * N * cfg["n_angles"] / (t["backproject_ms"] * 1e-3) / 1e9
        # ALU-bound steps against the measured FMA throughput of this GPU
        fp32 = bsct.fma_peak(bsct.F32)
        fp64 = bsct.fma_peak(bsct.F64)
        t["fma_peak_tflops"] = {"fp32": fp32 / 1e12, "fp64": fp64 / 1e12,
                                "how": "bsct_fma_peak: 8 independent FMA chains per thread, best of 3"}
        t["backproject_fp32_frac"] = N * N * cfg["n_angles"] * 70.0 / (t["backproject_ms"] * 1e-3) / fp32
        t["backproject_flop_per_pair"] = "70, algorithmic: <= 7 bins x degree-5 Horner per pixel-view pair"
        # the filter build against the FP64 pipe: 3.8e7 strip evaluations of the Gram kernel
        # at N = 2048 / 1800 views (each a degree-5 polynomial piece, ~10 FP64 FMA)
        if N == 2048 and cfg["n_angles"] == 1800:
            t["gram_build_fp64_frac"] = 3.8e7 * 20.0 / (t["gram_build_ms"] * 1e-3) / fp64
            t["gram_build_flop"] = "3.8e7 strip evaluations x 20 FP64 flop (whole build, spectrum included)"
        extras["hot_path_pass"] = t
        g2.close()
        # detector kernel of two boxes (widths 1.0 and 0.5) on the 512 x 512 / 720-view
        # geometry: filter build, back projection and forward projection, FP32, each timed
        # once after one untimed call
        cm = get_config("learned_eval_n512")
        am = np.arange(cm["n_angles"], dtype=np.float64) / cm["n_angles"]
        mb = {"workload": f"N={cm['N']}, {cm['n_angles']} views, {cm['n_bins']} bins, lambda_y={cm['lambda_y']}, "
                          "detector boxes of widths 1.0 and 0.5"}
        for widths, key in (((1.0, 0.5), "two_boxes"), (1.5, "one_box_1.5")):
            gm = bsct.Geometry(cm["N"], am, cm["n_bins"], cm["lambda_y"], widths)
            xm = torch.rand((cm["N"], cm["N"]), device=dev)
            sm = bsct.forward_project(gm, xm, bsct.F32)
            bsct.backproject(gm, sm, bsct.F32)
            bsct.gram_build(gm, bsct.F32).close()
            em = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            em[0].record(stream)
            gg = bsct.gram_build(gm, bsct.F32)
            em[1].record(stream)
            bsct.backproject(gm, sm, bsct.F32)
            em[2].record(stream)
            bsct.forward_project(gm, xm, bsct.F32)
            em[3].record(stream)
            torch.cuda.synchronize()
            gg.close()
            mb[key] = {"gram_build_ms": em[0].elapsed_time(em[1]), "backproject_ms": em[1].elapsed_time(em[2]),
                       "forward_project_ms": em[2].elapsed_time(em[3])}
        extras["multibox"] = mb
        # time to a 1e-4 relative residual on the learned-evaluation geometry: 20 held-out
        # seeds (phantoms generated on the device), medians and iteration counts
        from workloads.phantom import ellipse_params, ellipse_sinogram_torch, poisson_log_sinogram_torch

        c5 = get_config("learned_eval_n512")
        N5, na5 = c5["N"], c5["n_angles"]
        a5 = np.arange(na5, dtype=np.float64) / na5
        geom5 = bsct.Geometry(N5, a5, c5["n_bins"], c5["lambda_y"], c5["zeta"])
        g5 = bsct.gram_build(geom5, bsct.F32)
        gen5 = torch.Generator(device=dev).manual_seed(12345 + rank)
        b5s = []
        for k in range(20):
            pk = ellipse_params(N5, c5["n_ellipses"], c5.get("seed", 0), slice_id=1000 + 20 * rank + k)
            sk = ellipse_sinogram_torch(pk, a5, c5["n_bins"], c5["lambda_y"], c5["zeta"], device=dev,
                                        dtype=torch.float64)
            sk = poisson_log_sinogram_torch(sk, c5["I0"], gen5).float().contiguous()
            b5s.append(bsct.backproject(geom5, sk, bsct.F32))
        g5.cg_solve(b5s[0], max_iter=20)

        def timed(fn):
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            out = fn()
            torch.cuda.synchronize()
            return 1e3 * (time.perf_counter() - t0), out

        barrier()
        plain = [timed(lambda: g5.cg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=5)) for b in b5s]
        tt = {"workload": "N=512, 720 views, 726 bins, zeta=1, Poisson I0=1e5; 20 held-out phantom seeds",
              "plain_ms_median": float(np.median([t for t, _ in plain])),
              "plain_iters": [r["iterations"] for _, (_, r) in plain],
              "plain_true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in plain),
              "learned_ms_median": None}
        # preconditioned CG with the circulant preconditioner (the non-learned comparator)
        g5.pcg_solve(b5s[0], max_iter=5)
        pcg = [timed(lambda: g5.pcg_solve(b, max_iter=2000, rel_tol=1e-4, check_every=2)) for b in b5s]
        tt["pcg_circulant"] = {
            "eps": bsct.PRECOND_EPS, "ms_median": float(np.median([t for t, _ in pcg])),
            "iters": [r["iterations"] for _, (_, r) in pcg],
            "true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in pcg),
            "speedup_vs_plain": tt["plain_ms_median"] / float(np.median([t for t, _ in pcg]))}
        # the same two solvers as one CUDA graph each (device-side stopping test): one
        # launch and one synchronisation per solve; the output buffer is reused so the
        # executable graph is built once
        xg = torch.empty_like(b5s[0])
        for method, key in (("cg", "plain_graph"), ("pcg", "pcg_graph")):
            g5.solve_graph(b5s[0], method=method, max_iter=2000, rel_tol=1e-4, out=xg)
            runs = [timed(lambda: g5.solve_graph(b, method=method, max_iter=2000, rel_tol=1e-4, out=xg))
                    for b in b5s]
            tt[key] = {"ms_median": float(np.median([t for t, _ in runs])),
                       "iters": [r["iterations"] for _, (_, r) in runs],
                       "true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in runs)}
        if args.learned_pairs > 0:
            from paper_2005_13471_gb300 import learned

            t_tr = time.perf_counter()
            Xl, Yl = learned.generate_pairs(args.learned_pairs, N=256, n_angles=360, n_bins=364, zeta=1.0, I0=1e5,
                                            cg_iters=200, chunk=256, seed=rank)
            t_gen = time.perf_counter() - t_tr
            net = bsct.UNet(32, seed=rank)
            g_tr, w_tr = None, None
            if args.learned_loss == "gnorm":
                g_tr = bsct.gram_build(bsct.Geometry.uniform(256, 360, 364, 1.0, 1.0), bsct.F32)
                w_tr = learned.gnorm_weights(g_tr, Yl)
            losses = learned.train(net, Xl, Yl, epochs=args.learned_epochs, batch_size=8, lr=1e-3, lr_final=5e-5,
                                   log_every=25, loss=args.learned_loss, gram=g_tr, weights=w_tr)
            t_train = time.perf_counter() - t_tr - t_gen
            if g_tr is not None:
                g_tr.close()
            del Xl, Yl
            # network inference alone (the warm start's fixed cost per solve)
            xin = (b5s[0] / na5).unsqueeze(0).contiguous()
            net.forward(xin)
            torch.cuda.synchronize()
            e0.record(stream)
            for _ in range(5):
                net.forward(xin)
            e1.record(stream)
            torch.cuda.synchronize()
            infer_ms = e0.elapsed_time(e1) / 5
            g5.cg_solve_learned(net, b5s[0], 1.0 / na5, max_iter=5, rel_tol=0.0)
            warm = [timed(lambda: g5.cg_solve_learned(net, b, 1.0 / na5, max_iter=2000, rel_tol=1e-4,
                                                      check_every=5)) for b in b5s]
            fcg = [timed(lambda: g5.fcg_solve_learned(net, b, 1.0 / na5, max_iter=2000, rel_tol=1e-4,
                                                      precond_every=4)) for b in b5s[:5]]
            wpcg = [timed(lambda: g5.pcg_solve_learned(net, b, 1.0 / na5, max_iter=2000, rel_tol=1e-4))
                    for b in b5s]
            tt.update({
                "learned_ms_median": float(np.median([t for t, _ in warm])),
                "learned_iters": [r["iterations"] for _, (_, r) in warm],
                "learned_true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in warm),
                "warm_start_alpha": [r["alpha"] for _, (_, r) in warm][:5],
                "learned_pcg": {"ms_median": float(np.median([t for t, _ in wpcg])),
                                "iters": [r["iterations"] for _, (_, r) in wpcg],
                                "true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in wpcg),
                                "note": "warm start, then circulant-preconditioned CG (against pcg_circulant)"},
                "fcg_precond_every_4": {
                    "seeds": 5, "ms_median": float(np.median([t for t, _ in fcg])),
                    "iters": [r["iterations"] for _, (_, r) in fcg],
                    "network_applications": [r["n_precond"] for _, (_, r) in fcg],
                    "fallbacks": [r["n_fallback"] for _, (_, r) in fcg],
                    "true_rel_residual_max": max(r["true_rel_residual"] for _, (_, r) in fcg)},
                "inference_ms_n512": infer_ms,
                "training": {"pairs": args.learned_pairs, "geometry": "N=256, 360 views, 364 bins, zeta=1",
                             "target": "200-iteration CG", "epochs": args.learned_epochs, "loss": args.learned_loss,
                             "generate_s": t_gen, "train_s": t_train,
                             "loss_first_last": [losses[0], losses[-1]] if losses else None}})
            net.close()
        extras["time_to_1e-4"] = tt
        g5.close()

    # ---------------------------------------------------------------- accuracy study (Sec. 6, box-spline curves)
    if not args.quick:
        from paper_2005_13471_gb300 import study

        t_st = time.perf_counter()
        rows = study.accuracy_sweep(bsct, N=256, n_views=180, zeta=1.0, lambdas=(0.25, 0.5, 1.0, 1.5, 2.0),
                                    noise=(0.0, 0.01, 0.05), solver="sd", iters=100, n_ellipses=30, seed=rank)
        extras["accuracy_study"] = {
            "workload": "N=256, 180 views, zeta=1, 30-ellipse phantom, exact blurred sinogram, Gaussian noise "
                        "sigma relative to the largest sample, 100 steepest-descent steps",
            "rows": [{k: (round(v, 4) if isinstance(v, float) else v) for k, v in r.items()} for r in rows],
            "wall_s": time.perf_counter() - t_st}

    # ---------------------------------------------------------------- split-BF16 DFT-GEMM apply (tensor cores)
    if not args.quick:
        yd = torch.empty_like(y)
        g.apply(x, yd, mode=bsct.APPLY_DFTGEMM_BF16)  # allocates the DFT-GEMM scratch
        g.apply(x, y)
        torch.cuda.synchronize()
        nd = 5
        e0.record(stream)
        for _ in range(nd):
            g.apply(x, yd, mode=bsct.APPLY_DFTGEMM_BF16)
        e1.record(stream)
        torch.cuda.synchronize()
        dms = e0.elapsed_time(e1) / nd
        L = 2 * N
        P = 64 if L % 64 == 0 else 32
        Q = L // P
        gemm_flop = 4 * (2 * (2 * P) * (6 * P) * (Q * L) + 2 * (2 * Q) * (6 * Q) * (P * L))
        extras["dftgemm_bf16"] = {
            "ms_per_apply": dms, "applies_per_s": 1e3 / dms,
            "rel_l2_diff_vs_fp32_fft": float((yd - y).double().norm() / y.double().norm()),
            "gemm_flop_per_apply": gemm_flop, "gemm_tflops_effective": gemm_flop / (dms * 1e-3) / 1e12,
            "frac_of_bf16_peak": gemm_flop / (dms * 1e-3) / 1e12 / measured_bf16_tflops()[0],
            "bf16_peak_source": measured_bf16_tflops()[1] + " bf16_tflops (burst)",
            "note": "4 DFTs of 4096^2 as 8 split-BF16 GEMMs (tcgen05 kind::f16, FP32 accumulate in tensor memory) + split/twiddle kernels"}

    # ---------------------------------------------------------------- batched slices (one graph launch)
    if not args.quick and not args.no_batch:
        from workloads import configs as wcfg
        from workloads.phantom import ellipse_params, ellipse_sinogram_torch

        sl = wcfg.batch_slices(args.batch_slices, seed=rank)
        if not args.no_tune:
            for n_b in sorted({d["N"] for d in sl}):
                bsct.fft_autotune(n_b, bsct.F32, reps=10)
        geoms, sinos, cache = [], [], {}
        for i, d in enumerate(sl):
            key = (d["N"], d["n_angles"], d["zeta"])
            ang = np.arange(d["n_angles"]) / d["n_angles"]
            if key not in cache:
                cache[key] = ellipse_sinogram_torch(ellipse_params(d["N"], d["n_ellipses"], seed=len(cache)), ang,
                                                    d["n_bins"], 1.0, d["zeta"], device=dev, dtype=torch.float32)
            geoms.append(bsct.Geometry(d["N"], ang, d["n_bins"], 1.0, d["zeta"]))
            sinos.append(cache[key] * (1.0 + 0.01 * i))
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        batch = bsct.Batch(geoms)
        t_create = time.perf_counter() - t0
        xs = batch.solve(sinos, cg_iters=wcfg.BATCH_CG_ITERS)  # records the graph
        torch.cuda.synchronize()
        nrep = 3
        l0 = bsct.launch_count()
        e0.record(stream)
        for _ in range(nrep):
            batch.solve(sinos, xs=xs, cg_iters=wcfg.BATCH_CG_ITERS)
        e1.record(stream)
        torch.cuda.synchronize()
        bms = e0.elapsed_time(e1) / nrep
        launches_per_batch = (bsct.launch_count() - l0) / nrep
        info = batch.info()
        # time split: the same batch without CG iterations (prefilter, back projection and
        # CG start of every slice); the rest of the batch is the CG iterations
        batch.solve(sinos, xs=xs, cg_iters=0)  # records the shorter graph
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(nrep):
            batch.solve(sinos, xs=xs, cg_iters=0)
        e1.record(stream)
        torch.cuda.synchronize()
        bms0 = e0.elapsed_time(e1) / nrep
        extras["batched"] = {
            "workload": f"{len(sl)} slices, N in {wcfg.BATCH_SIZES_N}, views in {wcfg.BATCH_ANGLES}, "
                        f"bins=ceil(1.42N), zeta in {{0,1}}, {wcfg.BATCH_CG_ITERS} CG iterations each",
            "ms_per_batch": bms, "slices_per_s": len(sl) / (bms * 1e-3),
            "cg_iters_per_s_aggregate": len(sl) * wcfg.BATCH_CG_ITERS / (bms * 1e-3),
            "geometries": info["geometries"], "graph_nodes": info["graph_nodes"],
            "kernels_per_launch": info["kernels_per_launch"], "create_s": t_create,
            "launches_counted": launches_per_batch,
            "split_ms": {"backprojection_and_cg_start": bms0, "cg_iterations": bms - bms0}}
        batch.close()
        del sinos, xs

    # ---------------------------------------------------------------- host link (pinned copies)
    # one cudaMemcpyAsync per copy of one N x N FP32 image, host-to-device and device-to-host
    # at the same time on two streams: the peak the end-to-end rate is divided by
    nb = 4 * N * N
    hsrc = torch.empty(N * N, dtype=torch.float32, pin_memory=True)
    hdst = torch.empty(N * N, dtype=torch.float32, pin_memory=True)
    dsrc = torch.empty(N * N, dtype=torch.float32, device=dev)
    ddst = torch.empty(N * N, dtype=torch.float32, device=dev)
    s_h2d, s_d2h = torch.cuda.Stream(), torch.cuda.Stream()
    reps = 20
    for _ in range(3):
        ddst.copy_(hsrc, non_blocking=True)
        hdst.copy_(dsrc, non_blocking=True)
    torch.cuda.synchronize()
    link = {}
    for name, pairs in (("h2d", [(s_h2d, ddst, hsrc)]), ("d2h", [(s_d2h, hdst, dsrc)]),
                        ("both", [(s_h2d, ddst, hsrc), (s_d2h, hdst, dsrc)])):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for _ in range(reps):
            for st_, dst, src in pairs:
                with torch.cuda.stream(st_):
                    dst.copy_(src, non_blocking=True)
        torch.cuda.synchronize()
        link[name] = reps * nb / (time.perf_counter() - t0) / 1e9  # GB/s per direction
    e2e_link_gbs = e2e["value"] * nb / 1e9  # per direction
    e2e["host_link"] = {"h2d_GBs": link["h2d"], "d2h_GBs": link["d2h"], "both_per_direction_GBs": link["both"],
                        "e2e_GBs_per_direction": e2e_link_gbs, "frac": e2e_link_gbs / link["both"],
                        "how": f"pinned {nb >> 20} MiB image, one cudaMemcpyAsync per copy, {reps} copies per "
                               "direction, both directions on two streams for the concurrent figure"}
    del hsrc, hdst, dsrc, ddst

    # ---------------------------------------------------------------- FP64 apply (context)
    fp64_info = None
    if not args.quick:
        g64 = bsct.gram_build(geom, bsct.F64)
        x64 = x.double()
        y64 = torch.empty_like(x64)
        for _ in range(3):
            g64.apply(x64, y64)
        barrier()
        e0.record(stream)
        for _ in range(10):
            g64.apply(x64, y64)
        e1.record(stream)
        barrier()
        ms64 = e0.elapsed_time(e1) / 10
        fp64_info = {"ms_per_apply": ms64, "applies_per_s": 1e3 / ms64,
                     "algorithmic_bytes": 2 * apply_bytes,
                     "frac_of_hbm": 2 * apply_bytes / (ms64 * 1e-3) / 1e9 / hbm,
                     "rel_l2_vs_fp32": float((y64 - g.apply(x).double()).norm() / y64.norm()),
                     "l2": "not flushed between applies"}
        g64.close()
        del x64, y64

    # ---------------------------------------------------------------- CPU baseline (rank 0, N=1)
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cores = os.cpu_count() or 1
        suite = cpu_suite(cores)
        ga = suite["gram_apply_n2048"]
        cpu = {"value": ga["applies_per_s_all"], "unit": UNIT, "cores": cores, "kind": "oracle",
               "sample": f"FP64 oracle gram_apply_fft at N=2048 on {cores} host cores: {ga['sample']}",
               "single_core_value": ga["applies_per_s_1core"],
               "per_workload": suite}

    clocks = clk.summary()
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": step_ms / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": f"{args.workload}: N={N}, {cfg['n_angles']} views, {cfg['n_bins']} bins, "
                               f"lambda_y={cfg['lambda_y']:g}, zeta={cfg['zeta']:g}, 40-ellipse phantom",
                   "fft_grid": 2 * N, "l2": "flushed (256 MiB write) before every timed step, outside the events",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "cg_iters_per_s": cg_rate,
        "cg": {"iters": n_cg, "ms_per_iter": cg_ms / n_cg, "algorithmic_bytes_per_iter": cg_bytes,
               "frac_of_hbm": cg_bytes / (cg_ms / n_cg * 1e-3) / 1e9 / hbm,
               "l2": "not flushed between iterations (135 MB working set)"},
        "pcg": pcg_info,
        "fp64_apply": fp64_info,
        "autotune": tune,
        "forward_project": forward_info,
        "roofline": roofline,
        "e2e": e2e,
        "gpu_launches": int(launches),
        "wall_s_timed_loop": wall,
        "clocks": clocks,
        "cpu_baseline": cpu,
    }
    line.update(extras)
    if rank == 0:
        print(json.dumps(line))
    g.close()
    if world > 1:
        import torch.distributed as dist

        dist.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
