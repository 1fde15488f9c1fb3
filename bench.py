#!/usr/bin/env python3
"""Benchmark of the regional adaptive PSS-MLT chain step on one or more GB300s.

Workload (default): the two-rooms / 5 cm door-gap scene, 200k triangles
(seeded tessellated spheres and tori, 50 % Lambert, 50 % GGX), 512 x 512
image, 16-px regions (1024 regions), path depth <= 10 with next-event
estimation (D = 52), 2^16 chains, large-step probability 0.3, Kelemen small
steps s1 = 1/1024, s2 = 1/64, host-built SAH BVH, binary32 tracing.

One step = rmlt_step(1024): 1024 mutations of every chain (64 epochs of 16,
each epoch = one chain-kernel launch + one region-update launch).  The
metric is mutations/s (and rays/s) of the whole job; the image is the
regional adaptive estimate (plain target) and the L2 is flushed between
timed steps by writing a 256 MiB buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
from ctypes import byref, c_double as C_double, c_void_p as C_void_p
import math
import os
import statistics
import subprocess
import sys
import threading
import time
from pathlib import Path

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# FP32 operations the traversal needs per BVH4 node visit (four child boxes:
# 6 FMA + 6 min + 6 max per slab test, one compare each, and a 5-comparator
# sort) and per ray-triangle test (Moller-Trumbore: two cross products, three
# dot products, sign scaling, 5 compares, one division for a hit); an FMA
# counts as 2 floating-point operations.
FLOPS_PER_NODE = 4 * (6 * 2 + 12 + 1) + 5 * 2   # 110
FLOPS_PER_TRI = 2 * (6 * 2) + 3 * 5 + 3 + 5 + 1  # 48
BYTES_PER_NODE = 128   # BVH4 node: six float4 of child bounds, one of child refs, one unused
BYTES_PER_TRI = 48
SM_COUNT = 152
FP32_LANES = 128

WORKLOADS = {
    "two_rooms": dict(desc="two rooms joined by a 5 cm door gap, 200k triangles, 512x512, 16-px "
                           "regions, depth 10, 2^16 chains x 1024 mutations",
                      scene=("two_rooms", dict(n_tris=200_000, seed=0)),
                      params=dict(n_chains=1 << 16, width=512, height=512, region_px=16,
                                  max_depth=10, epoch_len=16, n_bootstrap=1 << 20, p_large=0.3,
                                  seed=1),
                      mutations=1024, cpu_chains=4096, cpu_epochs=4),
    "cornell": dict(desc="Cornell box, 34+2 triangles (brute force), 64x64, 8-px regions, depth 5, "
                         "64 chains x 1e4 mutations",
                    scene=("cornell_box", {}),
                    params=dict(n_chains=64, width=64, height=64, region_px=8, max_depth=5,
                                epoch_len=16, n_bootstrap=1 << 16, p_large=0.3, seed=1),
                    mutations=10000, cpu_chains=64, cpu_epochs=200),
    "cornell_d10": dict(desc="Cornell box (34+2 triangles, brute force), 64x64, 8-px regions, depth 10, "
                             "2^16 chains x 256 mutations (the Langevin comparison's population)",
                        scene=("cornell_box", {}),
                        params=dict(n_chains=1 << 16, width=64, height=64, region_px=8, max_depth=10,
                                    epoch_len=16, n_bootstrap=1 << 20, p_large=0.3, seed=1),
                        mutations=256, cpu_chains=256, cpu_epochs=8),
    "corridor": dict(desc="glossy corridor lit through a slit, 2M triangles, 1920x1080, 32-px "
                          "regions, depth 12, 2^20 chains x 256 mutations",
                     scene=("glossy_corridor", dict(n_tris=2_000_000, seed=0)),
                     params=dict(n_chains=1 << 20, width=1920, height=1080, region_px=32,
                                 max_depth=12, epoch_len=16, n_bootstrap=1 << 21, p_large=0.3,
                                 seed=1),
                     mutations=256, cpu_chains=1024, cpu_epochs=2),
}


def measured_traffic(workload: str = "two_rooms"):
    """DRAM bytes per chain-kernel launch from the committed ncu capture of the
    two-rooms workload, or None for another workload or when the kernel
    source changed since the capture."""
    import hashlib
    if workload != "two_rooms":
        return None
    try:
        rec = json.loads((ROOT / "profiles" / "chain_epoch_kernel_traffic.json").read_text())
        csrc = ROOT / "paper_2402_08273_gb300" / "csrc"
        src = (csrc / "rmlt_kernels.cu").read_bytes() + (csrc / "rmlt_device.cuh").read_bytes()
        if hashlib.sha256(src).hexdigest()[:16] != rec["kernel_source_sha256_16"]:
            return None
        return rec["dram_bytes_read_per_launch"] + rec["dram_bytes_write_per_launch"]
    except (OSError, KeyError, ValueError):
        return None


def shard_params(base: dict, rank: int, world: int) -> dict:
    """Rank `rank`'s share of the population of base["n_chains"] chains
    (global ids rank * C / world ..., the same seed on every rank).  One rank
    is the unsharded population."""
    p = dict(base)
    C = base["n_chains"]
    if world == 1:
        return p
    if C % world:
        raise ValueError(f"{C} chains do not split over {world} ranks")
    per = C // world
    p.update(n_chains=per, chain_first=rank * per, chains_total=C)
    return p


def step_sharded(chains, n_epochs: int, counts, sums, all_reduce):
    """n_epochs epochs of a sharded population: each epoch this rank's chains
    mutate, the region statistics they added are summed over the ranks (the
    only data-path exchange: 3 m + 1 integers and m doubles), and every rank
    runs the same region update on the summed tables.  `chains` is a CUDA
    Renderer or an oracle population (the same two calls)."""
    for _ in range(n_epochs):
        chains.epoch_mutate(counts, sums)
        all_reduce(counts)
        all_reduce(sums)
        chains.epoch_update(counts, sums)


def reduce_job(dist, world: int, t_local: float, counts: dict, device) -> tuple[float, dict]:
    """Whole-job numbers: the time is the maximum over ranks, counts are summed."""
    import torch
    t = torch.tensor([t_local], dtype=torch.float64, device=device)
    c = torch.tensor([float(v) for v in counts.values()], dtype=torch.float64, device=device)
    if world > 1:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(c, op=dist.ReduceOp.SUM)
    return float(t.item()), dict(zip(counts, c.tolist()))


def make_scene(w):
    from paper_2402_08273_gb300 import scenes
    name, kw = w["scene"]
    return getattr(scenes, name)(**kw)


# ----------------------------------------------------------------------------
# clocks during the timed region
# ----------------------------------------------------------------------------
class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines: list[str] = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.th = threading.Thread(target=self._read, daemon=True)
            self.th.start()
        except (OSError, FileNotFoundError):
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                smax.append(float(f[2]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ----------------------------------------------------------------------------
# the oracle on the host cores (CPU baseline and the reference arm)
# ----------------------------------------------------------------------------
def oracle_sample(w, chains: int, epochs: int) -> dict:
    """Time the CPU oracle (single thread, as it stands) on a bounded sample of
    the workload: `chains` chains x `epochs` epochs, the bootstrap excluded."""
    import oracle
    scene = make_scene(w)
    p = dict(w["params"])
    p.update(n_chains=chains, n_bootstrap=chains)
    osc = oracle.Scene(scene, use_bvh=True)
    keys = ("n_chains", "width", "height", "region_px", "max_depth", "epoch_len", "n_bootstrap",
            "p_large", "seed")
    ch = oracle.Chains(osc, **{k: p[k] for k in keys})
    ch.init()
    t0 = time.perf_counter()
    ch.run_epochs(epochs)
    dt = time.perf_counter() - t0
    st = ch.stats()
    n_mut = chains * epochs * p["epoch_len"]
    return {"value": n_mut / dt, "unit": "mutations/s", "rays_per_s": st["rays"] / dt, "cores": 1,
            "kind": "oracle", "seconds": dt,
            "sample": f"{chains} chains x {epochs * p['epoch_len']} mutations of the same scene and "
                      f"parameters (bootstrap excluded), single-threaded binary64 oracle"}


def _oracle_worker(wname, chains, epochs, worker, barrier, out):
    """One single-threaded oracle population (seed offset by the worker index:
    independent chains, like one GPU of the weak-scaling runs)."""
    import oracle
    w = WORKLOADS[wname]
    p = dict(w["params"])
    p.update(n_chains=chains, n_bootstrap=chains, seed=p["seed"] + 7919 * worker)
    keys = ("n_chains", "width", "height", "region_px", "max_depth", "epoch_len", "n_bootstrap",
            "p_large", "seed")
    ch = oracle.Chains(oracle.Scene(make_scene(w), use_bvh=True), **{k: p[k] for k in keys})
    ch.init()
    barrier.wait()
    t0 = time.perf_counter()
    ch.run_epochs(epochs)
    dt = time.perf_counter() - t0
    out.put((chains * epochs * p["epoch_len"], dt, ch.stats()["rays"]))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_sample_all_cores(wname, chains: int, epochs: int, workers: int) -> dict:
    """The oracle on every host core at once: `workers` independent
    single-threaded populations of `chains` chains x `epochs` epochs, started
    together (spawned processes; the CUDA context of this process is never
    forked); throughput = all mutations / the slowest worker's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(wname, chains, epochs, i, barrier, out))
             for i in range(workers)]
    for pr in procs:
        pr.start()
    res = [out.get() for _ in procs]
    for pr in procs:
        pr.join()
    n_mut = sum(r[0] for r in res)
    dt = max(r[1] for r in res)
    rays = sum(r[2] for r in res)
    ep = WORKLOADS[wname]["params"]["epoch_len"] * epochs
    return {"value": n_mut / dt, "unit": "mutations/s", "rays_per_s": rays / dt, "cores": workers,
            "kind": "oracle", "seconds": dt,
            "sample": f"{workers} processes x {chains} chains x {ep} mutations of the same scene and parameters "
                      f"(independent seeds, bootstrap excluded), single-threaded binary64 oracle in each"}


def run_reference(args, w):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    vals = []
    cores = host_cores()
    chains = max(64, w["cpu_chains"] // 8)
    for _ in range(args.warmup):
        oracle_sample_all_cores(args.workload, chains, 1, cores)
    cpu = None
    for _ in range(args.steps):
        cpu = oracle_sample_all_cores(args.workload, chains, 1, cores)
        vals.append(cpu["value"])
    v = statistics.median(vals)
    cpu["value"] = v
    line = {"impl": "reference", "metric": "mutations/s", "value": v, "unit": "mutations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": cpu["seconds"] * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"]},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "mutations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def run_ours(args, w):
    import torch
    import torch.distributed as dist
    from paper_2402_08273_gb300 import rmlt

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    def barrier():
        if world > 1:
            dist.barrier()

    scene = make_scene(w)
    # weak scaling: each GPU holds the workload's chain count; the population
    # of world x that many chains is split by global chain id
    base = dict(w["params"])
    base.update(n_chains=base["n_chains"] * world, n_bootstrap=base["n_bootstrap"] * world)
    params = shard_params(base, rank, world)
    M = w["mutations"]
    stream = torch.cuda.Stream(device=dev)
    R = rmlt.Renderer(device=local, stream=stream)
    t0 = time.perf_counter()
    R.load_scene(scene)
    t_load = time.perf_counter() - t0
    t0 = time.perf_counter()
    R.init_chains(**params)
    R.synchronize()
    t_init = time.perf_counter() - t0
    C = params["n_chains"]
    E = params["epoch_len"]
    epochs_per_step = -(-M // E)
    if world > 1:
        counts, sums = R.exchange_buffers()

        def all_reduce(t):
            with torch.cuda.stream(stream):
                dist.all_reduce(t)

        def step(n):
            step_sharded(R, -(-n // E), counts, sums, all_reduce)
    else:
        step = R.step

    # the traversal roofline's two ceilings, measured on this GPU
    l2_gbs, fp32_tflops = C_double(), C_double()
    rmlt._check(rmlt.lib().rmlt_probe_peaks(local, C_void_p(stream.cuda_stream), byref(l2_gbs), byref(fp32_tflops)))
    l2_gbs, fp32_tflops = l2_gbs.value, fp32_tflops.value

    for _ in range(args.warmup):
        step(M)
    R.synchronize()
    # execution form: forced, or the fastest candidate timed on the live chains
    from paper_2402_08273_gb300 import autotune
    tuned = None
    if args.form == "auto":
        best, timings = autotune.autotune(R, step=step)
        form = best["form"]
        tuned = {"chosen": best, "ms_per_epoch": [[c, round(t, 3)] for c, t in timings]}
    else:
        form = args.form
        autotune.apply(R, {"form": form})
    R.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st0 = R.read_stats()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(args.steps):
        with torch.cuda.stream(stream):
            flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        step(M)
        e1.record(stream)
        times.append((e0, e1))
    torch.cuda.synchronize()
    clk = clocks.stop()
    barrier()
    step_ms = [a.elapsed_time(b) for a, b in times]
    t_dev = sum(step_ms) / 1e3
    st1 = R.read_stats()
    t_max, tot = reduce_job(dist, world, t_dev, {"mutations": C * M * args.steps,
                                                  "rays": st1["rays"] - st0["rays"]}, dev)
    mutations, rays = tot["mutations"], tot["rays"]
    value = mutations / t_max

    # end to end through the public API: the step plus the image and region
    # histogram read into pinned host memory every step
    img_h = torch.empty((params["height"], params["width"], 3), dtype=torch.float64).pin_memory()
    hist_h = torch.empty(R.m, dtype=torch.int64).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step(M)
        R.read_image(out=img_h.numpy())
        R.read_region_hist(out=hist_h.numpy().view("uint64"))
    torch.cuda.synchronize()
    t_e2e, _ = reduce_job(dist, world, time.perf_counter() - t0, {"steps": args.steps}, dev)
    e2e_value = mutations / t_e2e
    d2h = img_h.numel() * 8 + hist_h.numel() * 8

    # work per ray from one instrumented step (same kernel with counters on)
    R.set_work_counters(True)
    sa = R.read_stats()
    step(params["epoch_len"] * 4)
    sb = R.read_stats()
    R.set_work_counters(False)
    dr = max(1, sb["rays"] - sa["rays"])
    nodes_per_ray = (sb["node_visits"] - sa["node_visits"]) / dr
    tris_per_ray = (sb["tri_tests"] - sa["tri_tests"]) / dr
    flops_ray = nodes_per_ray * FLOPS_PER_NODE + tris_per_ray * FLOPS_PER_TRI
    bytes_ray = nodes_per_ray * BYTES_PER_NODE + tris_per_ray * BYTES_PER_TRI
    rays_per_s_gpu = rays / world / t_max   # per GPU, for the per-kernel roofline
    # traversal roofline: rays/s_max = min(P_fp32 / flops_ray, BW_L2 / bytes_ray)
    alu_max = fp32_tflops * 1e12 / flops_ray
    l2_max = l2_gbs * 1e9 / bytes_ray
    alu = {"achieved_tflops": flops_ray * rays_per_s_gpu / 1e12, "peak_tflops": fp32_tflops,
           "rays_per_s_max": alu_max}
    alu["frac"] = alu["achieved_tflops"] / fp32_tflops
    l2 = {"achieved_gbs": bytes_ray * rays_per_s_gpu / 1e9, "peak_gbs": l2_gbs, "rays_per_s_max": l2_max}
    l2["frac"] = l2["achieved_gbs"] / l2_gbs
    if l2_max <= alu_max:
        bound, achieved, peak, unit = "l2", l2["achieved_gbs"], l2_gbs, "GB/s"
    else:
        bound, achieved, peak, unit = "alu", alu["achieved_tflops"], fp32_tflops, "TFLOP/s"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": measured_traffic(args.workload) if form == "chain" else None,
                "kernel": "chain_epoch_kernel" if form == "chain" else "wavefront waves (shade, setup, trace)",
                "rays_per_s": rays_per_s_gpu, "rays_per_s_max": min(alu_max, l2_max),
                "peak_source": "measured on this GPU by rmlt_probe_peaks before the timed region: L2 read "
                               "bandwidth over a resident quarter-L2 buffer with L1-bypassing 16-byte loads, "
                               "FP32 FMA rate with eight independent chains per thread",
                "ceilings": {"l2": l2, "alu": alu,
                             "alu_nominal_tflops": SM_COUNT * FP32_LANES * 2 * (clk["sm_mhz"] or 2070.0) / 1e6},
                "per_ray": {"nodes": nodes_per_ray, "tris": tris_per_ray, "flops": flops_ray,
                            "bytes": bytes_ray}}
    try:
        peaks = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
        hbm = float(peaks["hbm_gbs"])
        roofline["ceilings"]["hbm"] = {"achieved_gbs": l2["achieved_gbs"], "peak_gbs": hbm,
                                       "frac": l2["achieved_gbs"] / hbm,
                                       "note": "node and triangle bytes against the measured HBM copy rate; "
                                               "the bench scenes' BVH fits in L2"}
    except Exception:
        pass

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        # all host cores (independent populations) and one core, each a bounded sample
        cpu = oracle_sample_all_cores(args.workload, w["cpu_chains"], w["cpu_epochs"], host_cores())
        one = oracle_sample(w, w["cpu_chains"], w["cpu_epochs"])
        cpu["single_core"] = {"value": one["value"], "rays_per_s": one["rays_per_s"], "seconds": one["seconds"]}

    if rank == 0:
        line = {
            "metric": "mutations/s", "value": value, "unit": "mutations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_max * 1e3 / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "chains_per_gpu": C,
                       "mutations_per_step": M, "epochs_per_step": epochs_per_step,
                       "l2": "flushed between timed steps (256 MiB write)", "form": form,
                       "autotune": tuned,
                       "parallelism": (f"dp{world}: one population of {world} x {C} chains split by global "
                                       "chain id; per epoch one all-reduce of the region statistics"
                                       if world > 1 else "one GPU")},
            "rays_per_s": rays / t_max,
            "rays_per_mutation": rays / mutations,
            "gpu_launches": (2 * epochs_per_step * args.steps if form == "chain" else
                             3 * epochs_per_step * args.steps + 3 * (st1["waves"] - st0["waves"])),
            "roofline": roofline,
            "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "mutations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": d2h,
                    "note": "rmlt_step + image and region histogram read to pinned host memory"},
            "clocks": clk,
            "setup_s": {"scene_load_and_bvh": t_load, "init_chains_bootstrap": t_init},
            "stats": {k: st1[k] for k in ("accepted", "large", "small", "early_reject",
                                          "invalid_paths", "stack_overflow")},
        }
        print(json.dumps(line), flush=True)
    R.close()
    if world > 1:
        dist.destroy_process_group()


# ----------------------------------------------------------------------------
# matched relMSE: the variants of the paper's comparison (Sec. 7.1) on one GPU
# ----------------------------------------------------------------------------
def relmse(img, ref) -> float:
    """mean over pixels and channels of (I - R)^2 / (R^2 + 1e-2)"""
    import numpy as np
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + 1e-2)))


def run_relmse(args, w):
    """Fixed / Global / RA-Grid / RA-Quadtree / region-weighted against one
    long reference render (independent seed): relMSE after the same number of
    mutations, and the device time each variant needs to reach a common
    target (the Fixed variant's relMSE after `args.relmse_budget` mutations)."""
    import numpy as np
    import torch
    from paper_2402_08273_gb300 import rmlt
    scene = make_scene(w)
    base = dict(w["params"])
    W, H = base["width"], base["height"]
    variants = {
        "fixed": dict(gamma_max=0.0, gamma_scale=0.0),
        "global": dict(region_px=max(W, H)),
        "ra_grid": dict(),
        "ra_quadtree": dict(partition=1, qt_max_leaves=4096, qt_max_depth=10, qt_split=5000,
                            qt_refine=10_000_000),
        "weighted": dict(target_mode=1),
    }
    # 4-D partition in PSS: the grid's regions crossed with 2 x 2 cells over (u5, u6)
    variants["ra_grid_4d"] = dict(dir_cells=2)
    if all(int(t) == 0 for t in scene["mat_type"]):
        # Langevin strategy (differentiable, Lambertian scenes): 30 % of the
        # mutations, the rest as in the plain variants
        variants["mala"] = dict(p_mala=0.3, mala_tau=1e-3, mala_drift_max=0.1)
    R = rmlt.Renderer(stream=torch.cuda.Stream())
    R.load_scene(scene)
    R.init_chains(**dict(base, seed=base["seed"] + 1000))
    R.step(args.relmse_budget * args.relmse_ref_factor)
    ref = R.read_image()
    R.close()
    budget = args.relmse_budget
    marks = [budget // 8, budget // 4, budget // 2, budget, 2 * budget]
    out = {}
    for name, kw in variants.items():
        R = rmlt.Renderer(stream=torch.cuda.Stream())
        R.load_scene(scene)
        R.init_chains(**dict(base, **kw))
        done, t = 0, 0.0
        curve = []
        for mk in marks:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(R.stream)
            R.step(mk - done)
            e1.record(R.stream)
            torch.cuda.synchronize()
            t += e0.elapsed_time(e1) / 1e3
            done = mk
            curve.append((done, t, relmse(R.read_image(), ref)))
        st = R.read_stats()
        out[name] = {"curve": curve, "accept_rate": st["accepted"] / max(1, st["mutations"] * base["n_chains"]),
                     "regions": st["n_regions"]}
        R.close()
    target = [c for c in out["fixed"]["curve"] if c[0] == budget][0][2]
    for name, o in out.items():
        # device time to reach the target, log-log interpolation between marks
        tt = None
        cv = o["curve"]
        for (m0, t0, e0), (m1, t1, e1) in zip(cv, cv[1:]):
            if e0 >= target >= e1 and e0 > e1:
                a = (math.log(e0) - math.log(target)) / (math.log(e0) - math.log(e1))
                tt = math.exp(math.log(t0) + a * (math.log(t1) - math.log(t0)))
                break
        if tt is None and cv[0][2] <= target:
            tt = cv[0][1] * cv[0][2] / target
        o["seconds_to_target"] = tt
        o["relmse_at_budget"] = [c for c in cv if c[0] == budget][0][2]
    line = {"metric": "seconds to matched relMSE", "unit": "s", "higher_is_better": False,
            "config": {"workload": args.workload, "desc": w["desc"], "budget_mutations_per_chain": budget,
                       "reference_mutations_per_chain": budget * args.relmse_ref_factor,
                       "target_relmse": target, "relmse": "mean (I - R)^2 / (R^2 + 1e-2)"},
            "variants": out}
    print(json.dumps(line), flush=True)


def run_batched(args):
    """32 uneven problems (seeded procedural scenes of 1k-500k triangles,
    128^2-1024^2 images, 4-32 px regions, 2^10-2^17 chains, depth 5-12):
    rmlt_batch_step (one chain-kernel launch and one region-update launch per
    epoch for all members, replayed as a CUDA graph) against the plain form,
    every member stepping alone on its own stream.  Both forms give every
    member the same trajectory (tests/test_gpu_batch.py), so their relMSE is
    equal at equal mutations; the line reports throughput of both."""
    import torch
    from paper_2402_08273_gb300 import rmlt, scenes
    torch.cuda.set_device(0)
    work = scenes.batch_workload(args.batch_members, seed=0)
    main_stream = torch.cuda.Stream()
    Rs = []
    t0 = time.perf_counter()
    for scene, p in work:
        R = rmlt.Renderer(stream=torch.cuda.Stream())
        R.load_scene(scene)
        R.init_chains(**p)
        Rs.append(R)
    torch.cuda.synchronize()
    t_setup = time.perf_counter() - t0
    n = len(Rs)
    M = args.batch_mutations
    E = work[0][1]["epoch_len"]
    chains = sum(p["n_chains"] for _, p in work)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def plain_step(m):
        ev = torch.cuda.Event()
        ev.record(main_stream)
        for R in Rs:
            R.stream.wait_event(ev)
            R.step(m)
        for R in Rs:
            e = torch.cuda.Event()
            e.record(R.stream)
            main_stream.wait_event(e)

    B = rmlt.Batch(Rs)

    def timed(step, steps):
        spans = []
        for _ in range(steps):
            with torch.cuda.stream(main_stream):
                flush.fill_(1)
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(main_stream)
            step()
            b.record(main_stream)
            spans.append((a, b))
        torch.cuda.synchronize()
        return sum(x.elapsed_time(y) for x, y in spans) / 1e3

    def batch_step(m):
        ev = torch.cuda.Event()
        ev.record(main_stream)
        for R in Rs:
            R.stream.wait_event(ev)
        B.step(m)
        for R in Rs:
            e = torch.cuda.Event()
            e.record(R.stream)
            main_stream.wait_event(e)

    def rays_total():
        return sum(R.read_stats()["rays"] for R in Rs)

    def sequential_step(m):
        prev = torch.cuda.Event()
        prev.record(main_stream)
        for R in Rs:
            R.stream.wait_event(prev)
            R.step(m)
            prev = torch.cuda.Event()
            prev.record(R.stream)
        main_stream.wait_event(prev)

    for _ in range(args.warmup):
        plain_step(M)
    r0 = rays_total()
    t_plain = timed(lambda: plain_step(M), args.steps)
    rays_plain = rays_total() - r0
    t_seq = timed(lambda: sequential_step(M), args.steps)
    # launch order: autotuned over three candidates on the live chains
    alone = []
    for R in Rs:
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(R.stream)
        R.step(E)
        b.record(R.stream)
        b.synchronize()
        alone.append(a.elapsed_time(b))
    orders = {"given": list(range(n)),
              "most_chains_first": sorted(range(n), key=lambda i: -work[i][1]["n_chains"]),
              "slowest_alone_first": sorted(range(n), key=lambda i: -alone[i])}
    # candidates: launch mode x launch order x resident blocks per SM, each
    # timed on M mutations (the graph of the branch mode covers one call)
    order_ms = {}
    for mode in ("one_launch", "branches"):
        for ctas in ((4, 3) if mode == "one_launch" else (4,)):
            B.set_shape(ctas, mode == "branches")
            for name, o in orders.items():
                B.set_order(o)
                batch_step(M)
                order_ms[f"{mode}/{name}/{ctas}"] = timed(lambda: batch_step(M), 1) * 1e3 / (M // E)
    best = min(order_ms, key=order_ms.get)
    mode, name, ctas = best.split("/")
    B.set_shape(int(ctas), mode == "branches")
    B.set_order(orders[name])
    for _ in range(args.warmup):
        batch_step(M)
    clocks = ClockSampler(0)
    clocks.start()
    r0 = rays_total()
    t_batch = timed(lambda: batch_step(M), args.steps)
    rays_batch = rays_total() - r0
    clk = clocks.stop()
    # end to end: the batched step plus every member's region histogram read
    # into pinned host memory
    hists = [torch.empty(R.m, dtype=torch.int64).pin_memory() for R in Rs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        batch_step(M)
        for R, hh in zip(Rs, hists):
            R.read_region_hist(out=hh.numpy().view("uint64"))
    torch.cuda.synchronize()
    t_e2e = time.perf_counter() - t0
    mut = chains * M * args.steps
    value = mut / t_batch
    line = {"metric": "mutations/s", "value": value, "unit": "mutations/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_batch * 1e3 / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": f"batched_{n}", "desc": "uneven seeded problems (1k-500k triangles, "
                       "128^2-1024^2 images, 4-32 px regions, 2^10-2^17 chains, depth 5-12), epoch_len 16",
                       "members": n, "chains": chains, "mutations_per_step": M,
                       "l2": "flushed between timed steps (256 MiB write)",
                       "launch_order": best, "order_ms_per_epoch": order_ms},
            "rays_per_s": rays_batch / t_batch,
            "plain_form": {"value": mut / t_plain, "rays_per_s": rays_plain / t_plain,
                           "ms_per_step": t_plain * 1e3 / args.steps,
                           "note": "every member stepping alone on its own stream"},
            "sequential_form": {"value": mut / t_seq, "ms_per_step": t_seq * 1e3 / args.steps,
                                "note": "members stepping alone one after the other"},
            "batched_over_plain": t_plain / t_batch,
            "batched_over_sequential": t_seq / t_batch,
            "gpu_launches": (2 * n if mode == "branches" else 2) * (M // E) * args.steps,
            "e2e": {"value": mut / t_e2e, "unit": "mutations/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": sum(h.numel() * 8 for h in hists),
                    "note": "rmlt_batch_step + every member's region histogram read to pinned host memory"},
            "clocks": clk, "setup_s": t_setup}
    print(json.dumps(line), flush=True)
    B.close()


def run_profile(args, w):
    """The case a profiler captures: the workload's scene and chains (optionally
    fewer chains), `--profile-epochs` epochs in the chosen form, nothing else
    (no probes, no autotuning, no CPU leg)."""
    import torch
    from paper_2402_08273_gb300 import autotune, rmlt
    params = dict(w["params"])
    if args.chains:
        params["n_chains"] = args.chains
        params["n_bootstrap"] = max(params["n_chains"], min(params["n_bootstrap"], 16 * params["n_chains"]))
    R = rmlt.Renderer(stream=torch.cuda.Stream())
    R.load_scene(make_scene(w))
    R.init_chains(**params)
    autotune.apply(R, {"form": "chain" if args.form == "auto" else args.form})
    if args.host_loop:
        R.set_wavefront(host_loop=True)   # waves launched from the host: profilers see each kernel
    R.step(params["epoch_len"] * args.profile_epochs)
    R.synchronize()
    st = R.read_stats()
    print(json.dumps({"profile": args.workload, "form": args.form, "chains": params["n_chains"],
                      "epochs": st["epochs"], "rays": st["rays"]}), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=("ours", "reference"), default="ours")
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="two_rooms")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--form", choices=("auto", "chain", "wavefront"), default="auto",
                    help="epoch execution form: one thread per chain, waves of shade / setup / trace, "
                         "or the faster of the autotuner's candidates (default)")
    ap.add_argument("--relmse", action="store_true",
                    help="compare the Fixed / Global / RA-Grid / RA-Quadtree / weighted variants at matched relMSE")
    ap.add_argument("--batched", action="store_true",
                    help="uneven problems stepped by rmlt_batch_step against stepping each alone")
    ap.add_argument("--batch-members", type=int, default=32)
    ap.add_argument("--batch-mutations", type=int, default=64)
    ap.add_argument("--profile", action="store_true",
                    help="run --profile-epochs epochs of the workload and exit (the case ncu captures)")
    ap.add_argument("--profile-epochs", type=int, default=3)
    ap.add_argument("--chains", type=int, default=0, help="--profile: chain count instead of the workload's")
    ap.add_argument("--host-loop", action="store_true", help="--profile, wavefront form: launch waves from the host")
    ap.add_argument("--relmse-budget", type=int, default=1024)
    ap.add_argument("--relmse-ref-factor", type=int, default=32)
    args = ap.parse_args()
    w = WORKLOADS[args.workload]
    if args.profile:
        run_profile(args, w)
    elif args.batched and args.impl == "ours":
        run_batched(args)
    elif args.relmse:
        run_relmse(args, w)
    elif args.impl == "reference":
        run_reference(args, w)
    else:
        run_ours(args, w)


if __name__ == "__main__":
    main()
