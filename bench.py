#!/usr/bin/env python3
"""Benchmark of the regional adaptive PSS-MLT chain step on one or more GB300s.

Headline workload (default, `--workload corridor`): a 20 m glossy GGX
corridor lit only through a 5 cm slit in its ceiling, a near-specular sphere
(GGX alpha 0.02), seeded jittered spheres and tori up to 2M triangles;
1920 x 1080 image, 32-px regions (60 x 34, partial last row), path depth
<= 12 with next-event estimation (D = 62), 2^20 chains, large-step
probability 0.3, Kelemen small steps s1 = 1/1024, s2 = 1/64, host-built SAH
BVH4, binary32 tracing, binary64 splats and normaliser.

One step = 256 mutations of every chain (16 epochs of 16; rmlt_step on one
GPU, the sharded epoch loop with one all-reduce of the region statistics per
epoch on N GPUs).  The metric is mutations/s (and rays/s) of the whole job;
the line also carries, measured in the same run: the time the paper's
variants (Fixed, Global, RA-Grid, RA-Quadtree, and the region-weighted
target) need to reach a matched relMSE; the traversal roofline with the
kernel's per-ray work cross-checked by an independent host traversal of the
same BVH; the two-rooms workload as a second line; the CPU oracle on the
host cores.  The L2 is flushed between timed steps by writing a 256 MiB
buffer.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference] [--workload NAME]
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

import numpy as np

ROOT = Path(__file__).resolve().parent
sys.path.insert(0, str(ROOT))

# FP32 operations the traversal needs per BVH4 node visit, by node size (128
# bytes, binary32 bounds: four child boxes of 6 FMA + 6 min + 6 max per slab
# test, one compare each, and a 5-comparator sort; 64 bytes, quantised: the
# node grid's three scales and offsets along the ray, 3 mul + 3 FMA, and 6
# grid-index decodes per child, an add each, on top) and per ray-triangle
# test (Moller-Trumbore: two cross products, three dot products, sign
# scaling, 5 compares, one division for a hit); an FMA counts as 2
# floating-point operations.
FLOPS_PER_NODE = {128: 4 * (6 * 2 + 12 + 1) + 5 * 2,                         # 110
                  64: 3 + 3 * 2 + 4 * (6 + 6 * 2 + 12 + 1) + 5 * 2}          # 143
FLOPS_PER_TRI = 2 * (6 * 2) + 3 * 5 + 3 + 5 + 1  # 48
BYTES_PER_NODE = 64    # quantised BVH4 node (the library reports the loaded scene's own: 128 for binary32 nodes)
BYTES_PER_TRI = 48
SM_COUNT = 152
FP32_LANES = 128

WORKLOADS = {
    "corridor": dict(desc="glossy corridor lit through a 5 cm ceiling slit, 2M triangles, 1920x1080, 32-px "
                          "regions, depth 12, 2^20 chains x 256 mutations",
                     scene=("glossy_corridor", dict(n_tris=2_000_000, seed=0)),
                     params=dict(n_chains=1 << 20, width=1920, height=1080, region_px=32,
                                 max_depth=12, epoch_len=16, n_bootstrap=1 << 21, p_large=0.3,
                                 seed=1),
                     mutations=256, cpu_chains=512, cpu_epochs=2, relmse_budget=128),
    "two_rooms": dict(desc="two rooms joined by a 5 cm door gap, 200k triangles, 512x512, 16-px "
                           "regions, depth 10, 2^16 chains x 1024 mutations",
                      scene=("two_rooms", dict(n_tris=200_000, seed=0)),
                      params=dict(n_chains=1 << 16, width=512, height=512, region_px=16,
                                  max_depth=10, epoch_len=16, n_bootstrap=1 << 20, p_large=0.3,
                                  seed=1),
                      mutations=1024, cpu_chains=4096, cpu_epochs=4, relmse_budget=256),
    "cornell": dict(desc="Cornell box, 34+2 triangles (brute force), 64x64, 8-px regions, depth 5, "
                         "64 chains x 1e4 mutations",
                    scene=("cornell_box", {}),
                    params=dict(n_chains=64, width=64, height=64, region_px=8, max_depth=5,
                                epoch_len=16, n_bootstrap=1 << 16, p_large=0.3, seed=1),
                    mutations=10000, cpu_chains=64, cpu_epochs=200, relmse_budget=2000),
    "cornell_d10": dict(desc="Cornell box (34+2 triangles, brute force), 64x64, 8-px regions, depth 10, "
                             "2^16 chains x 256 mutations (the Langevin comparison's population)",
                        scene=("cornell_box", {}),
                        params=dict(n_chains=1 << 16, width=64, height=64, region_px=8, max_depth=10,
                                    epoch_len=16, n_bootstrap=1 << 20, p_large=0.3, seed=1),
                        mutations=256, cpu_chains=256, cpu_epochs=8, relmse_budget=256),
}
SECONDARY = {"corridor": "two_rooms"}


def measured_traffic(workload: str, form: str):
    """DRAM traffic of the workload's dominant kernel from the committed ncu
    capture (profiles/traffic.json): bytes per launch, or bytes per ray for a
    kernel launched once per wave (scaled to the step by its rays); None when
    there is no capture for this workload and form or the kernel source
    changed since."""
    import hashlib
    try:
        rec = json.loads((ROOT / "profiles" / "traffic.json").read_text())[f"{workload}/{form}"]
        csrc = ROOT / "paper_2402_08273_gb300" / "csrc"
        # the files that hold the kernel's device code
        files = rec.get("kernel_sources", ("rmlt_kernels.cu", "rmlt_device.cuh", "rmlt_wavefront.cu"))
        src = b"".join((csrc / f).read_bytes() for f in files)
        if hashlib.sha256(src).hexdigest()[:16] != rec["kernel_source_sha256_16"]:
            return None
        return {"bytes_per_launch": rec.get("dram_bytes_per_launch"), "bytes_per_ray": rec.get("dram_bytes_per_ray"),
                "kernel": rec["kernel"], "scaled_from": rec.get("scaled_from")}
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
ORACLE_KEYS = ("n_chains", "width", "height", "region_px", "max_depth", "epoch_len", "n_bootstrap", "p_large",
               "seed")


def _oracle_worker(wname, chains, epochs, worker, rounds, barrier, out):
    """One single-threaded oracle population (seed offset by the worker
    index: independent chains), built once; each round times `epochs` epochs."""
    import oracle
    w = WORKLOADS[wname]
    p = dict(w["params"])
    p.update(n_chains=chains, n_bootstrap=chains, seed=p["seed"] + 7919 * worker)
    ch = oracle.Chains(oracle.Scene(make_scene(w), use_bvh=True), **{k: p[k] for k in ORACLE_KEYS})
    ch.init()
    for r in range(rounds):
        barrier.wait()
        r0 = ch.stats()["rays"]
        t0 = time.perf_counter()
        ch.run_epochs(epochs)
        dt = time.perf_counter() - t0
        out.put((r, chains * epochs * p["epoch_len"], dt, ch.stats()["rays"] - r0))


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_rounds(wname, chains: int, epochs: int, workers: int, rounds: int) -> list[dict]:
    """The oracle on `workers` host cores at once: independent single-threaded
    populations of `chains` chains, built once (spawned processes: the CUDA
    context of this process is never forked), then `rounds` rounds of
    `epochs` epochs started together.  Per round: all mutations over the
    slowest worker's time."""
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    barrier = ctx.Barrier(workers)
    out = ctx.Queue()
    procs = [ctx.Process(target=_oracle_worker, args=(wname, chains, epochs, i, rounds, barrier, out))
             for i in range(workers)]
    for pr in procs:
        pr.start()
    res = [out.get() for _ in range(workers * rounds)]
    for pr in procs:
        pr.join()
    ep = WORKLOADS[wname]["params"]["epoch_len"] * epochs
    lines = []
    for r in range(rounds):
        rr = [x for x in res if x[0] == r]
        n_mut = sum(x[1] for x in rr)
        dt = max(x[2] for x in rr)
        rays = sum(x[3] for x in rr)
        lines.append({"value": n_mut / dt, "unit": "mutations/s", "rays_per_s": rays / dt, "cores": workers,
                      "kind": "oracle", "seconds": dt,
                      "sample": f"{workers} processes x {chains} chains x {ep} mutations of the same scene and "
                                f"parameters (independent seeds, bootstrap excluded), single-threaded binary64 "
                                f"oracle in each"})
    return lines


def run_reference(args, w):
    """The reference arm: the CPU oracle, as it stands, on every host core,
    each step a bounded sample of the workload."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    cores = host_cores()
    chains = max(32, w["cpu_chains"] // 2)
    rounds = oracle_rounds(args.workload, chains, 1, cores, args.warmup + args.steps)[args.warmup:]
    v = statistics.median(r["value"] for r in rounds)
    cpu = dict(rounds[-1])
    cpu["value"] = v
    line = {"impl": "reference", "metric": "mutations/s", "value": v, "unit": "mutations/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": statistics.median(r["seconds"] for r in rounds) * 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"]},
            "cpu_baseline": cpu,
            "e2e": {"value": v, "unit": "mutations/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(wname) -> dict:
    """The oracle on all host cores (one round) and on one core, each a
    bounded sample of the workload."""
    w = WORKLOADS[wname]
    cpu = oracle_rounds(wname, w["cpu_chains"], w["cpu_epochs"], host_cores(), 1)[0]
    one = oracle_rounds(wname, w["cpu_chains"], w["cpu_epochs"], 1, 1)[0]
    cpu["single_core"] = {"value": one["value"], "rays_per_s": one["rays_per_s"], "seconds": one["seconds"]}
    return cpu


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------
def traversal_crosscheck(R, n_sample: int = 4096) -> dict:
    """Per-ray traversal work of the chain kernel's own traversal against an
    independent reference traversal of the same uploaded BVH on the host
    (binary64, nearest child first), on every ray of the paths of a sample of
    the chains' current states."""
    import torch
    q = R.read_chain_state()["q"]
    C = q.shape[1]
    pick = np.arange(0, C, max(1, C // n_sample))[:n_sample]
    qs = torch.from_numpy(np.ascontiguousarray(q[:, pick]).view(np.int32)).cuda(R.device)
    rays, work = R.record_paths(qs)
    live = rays[..., 3] >= 0
    t0 = time.perf_counter()
    host = R.walk_rays_host(rays)
    t_host = time.perf_counter() - t0
    k, h = work[live], host[live]
    same_hit = k[:, 0] == h[:, 0]
    same_work = (k[:, 2] == h[:, 2]) & (k[:, 3] == h[:, 3])
    return {"paths": int(len(pick)), "rays": int(live.sum()),
            "kernel_nodes_per_ray": float(k[:, 2].mean()), "host_nodes_per_ray": float(h[:, 2].mean()),
            "kernel_tris_per_ray": float(k[:, 3].mean()), "host_tris_per_ray": float(h[:, 3].mean()),
            "same_hit_frac": float(same_hit.mean()), "same_work_frac": float(same_work.mean()),
            "host_seconds": t_host,
            "method": "every ray of the paths of a sample of the chains' states: the chain kernel's traversal "
                      "(rmlt_record_paths) against a binary64 host traversal of the same BVH (rmlt_walk_rays_host)"}


def relmse(img, ref) -> float:
    """mean over pixels and channels of (I - R)^2 / (R^2 + 1e-2)"""
    return float(np.mean((img - ref) ** 2 / (ref ** 2 + 1e-2)))


RELMSE_VARIANTS = {
    "fixed": dict(gamma_max=0.0, gamma_scale=0.0),
    "global": dict(region_px=1 << 16),
    "ra_grid": dict(),
    "ra_quadtree": dict(partition=1, qt_max_leaves=4096, qt_max_depth=10, qt_split=5000, qt_refine=10_000_000),
    "weighted": dict(target_mode=1),
}


def relmse_block(R, w, budget: int, ref_factor: int, variants: dict, sync) -> dict:
    """The paper's equal-error comparison (Sec. 7.1) on the loaded scene: a
    reference render (independent seed, ref_factor x longer), then each
    variant's relMSE after budget / 4 .. 2 budget mutations per chain and the
    device time it needs to reach the Fixed variant's relMSE at `budget`
    (log-log interpolation between marks)."""
    import torch
    base = dict(w["params"])
    R.init_chains(**dict(base, seed=base["seed"] + 1000))
    R.step(budget * ref_factor)
    ref = R.read_image()
    marks = [budget // 4, budget // 2, budget, 2 * budget]
    out = {}
    for name, kw in variants.items():
        p = dict(base, **kw)
        if p["region_px"] > max(p["width"], p["height"]):
            p["region_px"] = max(p["width"], p["height"])
        R.init_chains(**p)
        sync()
        done, t = 0, 0.0
        curve = []
        for mk in marks:
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(R.stream)
            R.step(mk - done)
            e1.record(R.stream)
            e1.synchronize()
            t += e0.elapsed_time(e1) / 1e3
            done = mk
            curve.append((done, t, relmse(R.read_image(), ref)))
        st = R.read_stats()
        out[name] = {"curve": curve, "accept_rate": st["accepted"] / max(1, st["mutations"] * p["n_chains"]),
                     "regions": st["n_regions"]}
    target = [c for c in out["fixed"]["curve"] if c[0] == budget][0][2]
    for name, o in out.items():
        tt = None
        cv = o["curve"]
        for (m0, t0, e0), (m1, t1, e1) in zip(cv, cv[1:]):
            if e0 >= target >= e1 and e0 > e1:
                a = (math.log(e0) - math.log(target)) / (math.log(e0) - math.log(e1))
                tt = math.exp(math.log(t0) + a * (math.log(t1) - math.log(t0)))
                break
        if tt is None and cv[0][2] <= target and target > 0:
            tt = cv[0][1] * cv[0][2] / target
        o["seconds_to_target"] = tt
        o["relmse_at_budget"] = [c for c in cv if c[0] == budget][0][2]
    return {"budget_mutations_per_chain": budget, "reference_mutations_per_chain": budget * ref_factor,
            "target_relmse": target, "relmse": "mean (I - R)^2 / (R^2 + 1e-2)",
            "reference": "the same workload with an independent seed, run ref_factor x longer", "variants": out}


def gpu_launches(form: str, epochs: int, waves: int, world: int) -> int:
    """Kernels of this library launched for `epochs` epochs: the chain kernel
    and the region update per epoch; the wavefront form's begin, two
    transposes, end and three kernels per wave; the sharded epoch's snapshot,
    pack and unpack."""
    n = (2 if form == "chain" else 5) * epochs + (3 * waves if form != "chain" else 0)
    return n + (3 * epochs if world > 1 else 0)


def measure(wname, steps, warmup, form_arg, world=1, rank=0, local=0, dist=None, peaks=None, full=True):
    """Time `steps` steps of workload `wname` (after `warmup`), with its
    roofline, end-to-end figure and (full) the traversal cross-check and the
    matched-relMSE block."""
    import torch
    from paper_2402_08273_gb300 import autotune, rmlt
    w = WORKLOADS[wname]
    dev = torch.device("cuda", local)
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

    def barrier():
        if world > 1:
            dist.barrier()

    for _ in range(warmup):
        step(M)
    R.synchronize()
    # execution form: forced, or the fastest candidate timed on the live chains
    tuned = None
    if form_arg == "auto":
        best, timings = autotune.autotune(R, step=step)
        form = best["form"]
        tuned = {"chosen": best, "ms_per_epoch": [[c, round(t, 3)] for c, t in timings]}
    else:
        form = form_arg
        autotune.apply(R, {"form": form})
    R.synchronize()
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)
    st0 = R.read_stats()
    clocks = ClockSampler(local)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    times = []
    for _ in range(steps):
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
    t_dev = sum(a.elapsed_time(b) for a, b in times) / 1e3
    st1 = R.read_stats()
    t_max, tot = reduce_job(dist, world, t_dev, {"mutations": C * M * steps, "rays": st1["rays"] - st0["rays"]},
                            dev)
    mutations, rays = tot["mutations"], tot["rays"]
    value = mutations / t_max

    # end to end through the public API: the step plus the image and region
    # histogram read into pinned host memory every step
    e2e_steps = min(steps, 5)
    img_h = torch.empty((params["height"], params["width"], 3), dtype=torch.float64).pin_memory()
    hist_h = torch.empty(R.m, dtype=torch.int64).pin_memory()
    barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(M)
        R.read_image(out=img_h.numpy())
        R.read_region_hist(out=hist_h.numpy().view("uint64"))
    torch.cuda.synchronize()
    t_e2e, _ = reduce_job(dist, world, time.perf_counter() - t0, {"steps": e2e_steps}, dev)
    e2e = {"value": C * world * M * e2e_steps / t_e2e, "unit": "mutations/s", "h2d_bytes_per_step": 0,
           "d2h_bytes_per_step": img_h.numel() * 8 + hist_h.numel() * 8, "steps": e2e_steps,
           "note": "the step through the public API plus the image and region histogram read to pinned host "
                   "memory; the chain state stays on the device, so no input is copied in per step"}

    # work per ray from one instrumented run (the same kernels with counters on)
    R.set_work_counters(True)
    sa = R.read_stats()
    step(E * 4)
    sb = R.read_stats()
    R.set_work_counters(False)
    dr = max(1, sb["rays"] - sa["rays"])
    nodes_per_ray = (sb["node_visits"] - sa["node_visits"]) / dr
    tris_per_ray = (sb["tri_tests"] - sa["tri_tests"]) / dr
    node_bytes = sb["node_bytes"] or BYTES_PER_NODE
    flops_ray = nodes_per_ray * FLOPS_PER_NODE[node_bytes] + tris_per_ray * FLOPS_PER_TRI
    bytes_ray = nodes_per_ray * node_bytes + tris_per_ray * BYTES_PER_TRI
    rays_per_s_gpu = rays / world / t_max   # per GPU, for the per-kernel roofline
    l2_gbs, fp32_tflops = peaks["l2_gbs"], peaks["fp32_tflops"]
    # traversal roofline: rays/s_max = min(P_fp32 / flops_ray, BW / bytes_ray)
    alu_max = fp32_tflops * 1e12 / flops_ray
    l2_max = l2_gbs * 1e9 / bytes_ray
    alu = {"achieved_tflops": flops_ray * rays_per_s_gpu / 1e12, "peak_tflops": fp32_tflops,
           "rays_per_s_max": alu_max}
    alu["frac"] = alu["achieved_tflops"] / fp32_tflops
    l2 = {"achieved_gbs": bytes_ray * rays_per_s_gpu / 1e9, "peak_gbs": l2_gbs, "rays_per_s_max": l2_max}
    l2["frac"] = l2["achieved_gbs"] / l2_gbs
    bound, achieved, peak, unit = ("l2", l2["achieved_gbs"], l2_gbs, "GB/s") if l2_max <= alu_max else \
        ("alu", alu["achieved_tflops"], fp32_tflops, "TFLOP/s")
    tr = measured_traffic(wname, form)
    traffic, traffic_per = None, None
    if tr and tr["bytes_per_ray"] is not None:
        # every trace launch of one step: the captured bytes per ray times the step's rays (per GPU)
        traffic, traffic_per = tr["bytes_per_ray"] * rays / world / steps, "step (all of the kernel's launches)"
    elif tr:
        traffic, traffic_per = tr["bytes_per_launch"], "launch"
    roofline = {"bound": bound, "achieved": achieved, "peak": peak, "unit": unit, "frac": achieved / peak,
                "traffic": traffic, "traffic_per": traffic_per,
                "traffic_algorithmic": bytes_ray * rays / world / steps,
                "traffic_kernel": (tr["kernel"] if tr else None),
                "traffic_source": (tr["scaled_from"] if tr else None),
                "kernel": "chain_epoch_kernel" if form == "chain" else "wavefront waves (shade, setup, trace)",
                "achieved_over": "the whole step's device time (every kernel of the step), so the dominant "
                                 "kernel's own rate is higher by its share of the step",
                "rays_per_s": rays_per_s_gpu, "rays_per_s_max": min(alu_max, l2_max),
                "peak_source": "measured on this GPU by rmlt_probe_peaks before the timed region: L2 read "
                               "bandwidth over a resident quarter-L2 buffer with L1-bypassing 16-byte loads, "
                               "FP32 FMA rate with eight independent chains per thread",
                "ceilings": {"l2": l2, "alu": alu,
                             "alu_nominal_tflops": SM_COUNT * FP32_LANES * 2 * (clk["sm_mhz"] or 2070.0) / 1e6},
                "per_ray": {"nodes": nodes_per_ray, "tris": tris_per_ray, "flops": flops_ray, "bytes": bytes_ray,
                            "node_bytes": node_bytes,
                            "source": "the kernels' work counters over every ray of four epochs"}}
    if peaks.get("hbm_gbs"):
        hbm = peaks["hbm_gbs"]
        roofline["ceilings"]["hbm"] = {"achieved_gbs": l2["achieved_gbs"], "peak_gbs": hbm,
                                       "frac": l2["achieved_gbs"] / hbm, "peak_source": peaks["hbm_source"],
                                       "note": "node and triangle bytes against the measured HBM copy rate "
                                               "(binding where the BVH and triangles exceed the L2)"}
    out = {"value": value, "ms_per_step": t_max * 1e3 / steps, "rays": rays, "mutations": mutations,
           "rays_per_s": rays / t_max, "form": form, "autotune": tuned, "roofline": roofline, "e2e": e2e,
           "clocks": clk, "setup_s": {"scene_load_and_bvh": t_load, "init_chains_bootstrap": t_init},
           "stats": {k: st1[k] for k in ("accepted", "large", "small", "early_reject", "invalid_paths",
                                         "stack_overflow", "boot_overflow")},
           "gpu_launches": gpu_launches(form, epochs_per_step * steps, st1["waves"] - st0["waves"], world),
           "chains_per_gpu": C, "epochs_per_step": epochs_per_step, "M": M}
    if full and rank == 0 and world == 1:
        out["crosscheck"] = traversal_crosscheck(R)
        roofline["per_ray"]["crosscheck"] = out["crosscheck"]
        t0 = time.perf_counter()
        out["relmse"] = relmse_block(R, w, w["relmse_budget"], 16, RELMSE_VARIANTS, R.synchronize)
        out["relmse"]["seconds_wall"] = time.perf_counter() - t0
        out["relmse"]["form"] = form
    R.close()
    return out


def probe_peaks(local, stream) -> dict:
    from paper_2402_08273_gb300 import rmlt
    l2_gbs, fp32_tflops = C_double(), C_double()
    rmlt._check(rmlt.lib().rmlt_probe_peaks(local, C_void_p(stream.cuda_stream), byref(l2_gbs), byref(fp32_tflops)))
    p = {"l2_gbs": l2_gbs.value, "fp32_tflops": fp32_tflops.value, "hbm_gbs": None}
    try:
        mp = json.loads((ROOT / "MEASURED_PEAKS.json").read_text())
        p["hbm_gbs"], p["hbm_source"] = float(mp["hbm_gbs"]), "MEASURED_PEAKS.json (measured copy rate)"
    except Exception:
        p["hbm_gbs"], p["hbm_source"] = 6800.0, "fallback 6.8 TB/s (no measured peaks file)"
    return p


def run_ours(args, w):
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    peaks = probe_peaks(local, torch.cuda.Stream())
    m = measure(args.workload, args.steps, args.warmup, args.form, world, rank, local, dist, peaks,
                full=not args.quick)
    secondary = None
    sec_name = SECONDARY.get(args.workload)
    if rank == 0 and world == 1 and sec_name and not args.quick:
        s = measure(sec_name, min(args.steps, 5), min(args.warmup, 3), args.form, peaks=peaks, full=False)
        secondary = {"workload": sec_name, "desc": WORKLOADS[sec_name]["desc"], "value": s["value"],
                     "unit": "mutations/s", "rays_per_s": s["rays_per_s"], "ms_per_step": s["ms_per_step"],
                     "steps": min(args.steps, 5), "form": s["form"],
                     "roofline": {k: s["roofline"][k] for k in ("bound", "achieved", "peak", "unit", "frac",
                                                                "traffic", "per_ray")},
                     "e2e": s["e2e"], "clocks": s["clocks"]}
    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        cpu = cpu_baseline(args.workload)
    if rank == 0:
        line = {
            "metric": "mutations/s", "value": m["value"], "unit": "mutations/s", "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": m["ms_per_step"],
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": args.workload, "desc": w["desc"], "chains_per_gpu": m["chains_per_gpu"],
                       "mutations_per_step": m["M"], "epochs_per_step": m["epochs_per_step"],
                       "l2": "flushed between timed steps (256 MiB write)", "form": m["form"],
                       "autotune": m["autotune"],
                       "parallelism": (f"dp{world}: one population of {world} x {m['chains_per_gpu']} chains split "
                                       "by global chain id; per epoch one all-reduce of the region statistics"
                                       if world > 1 else "one GPU")},
            "rays_per_s": m["rays_per_s"],
            "rays_per_mutation": m["rays"] / m["mutations"],
            "gpu_launches": m["gpu_launches"],
            "roofline": m["roofline"],
            "relmse": m.get("relmse"),
            "cpu_baseline": cpu,
            "e2e": m["e2e"],
            "clocks": m["clocks"],
            "setup_s": m["setup_s"],
            "stats": m["stats"],
            "secondary": secondary,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def run_relmse(args, w):
    """--relmse: the variants of the paper's comparison (Sec. 7.1), plus the
    4-D partition and (Lambertian scenes) the Langevin strategy, at a chosen
    budget against a long reference render."""
    import torch
    from paper_2402_08273_gb300 import autotune, rmlt
    scene = make_scene(w)
    variants = dict(RELMSE_VARIANTS)
    variants["ra_grid_4d"] = dict(dir_cells=2)
    if all(int(t) == 0 for t in scene["mat_type"]):
        variants["mala"] = dict(p_mala=0.3, mala_tau=1e-3, mala_drift_max=0.1)
    R = rmlt.Renderer(stream=torch.cuda.Stream())
    R.load_scene(scene)
    if args.form != "auto":
        R.init_chains(**w["params"])
        autotune.apply(R, {"form": args.form})
    blk = relmse_block(R, w, args.relmse_budget or w["relmse_budget"], args.relmse_ref_factor, variants,
                       R.synchronize)
    R.close()
    line = {"metric": "seconds to matched relMSE", "unit": "s", "higher_is_better": False,
            "config": {"workload": args.workload, "desc": w["desc"]}, **blk}
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
    ap.add_argument("--workload", choices=tuple(WORKLOADS), default="corridor")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--quick", action="store_true",
                    help="the timed steps only: no cross-check, matched-relMSE block or second workload")
    ap.add_argument("--form", choices=("auto", "chain", "wavefront"), default="auto",
                    help="epoch execution form: one thread per chain, waves of shade / setup / trace, "
                         "or the faster of the autotuner's candidates (default)")
    ap.add_argument("--relmse", action="store_true",
                    help="only the variants of the paper's comparison at matched relMSE (and 4-D, Langevin)")
    ap.add_argument("--batched", action="store_true",
                    help="uneven problems stepped by rmlt_batch_step against stepping each alone")
    ap.add_argument("--batch-members", type=int, default=32)
    ap.add_argument("--batch-mutations", type=int, default=64)
    ap.add_argument("--profile", action="store_true",
                    help="run --profile-epochs epochs of the workload and exit (the case ncu captures)")
    ap.add_argument("--profile-epochs", type=int, default=3)
    ap.add_argument("--chains", type=int, default=0, help="--profile: chain count instead of the workload's")
    ap.add_argument("--host-loop", action="store_true", help="--profile, wavefront form: launch waves from the host")
    ap.add_argument("--relmse-budget", type=int, default=0, help="--relmse: mutations per chain (0: the workload's)")
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
