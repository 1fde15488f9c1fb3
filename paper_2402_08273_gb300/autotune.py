"""Launch-shape autotuner for rmlt_step.

The execution form of an epoch (one thread per chain, or waves of shade /
setup / trace kernels) and its knobs change speed only, never results: every
form draws the same Philox numbers and evaluates each path with the same
arithmetic.  So the tuner times each candidate on the live chains for a few
epochs (CUDA events on the renderer's stream) and leaves the fastest one set.
Which form wins depends on the population: a wave costs the latency of its
slowest ray, so waves pay off once there are many more chains than lanes to
run them on.
"""
from __future__ import annotations

CANDIDATES = (
    {"form": "chain", "batch_shade": 12, "batch_setup": 10},
    {"form": "chain", "batch_shade": 12, "batch_setup": 8},
    {"form": "chain", "batch_shade": 12, "batch_setup": 12},
    {"form": "chain", "batch_shade": 8, "batch_setup": 10},
    {"form": "chain", "batch_shade": 16, "batch_setup": 10},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 8},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 6},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 16},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 8, "short_stack": True},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 8, "leaf_batch": 6},
    {"form": "wavefront", "trace_ctas_per_sm": 0, "refill_lanes": 8, "leaf_batch": 10},
)


def apply(R, cand: dict) -> None:
    """Set candidate `cand` on renderer R."""
    if cand["form"] == "chain":
        R.set_tuning(batch_shade=cand.get("batch_shade", 12), batch_setup=cand.get("batch_setup", 10))
    else:
        R.set_tuning(wavefront=True)
        R.set_trace_leaf_batch(cand.get("leaf_batch", 8))
        R.set_wavefront(trace_ctas_per_sm=cand.get("trace_ctas_per_sm", 0),
                        setup_ctas_per_sm=cand.get("setup_ctas_per_sm", 0),
                        refill_lanes=cand.get("refill_lanes", 8), short_stack=cand.get("short_stack", False),
                        host_loop=cand.get("host_loop", False))


def autotune(R, epochs: int = 2, candidates=CANDIDATES, step=None):
    """Time each candidate for `epochs` epochs after one untimed epoch (graph
    build, caches); set the fastest.  `step(n_mutations)` advances the chains
    (default R.step; a sharded population passes its epoch loop).  Returns
    (best, [(cand, ms_per_epoch)])."""
    import torch
    step = step or R.step
    E = R.params["epoch_len"]
    timings = []
    for cand in candidates:
        apply(R, cand)
        step(E)
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(R.stream)
        step(epochs * E)
        b.record(R.stream)
        b.synchronize()
        timings.append((dict(cand), a.elapsed_time(b) / epochs))
    best = min(timings, key=lambda t: t[1])[0]
    apply(R, best)
    return best, timings
