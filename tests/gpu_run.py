"""Helpers that run the CUDA library with the trace instrument (GPU tests only)."""
from __future__ import annotations

import numpy as np

from paper_2402_08273_gb300 import rmlt


def traced_run(scene=None, toy=None, n_epochs=4, stride=1, brute_force_max=0, **params):
    """Initialise, trace `n_epochs` epochs of every `stride`-th chain, and
    return the trace together with the initial and final state."""
    import torch
    R = rmlt.Renderer()
    if toy is not None:
        R.load_toy_integrand(toy)
    else:
        R.load_scene(scene, brute_force_max=brute_force_max)
    R.init_chains(**params)
    p = R.params
    init = R.read_chain_state()
    E = p["epoch_len"]
    n_traced = -(-p["n_chains"] // stride)
    rec = torch.zeros(n_epochs * n_traced * E * rmlt.TRACE_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    lam = torch.zeros(n_epochs * R.m, dtype=torch.float64, device="cuda")
    R.set_trace(rec, lam, stride)
    R.step(n_epochs * E)
    R.synchronize()
    R.set_trace(None)
    out = {
        "R": R,
        "params": p,
        "init": init,
        "trace": rmlt.trace_to_numpy(rec).reshape(n_epochs, n_traced, E),
        "lambdas": lam.cpu().numpy().reshape(n_epochs, R.m),
        "final": R.read_chain_state(),
        "hist": R.read_region_hist(),
        "region": R.read_region_params(),
        "image": R.read_image(normalized=True),
        "image_raw": R.read_image(normalized=False),
        "stats": R.read_stats(),
    }
    return out


def oracle_params(p: dict) -> dict:
    keys = ("n_chains", "width", "height", "region_px", "max_depth", "epoch_len", "L", "target_mode",
            "n_bootstrap", "seed", "p_large", "s1", "s2", "alpha_star", "gamma_max", "gamma_scale",
            "lambda_init", "lambda_min", "lambda_max", "w_floor")
    return {k: p[k] for k in keys}
