"""Helpers that run the CUDA library with the trace instrument (GPU tests only)."""
from __future__ import annotations

import numpy as np

from paper_2402_08273_gb300 import rmlt


def traced_run(scene=None, toy=None, n_epochs=4, stride=1, brute_force_max=0, bvh_width=0, tuning=None,
               wavefront=None, words=False, node_format="auto", **params):
    """Initialise, trace `n_epochs` epochs of every `stride`-th chain, and
    return the trace together with the initial and final state.  `tuning`
    (keyword arguments of Renderer.set_tuning) and `wavefront` (of
    Renderer.set_wavefront, and `leaf_batch` of set_trace_leaf_batch) select
    the execution form."""
    import torch
    R = rmlt.Renderer()
    if toy is not None:
        R.load_toy_integrand(toy)
    else:
        R.load_scene(scene, brute_force_max=brute_force_max, bvh_width=bvh_width, node_format=node_format)
    if tuning:
        R.set_tuning(**tuning)
    if wavefront:
        wavefront = dict(wavefront)
        if "leaf_batch" in wavefront:
            R.set_trace_leaf_batch(wavefront.pop("leaf_batch"))
        R.set_wavefront(**wavefront)
    R.init_chains(**params)
    p = R.params
    init = R.read_chain_state()
    E = p["epoch_len"]
    n_traced = -(-p["n_chains"] // stride)
    rec = torch.zeros(n_epochs * n_traced * E * rmlt.TRACE_DTYPE.itemsize, dtype=torch.uint8,
                      device="cuda")
    lam = torch.zeros(n_epochs * R.m, dtype=torch.float64, device="cuda")
    R.set_trace(rec, lam, stride)
    wbuf = None
    if words:   # every record's proposal words, for replays that adopt proposals
        wbuf = torch.zeros(n_epochs * n_traced * E * R.D, dtype=torch.int32, device="cuda")
        R.set_trace_words(wbuf)
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
    if p.get("partition", 0) == 1:
        out["quadtree"] = R.read_quadtree()
    if wbuf is not None:
        out["words"] = wbuf.cpu().numpy().view(np.uint32).reshape(n_epochs, n_traced, E, R.D)
    return out


def oracle_params(p: dict) -> dict:
    keys = ("n_chains", "width", "height", "region_px", "max_depth", "epoch_len", "L", "target_mode",
            "n_bootstrap", "seed", "p_large", "s1", "s2", "alpha_star", "gamma_max", "gamma_scale",
            "lambda_init", "lambda_min", "lambda_max", "w_floor", "partition", "qt_max_leaves",
            "qt_max_depth", "qt_split", "qt_refine", "kernel", "dir_cells", "p_mala", "mala_tau", "mala_drift_max")
    return {k: p[k] for k in keys}


def replay_full(oracle_mod, gpu, scene_obj, max_adopt=2, **replay_kw):
    """Replay every traced mutation with the oracle (full population)."""
    from oracle.replay import Replay, adopt_initial_states
    p = gpu["params"]
    ch = oracle_mod.Chains(scene_obj, **oracle_params(p))
    ch.init()
    adopted = adopt_initial_states(ch, gpu["init"]["q"], max_adopt)
    rp = Replay(ch, gpu["trace"], gpu["lambdas"], init_f=gpu["init"]["f"], words=gpu.get("words"), **replay_kw)
    rp.run_full(gpu["trace"].shape[0])
    return ch, rp, adopted


def check_counters(ch, gpu, rp, pins: dict | None = None, adopted: int = 0, max_adopted: int = 0):
    """Exact integer state and tolerance-bounded sums after a full replay.

    `pins`: the most mutations each window may let through in this test
    (f_bounded, f_excluded, decision_excluded, update_excluded), pinned at
    the counts measured on a GB300 so that a regression that stays inside the
    windows still fails; missing keys pin 0."""
    print("replay counts:", rp.counts(), "adopted", adopted, "f_max_rel", rp.f_max_rel,
          "a_max_rel", rp.a_max_rel, "bound_use", rp.bound_use)
    assert rp.ok(), rp.summary()
    reg = gpu["region"]
    assert np.array_equal(ch.hist, gpu["hist"]), "h_k differs"
    assert np.array_equal(ch.visits, reg["i"]), "i_k differs"
    assert np.array_equal(ch.n_updates, reg["n"]), "n_k differs"
    assert np.array_equal(ch.lam, reg["lambda"]), "lambda_k differs"
    assert np.array_equal(ch.q, gpu["final"]["q"].T), "final chain states differ"
    # the GPU's A_k is exactly the sum of its own recorded acceptance
    # probabilities; the oracle's differs by at most what the a's differ by
    if rp.stride == 1:
        m = len(reg["A"])
        assert np.array_equal(rp.gpu_accsum()[:m], reg["A"]), "A_k is not the sum of the GPU's own a"
    A_o, A_g = ch.accsum.astype(np.float64), reg["A"].astype(np.float64)
    i_k = reg["i"].astype(np.float64)
    assert np.all(np.abs(A_g - A_o) <= 2.0 ** 32 * i_k * rp.a_max_rel + i_k + 1), "A_k differs"
    raw_o = ch.image_acc
    # each splat is a state's f / pi, and f may differ from the oracle's by up
    # to the replay's largest relative difference (within its binary32
    # bound): a pixel's sum of positive splats then differs by at most twice
    # that (f and its luminance)
    rtol = 2.0 * max(rp.f_max_rel, 5e-6) + 1e-9
    np.testing.assert_allclose(gpu["image_raw"], raw_o, rtol=rtol, atol=1e-7 * max(1.0, raw_o.max()))
    pins = pins or {}
    for key, n in rp.counts().items():
        assert n <= pins.get(key, 0), (key, n, pins.get(key, 0))
    assert adopted <= max_adopted, adopted
