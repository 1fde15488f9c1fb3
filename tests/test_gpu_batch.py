"""Batched stepping (rmlt_batch_*): several contexts of uneven size advanced by
one chain-kernel launch and one region-update launch per epoch must end
exactly where stepping each context alone ends: chain states, region counts
and parameters, quadtree, statistics bit for bit; images up to the order of
the binary64 atomic splats."""
import numpy as np
import pytest

from paper_2402_08273_gb300 import scenes as S

pytestmark = pytest.mark.gpu


def _members(n=5, seed=3):
    from paper_2402_08273_gb300 import rmlt
    work = S.batch_workload(n, seed=seed, tri_range=(2_000, 30_000), chain_range=(100, 5000))
    if n > 1:
        p = work[1][1]
        p.update(partition=1, qt_max_leaves=256, qt_max_depth=6, qt_split=200, qt_refine=p["n_chains"] * 32)
    if n > 2:
        work[2][1].update(target_mode=1)
    out = []
    for scene, params in work:
        R = rmlt.Renderer()
        R.load_scene(scene)
        R.init_chains(**params)
        out.append(R)
    return out


def _snapshot(R):
    st = R.read_stats()
    snap = {"state": R.read_chain_state(), "hist": R.read_region_hist(), "region": R.read_region_params(),
            "image": R.read_image(normalized=False),
            "stats": {k: st[k] for k in ("mutations", "accepted", "large", "small", "early_reject",
                                         "invalid_paths", "rays", "stack_overflow", "epochs", "n_regions")}}
    if R.params.get("partition", 0) == 1:
        snap["quadtree"] = R.read_quadtree()
    return snap


def _assert_same(a, b):
    for k in ("q", "f", "k"):
        assert np.array_equal(a["state"][k], b["state"][k]), k
    assert np.array_equal(a["hist"], b["hist"])
    for k, v in a["region"].items():
        assert np.array_equal(v, b["region"][k]), k
    assert a["stats"] == b["stats"]
    np.testing.assert_allclose(b["image"], a["image"], rtol=1e-12, atol=1e-300)
    if "quadtree" in a:
        for x, y in zip(a["quadtree"], b["quadtree"]):
            assert np.array_equal(x, y)


@pytest.mark.parametrize("ctas,branches", [(4, False), (3, False), (4, True)])
def test_batch_equals_individual_steps(ctas, branches):
    from paper_2402_08273_gb300 import rmlt
    alone, batched = _members(), _members()
    for R in alone:
        R.step(96)
    batch = rmlt.Batch(batched)
    batch.set_shape(ctas, branches)
    batch.step(48)
    batch.step(48)   # replays the captured graph
    batch.close()
    for a, b in zip(alone, batched):
        _assert_same(_snapshot(a), _snapshot(b))
    assert alone[1].n_regions() > 1   # the quadtree member refined


def test_batch_order_and_interleaving_change_nothing():
    from paper_2402_08273_gb300 import rmlt
    alone, batched = _members(4, seed=7), _members(4, seed=7)
    for R in alone:
        R.step(64)
    batch = rmlt.Batch(batched)
    batch.set_order([3, 1, 0, 2])
    batch.step(32)
    batched[2].step(16)          # a member stepped alone between batch steps
    batch.set_order([0, 1, 2, 3])
    batch.set_shape(4, True)
    batch.step(16)
    for i in (0, 1, 3):
        batched[i].step(16)
    batch.close()
    for a, b in zip(alone, batched):
        _assert_same(_snapshot(a), _snapshot(b))


def test_batch_rejects_unsupported_members():
    from paper_2402_08273_gb300 import rmlt
    ok = _members(2, seed=1)
    cb = rmlt.Renderer()
    cb.load_scene(S.cornell_box())   # brute force
    cb.init_chains(n_chains=64, width=64, height=64, region_px=8, max_depth=5, n_bootstrap=1 << 14)
    with pytest.raises(rmlt.RmltError):
        rmlt.Batch(ok + [cb])
    other = _members(1, seed=2)[0]
    p = dict(other.params)
    p["epoch_len"] = 8
    other.init_chains(**p)
    with pytest.raises(rmlt.RmltError):
        rmlt.Batch(ok + [other])
    ok[0].set_tuning(wavefront=True)
    with pytest.raises(rmlt.RmltError):
        rmlt.Batch(ok)
    ok[0].set_tuning()
    b = rmlt.Batch(ok)
    with pytest.raises(rmlt.RmltError):
        b.set_order([0, 0])
    b.step(16)
    b.close()


# the most mutations each window may let through, measured on a GB300
PINS_REPLAY = {0: {"f_bounded": 1, "f_excluded": 1}, 1: {"f_bounded": 1, "f_excluded": 1}}


def test_batched_members_replayed_by_the_oracle(oracle_mod):
    """Two members of one batched launch (a BVH scene on the grid partition and
    one on the quadtree partition), traced inside the batched kernel and
    replayed mutation by mutation by the oracle: proposals, decisions, region
    tables, lambda after every update, the quadtree and final states."""
    import torch
    from paper_2402_08273_gb300 import rmlt
    from gpu_run import check_counters, oracle_params
    from oracle.replay import Replay, adopt_initial_states
    scenes = [S.two_rooms(20_000, seed=6), S.two_rooms(20_000, seed=7)]
    params = [dict(n_chains=96, width=96, height=96, region_px=16, max_depth=6, n_bootstrap=1 << 12, seed=8),
              dict(n_chains=160, width=64, height=64, region_px=16, max_depth=5, n_bootstrap=1 << 12, seed=9,
                   partition=1, qt_max_leaves=64, qt_max_depth=4, qt_split=150, qt_refine=160 * 16 * 3)]
    n_ep = 12
    Rs, bufs, init = [], [], []
    for scene, p in zip(scenes, params):
        R = rmlt.Renderer()
        R.load_scene(scene)
        R.init_chains(**p)
        E = R.params["epoch_len"]
        rec = torch.zeros(n_ep * p["n_chains"] * E * rmlt.TRACE_DTYPE.itemsize, dtype=torch.uint8, device="cuda")
        lam = torch.zeros(n_ep * R.m, dtype=torch.float64, device="cuda")
        R.set_trace(rec, lam, 1)
        init.append(R.read_chain_state())
        Rs.append(R)
        bufs.append((rec, lam))
    B = rmlt.Batch(Rs)
    B.set_shape(4, False)
    B.step(n_ep * 16)
    torch.cuda.synchronize()
    for i, (R, scene) in enumerate(zip(Rs, scenes)):
        p = R.params
        gpu = {"trace": rmlt.trace_to_numpy(bufs[i][0]).reshape(n_ep, p["n_chains"], p["epoch_len"]),
               "lambdas": bufs[i][1].cpu().numpy().reshape(n_ep, R.m), "init": init[i],
               "final": R.read_chain_state(), "hist": R.read_region_hist(), "region": R.read_region_params(),
               "image_raw": R.read_image(normalized=False)}
        ch = oracle_mod.Chains(oracle_mod.Scene(scene, use_bvh=True), **oracle_params(p))
        ch.init()
        adopted = adopt_initial_states(ch, gpu["init"]["q"], 0)
        rp = Replay(ch, gpu["trace"], gpu["lambdas"], init_f=gpu["init"]["f"])
        rp.run_full(n_ep)
        check_counters(ch, gpu, rp, PINS_REPLAY[i], adopted, 0)
        if p["partition"] == 1:
            for a, b in zip(R.read_quadtree(), ch.quadtree()):
                assert np.array_equal(a, b), "quadtree differs"
            assert R.read_stats()["n_regions"] > 1
    B.close()
