"""The sharded population on CPU ranks (gloo, world size 2).

A population of C chains is split over ranks by global chain id (Philox keyed
by the global id, every rank drawing the whole bootstrap).  Each epoch every
rank runs its chains, the region statistics the epoch added (i_k, A_k, h_k
and the large-step count as integers; the large-step sums of pi per region as
doubles) are summed over ranks by an all-reduce, and every rank runs the same
epoch boundary (Alg. 1, region update) on the summed tables -- the paper's
threads share i_k and A_k the same way (Sec. 6).  Here each rank runs the CPU
oracle's shard through bench.py's own epoch loop (`step_sharded`), and the
result must equal one unsharded oracle run bit for bit: region tables, lambda,
n, weights, the quadtree and every chain's final state.  The image shares sum
to the unsharded image up to rounding.  The job's time is the maximum over
ranks (bench.reduce_job).
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2402_08273_gb300 import scenes as S

WORLD = 2
CASES = {
    "toy_grid": dict(scene="toy", epochs=12,
                     params=dict(n_chains=32, width=32, height=32, region_px=8, max_depth=0, epoch_len=8,
                                 n_bootstrap=1 << 10, seed=11, p_large=0.25)),
    "toy_weighted": dict(scene="toy", epochs=12,
                         params=dict(n_chains=32, width=32, height=32, region_px=8, max_depth=0, epoch_len=8,
                                     n_bootstrap=1 << 10, seed=12, p_large=0.25, target_mode=1)),
    "toy_quadtree": dict(scene="toy", epochs=12,
                         params=dict(n_chains=32, width=32, height=32, region_px=8, max_depth=0, epoch_len=8,
                                     n_bootstrap=1 << 10, seed=13, p_large=0.25, partition=1, qt_max_leaves=64,
                                     qt_max_depth=4, qt_split=40, qt_refine=512)),
    "cornell": dict(scene="cornell", epochs=3,
                    params=dict(n_chains=8, width=32, height=32, region_px=8, max_depth=3, epoch_len=8,
                                n_bootstrap=1 << 8, seed=14, p_large=0.3)),
}


def _chains(case, **shard):
    import oracle
    c = CASES[case]
    scene = oracle.Scene(toy=S.TOY_DEFAULT) if c["scene"] == "toy" else oracle.Scene(S.cornell_box(), use_bvh=False)
    ch = oracle.Chains(scene, **dict(c["params"], **shard))
    ch._scene_ref = scene
    ch.init()
    return ch


def _snapshot(ch):
    out = {"i": ch.visits.copy(), "A": ch.accsum.copy(), "h": ch.hist.copy(), "lam": ch.lam.copy(),
           "n": ch.n_updates.copy(), "w": ch.weight.copy(), "q": ch.q.copy(), "img": ch.image(),
           "bhat": ch.bhat}
    if ch.params.partition == 1:
        out["tree"] = ch.quadtree()
    return out


def _allreduce_numpy(dist):
    import torch

    def reduce(a: np.ndarray):
        # u64 sums wrap: a signed 64-bit reduction gives the same bits
        t = torch.from_numpy(a.view(np.int64) if a.dtype == np.uint64 else a)
        dist.all_reduce(t)
        a[...] = t.numpy().view(a.dtype)
    return reduce


def _worker(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        res = {}
        for case, c in CASES.items():
            p = bench.shard_params(c["params"], rank, world)
            ch = _chains(case, chain_first=p["chain_first"], chains_total=p["chains_total"],
                         n_chains=p["n_chains"])
            counts, sums = ch.exchange_buffers()
            bench.step_sharded(ch, c["epochs"], counts, sums, _allreduce_numpy(dist))
            res[case] = _snapshot(ch)
        t, _ = bench.reduce_job(dist, world, 1.0 + rank, {"x": 1.0}, "cpu")
        out.put((rank, res, t))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


@pytest.fixture(scope="module")
def shards(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, WORLD, port, q)) for r in range(WORLD)]
    for p in procs:
        p.start()
    got = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    return {rank: (res, t) for rank, res, t in got}


def test_job_time_is_the_maximum_over_ranks(shards):
    assert all(t == float(WORLD) for _, t in shards.values())


@pytest.mark.parametrize("case", list(CASES))
def test_shards_equal_one_population(shards, case):
    one = _chains(case)
    one.run_epochs(CASES[case]["epochs"])
    ref = _snapshot(one)
    C = CASES[case]["params"]["n_chains"]
    per = C // WORLD
    for rank in range(WORLD):
        got = shards[rank][0][case]
        # integer tables and everything computed from them: identical
        for key in ("i", "A", "h", "n"):
            assert np.array_equal(got[key], ref[key]), (case, rank, key)
        assert np.array_equal(got["lam"], ref["lam"]), (case, rank, "lambda")
        assert np.array_equal(got["w"], ref["w"]), (case, rank, "w")
        assert got["bhat"] == ref["bhat"]
        assert np.array_equal(got["q"], ref["q"][rank * per:(rank + 1) * per]), (case, rank, "states")
        if "tree" in ref:
            for a, b in zip(got["tree"], ref["tree"]):
                assert np.array_equal(a, b), (case, rank, "quadtree")
    # the image shares sum to the image (binary64, summed in another order)
    img = sum(shards[r][0][case]["img"] for r in range(WORLD))
    np.testing.assert_allclose(img, ref["img"], rtol=1e-12, atol=1e-12 * max(1.0, float(ref["img"].max())))


def test_quadtree_case_refines(shards):
    """The quadtree case exercises refinement passes driven by the summed counts."""
    child, leaf, depth = shards[0][0]["toy_quadtree"]["tree"]
    assert len(child) > 1


def test_sharding_changes_nothing_but_the_split():
    """A planted mistake on the host side of the exchange (one rank's additions
    dropped) is visible in the tables: the test would catch a reduction that
    is not a sum over ranks."""
    import bench
    c = CASES["toy_grid"]
    shards_ = []
    for rank in range(WORLD):
        p = bench.shard_params(c["params"], rank, WORLD)
        shards_.append(_chains("toy_grid", chain_first=p["chain_first"], chains_total=p["chains_total"],
                               n_chains=p["n_chains"]))
    bufs = [s.exchange_buffers() for s in shards_]
    for _ in range(4):
        for s, (cn, sm) in zip(shards_, bufs):
            s.epoch_mutate(cn, sm)
        # only rank 0's additions reach the update (the planted mistake)
        for s in shards_:
            s.epoch_update(bufs[0][0].copy(), bufs[0][1].copy())
    one = _chains("toy_grid")
    one.run_epochs(4)
    assert not np.array_equal(shards_[0].hist, one.hist)
