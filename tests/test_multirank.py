"""The N > 1 path of bench.py on CPU ranks (gloo, world size 2).

Every GPU runs an independent chain population (Philox key offset by the
rank, no data-path collective); the job's time is the maximum over ranks and
its counts are summed.  Here each rank runs the CPU oracle on its population
instead of the GPU, and the reduced numbers must equal what two separate
single-process runs give.
"""
import os
import socket

import numpy as np
import torch.multiprocessing as mp

from paper_2402_08273_gb300 import scenes as S

BASE = dict(n_chains=32, width=32, height=32, region_px=8, max_depth=0, epoch_len=8, n_bootstrap=1 << 10,
            seed=11, p_large=0.25)


def _population(rank):
    import oracle
    import bench
    p = bench.population_params(BASE, rank)
    ch = oracle.Chains(oracle.Scene(toy=S.TOY_DEFAULT), **p)
    ch.init()
    ch.run_epochs(20)
    return ch


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ch = _population(rank)
    t_local = 1.0 + rank            # stand-in durations: the max must win
    st = ch.stats()
    t, tot = bench.reduce_job(dist, world, t_local, {"mutations": st["mutations"], "rays": st["rays"]}, "cpu")
    h = torch.tensor(ch.hist.astype(np.int64))
    dist.all_reduce(h)
    if rank == 0:
        out.put((t, tot, h.numpy()))
    dist.barrier()
    dist.destroy_process_group()


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def test_two_rank_populations_reduce_like_separate_runs(oracle_mod):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    t, tot, h = q.get(timeout=300)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    a, b = _population(0), _population(1)
    assert t == 2.0
    assert tot["mutations"] == a.stats()["mutations"] + b.stats()["mutations"]
    assert tot["rays"] == a.stats()["rays"] + b.stats()["rays"]
    assert np.array_equal(h, (a.hist + b.hist).astype(np.int64))
    # the two populations are different chains (different Philox keys)
    assert not np.array_equal(a.q, b.q)
