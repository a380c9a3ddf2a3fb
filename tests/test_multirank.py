"""The N > 1 path of the bench on CPU: two gloo ranks.  Ranks draw disjoint
sampler streams (weak scaling, no collective on the data path) and the job's
time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2206_14307_gb300 import synth
    local = [10.0 + rank, 20.0 - rank, 5.0 * (rank + 1)]
    got = bench.max_over_ranks(local, device="cpu")
    seeds = [bench.rank_seed(rank, k) for k in range(4)]
    p = synth.random_params(16, 16, 1, std=0.01, seed=1)
    om = oracle.Model(4, 1.0, 0.5, K=1, M=16, params=p)
    chains, _ = om.sample(seeds[0], 4, 8, 2, 4)
    gathered = [None] * world
    dist.all_gather_object(gathered, dict(seeds=seeds, chains=np.asarray(chains).tolist(), maxed=got))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_disjoint_streams_and_max_timing():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0, r1 = res
    assert r0["maxed"] == r1["maxed"] == [11.0, 20.0, 10.0]
    assert not set(r0["seeds"]) & set(r1["seeds"])
    assert r0["chains"] != r1["chains"]
