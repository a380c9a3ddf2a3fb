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


def _raw_sums(h1, h2):
    """The 7 raw FP64 sums of one process's samples, in the order of
    nnqs_lanczos_partial: n, sum Re h1, sum |h1|^2, sum Re(conj h1 h2),
    sum Im h1, sum Im(conj h1 h2), sum |h2|^2."""
    c = np.conj(h1) * h2
    return np.array([len(h1), h1.real.sum(), (np.abs(h1) ** 2).sum(), c.real.sum(), h1.imag.sum(), c.imag.sum(),
                     (np.abs(h2) ** 2).sum()])


def _moments_rank_main(rank, world, port, out):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    import oracle
    from paper_2206_14307_gb300 import nnqs, synth
    p = synth.random_params(16, 16, 1, std=0.2, seed=4)
    om = oracle.Model(4, 1.0, 0.5, K=1, M=16, proj_t=True, proj_p=True, spin_inv=1, params=p)
    # this rank's chains: its own Philox stream (disjoint from the other rank's)
    s, _ = om.sample(bench.rank_seed(rank, 0), 6, 3, 4, 20)
    h1, h2 = om.lanczos_h(s)
    sums = torch.from_numpy(_raw_sums(h1, h2))
    nnqs.allreduce_sums(sums)                     # the exchange step of the distributed Lanczos step
    gathered = [None] * world
    dist.all_gather_object(gathered, dict(s=s.tolist(), h1=h1.tolist(), h2=h2.tolist(), sums=sums.tolist()))
    if rank == 0:
        out.put(gathered)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_allreduced_moments_equal_the_union():
    """Two ranks on disjoint chains: after the all-reduce of the 7 raw sums
    every rank holds the sums of the union of samples, whose moments and p = 1
    energy (Sec. 3.3) equal those of one process holding all samples, to FP64
    rounding."""
    import oracle
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_moments_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = q.get(timeout=300)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    r0, r1 = res
    assert r0["s"] != r1["s"]
    np.testing.assert_array_equal(r0["sums"], r1["sums"])        # every rank holds the same sums
    h1 = np.concatenate([np.asarray(r["h1"]) for r in res])
    h2 = np.concatenate([np.asarray(r["h2"]) for r in res])
    union = oracle.moments(h1, h2)
    sums = np.asarray(r0["sums"])
    assert sums[0] == len(h1)
    m = np.array([1.0, sums[1] / sums[0], sums[2] / sums[0], sums[3] / sums[0]])
    np.testing.assert_allclose(m, union["m"], rtol=1e-13)
    np.testing.assert_allclose(sums[6] / sums[0], union["m4"], rtol=1e-13)
    e_dist = oracle.lanczos_step(m)["E"]
    e_union = oracle.lanczos_step(union["m"])["E"]
    assert abs(e_dist - e_union) <= 1e-11 * abs(e_union)
