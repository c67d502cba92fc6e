"""Multi-rank host logic of the replica path, on CPU with gloo (world size 2)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1811_06127_gb300 import replicas


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), WORLD_SIZE=str(world),
                      RANK=str(rank), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, lr = replicas.env_rank()
        seconds = [1.5, 2.5][rank]
        reads = [1000, 1000][rank]
        tput = replicas.job_throughput(reads, seconds)
        mx = replicas.max_over_ranks(float(rank) + 0.25)
        seed = replicas.shard_seed(1811061274, rank)
        counts = torch.arange(rank + 3, dtype=torch.int32)
        gathered = replicas.gather_counts(counts)
        replicas.barrier()
        q.put((rank, w, r, lr, tput, mx, seed,
               None if gathered is None else [g.tolist() for g in gathered]))
    finally:
        dist.destroy_process_group()


def test_gloo_two_ranks():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in procs:
        rank, *rest = q.get(timeout=120)
        out[rank] = rest
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank in (0, 1):
        w, r, lr, tput, mx, seed, gathered = out[rank]
        assert (w, r, lr) == (2, rank, rank)
        assert tput == pytest.approx(2000 / 2.5)      # all reads / slowest rank
        assert mx == pytest.approx(1.25)
    assert out[0][5] != out[1][5] and out[0][5] == 1811061274
    assert out[0][6] == [[0, 1, 2], [0, 1, 2, 3]]     # rank 0 gathers both ranks' counts
    assert out[1][6] is None


def test_shard_range_covers():
    for n in (0, 1, 7, 1000):
        for world in (1, 2, 3, 8):
            parts = [replicas.shard_range(n, world, r) for r in range(world)]
            covered = [i for s, e in parts for i in range(s, e)]
            assert covered == list(range(n))


def test_single_process_defaults():
    assert replicas.max_over_ranks(3.0) == 3.0
    assert replicas.job_throughput(10, 2.0) == 5.0
    assert replicas.gather_counts(torch.tensor([1, 2]))[0].tolist() == [1, 2]

