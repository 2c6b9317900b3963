"""Multi-rank host logic on CPU (gloo, world size 2 and 3): sharding of the
bitstrings, the max-over-ranks timing and the gather of amplitudes."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_1712_05384_gb300 import shard as S


def test_shard_range_partitions():
    for total in (0, 1, 7, 1000, 1024):
        for world in (1, 2, 3, 8):
            got = []
            for r in range(world):
                lo, hi = S.shard_range(total, r, world)
                assert 0 <= hi - lo <= total // world + 1
                got.extend(range(lo, hi))
            assert got == list(range(total))
    with pytest.raises(ValueError):
        S.shard_range(10, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, total, q):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    bits = np.arange(total, dtype=np.uint64)
    mine = S.shard(bits, rank, world)
    # stand-in amplitudes derived from the bitstrings (no GPU here)
    amps = mine.astype(np.float64) + 1j * (mine.astype(np.float64) * 0.5)
    t = S.max_over_ranks(0.1 * (rank + 1), dist)
    allamps = S.gather_amplitudes(amps, total, dist)
    if rank == 0:
        q.put((t, allamps))
    dist.destroy_process_group()


@pytest.mark.parametrize("world,total", [(2, 1024), (3, 1000)])
def test_gloo_sharding_and_gather(world, total):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, total, q)) for r in range(world)]
    for p in procs:
        p.start()
    t, allamps = q.get(timeout=120)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert abs(t - 0.1 * world) < 1e-12
    b = np.arange(total, dtype=np.float64)
    assert np.array_equal(allamps, b + 1j * 0.5 * b)
