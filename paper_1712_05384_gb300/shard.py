"""Sharding of a bitstring workload over ranks (one process per GPU).

Amplitudes of different bitstrings are independent (the paper notes the
computation of many amplitudes is embarrassingly parallel across machines),
so N ranks take disjoint contiguous blocks of the bitstrings with no
collective on the data path.  The only collectives are host-side: the
slowest rank's time (max) for throughput, and an optional gather of the
amplitudes to rank 0.
"""
from __future__ import annotations

import numpy as np


def shard_range(total: int, rank: int, world: int):
    """[lo, hi) of rank's contiguous block; blocks differ in size by <= 1."""
    if world < 1 or not 0 <= rank < world or total < 0:
        raise ValueError("bad shard arguments")
    base, extra = divmod(total, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


def shard(bits: np.ndarray, rank: int, world: int) -> np.ndarray:
    lo, hi = shard_range(len(bits), rank, world)
    return bits[lo:hi]


def max_over_ranks(seconds: float, dist) -> float:
    """Slowest rank's time (throughput of the whole job divides by this)."""
    import torch
    t = torch.tensor([seconds], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def gather_amplitudes(local: np.ndarray, total: int, dist) -> np.ndarray:
    """Concatenate every rank's complex amplitudes in rank order (all ranks get them)."""
    import torch
    world = dist.get_world_size()
    sizes = [shard_range(total, r, world) for r in range(world)]
    width = max(hi - lo for lo, hi in sizes)
    buf = torch.zeros(2 * width, dtype=torch.float64)
    buf[:2 * len(local)] = torch.from_numpy(np.stack([local.real, local.imag], 1).reshape(-1))
    parts = [torch.zeros_like(buf) for _ in range(world)]
    dist.all_gather(parts, buf)
    out = []
    for (lo, hi), t in zip(sizes, parts):
        v = t.numpy()[:2 * (hi - lo)]
        out.append(v[0::2] + 1j * v[1::2])
    return np.concatenate(out)
