"""Multi-process layout of the path: one process per GPU.

Inference: query rows are independent, so ranks take disjoint shards and
never exchange data; the job's throughput is all rows over the slowest
rank's time (weak scaling: each rank keeps its own batch size).

Training: samples are sharded; bundling and each retraining epoch produce
integer class-accumulator contributions that are summed across ranks with
one all-reduce per epoch.  Retraining is epoch-synchronous (predictions use
the class hypervectors from the start of the epoch), so the sharded result
equals the single-process one exactly: integer sums do not depend on order.

The local compute is passed in (the GPU kernels in production, the CPU
oracle in the host-side tests), so this module holds only the exchange.
"""
from __future__ import annotations

import torch
import torch.distributed as dist


def shard_range(n: int, rank: int, world: int) -> tuple:
    """Contiguous, balanced [lo, hi) of n units for this rank."""
    lo = n * rank // world
    hi = n * (rank + 1) // world
    return lo, hi


def max_over_ranks(seconds: float, device=None) -> float:
    """The slowest rank's elapsed time (the job's wall time)."""
    if not dist.is_available() or not dist.is_initialized() or dist.get_world_size() == 1:
        return seconds
    t = torch.tensor([seconds], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(units_per_rank: int, steps: int, world: int, max_seconds: float) -> float:
    """Units per second of the whole job."""
    return units_per_rank * steps * world / max_seconds


def allreduce_sum_(t: torch.Tensor) -> torch.Tensor:
    """In-place integer sum over ranks (no-op on one process)."""
    if dist.is_available() and dist.is_initialized() and dist.get_world_size() > 1:
        dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return t


def sharded_train(bits_local, y_local, C: int, epochs: int, bundle, retrain_delta, class_bits):
    """Bundling + `epochs` retraining epochs over sharded samples.

    bundle(bits, y, C) -> local int64 accumulator contribution (C x D);
    class_bits(acc) -> the class hypervectors used for prediction;
    retrain_delta(bits, y, cls) -> (local accumulator delta, local updates).
    Returns (global acc, per-epoch global update counts).
    """
    acc = torch.as_tensor(bundle(bits_local, y_local, C)).to(torch.int64).clone()
    allreduce_sum_(acc)
    updates = []
    for _ in range(epochs):
        cls = class_bits(acc)
        delta, n_up = retrain_delta(bits_local, y_local, cls)
        delta = torch.as_tensor(delta).to(torch.int64).clone()
        n = torch.tensor([int(n_up)], dtype=torch.int64)
        allreduce_sum_(delta)
        allreduce_sum_(n)
        acc += delta
        updates.append(int(n.item()))
    return acc, updates
