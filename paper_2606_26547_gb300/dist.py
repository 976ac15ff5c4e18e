"""Multi-process layout of the path: one process per GPU.

Inference: query rows are independent, so ranks take disjoint shards and
never exchange data; the job's throughput is all rows over the slowest
rank's time (weak scaling: each rank keeps its own batch size).

Training: samples are sharded; bundling and each retraining epoch produce
integer class-accumulator contributions that are summed across ranks with
one all-reduce per epoch.  Retraining is epoch-synchronous (predictions use
the class hypervectors from the start of the epoch), so the sharded result
equals the single-process one exactly: integer sums do not depend on order.

`sharded_train` takes the local compute as callables (the CPU oracle in the
host-side tests); `gpu_sharded_train` is the same schedule on the library's
kernels: hdc_train_epoch mode 0 (a shard's bundle) and mode 2 (a shard's
retraining delta against the shared start-of-epoch classes), an int32
all-reduce of each, and hdc_train_apply (add the summed delta, re-binarise).
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


def gpu_sharded_train(H_local: torch.Tensor, y_local: torch.Tensor, D: int, C: int, epochs: int,
                      stream=None, exchange=allreduce_sum_):
    """Bundling + `epochs` retraining epochs of this rank's packed samples
    (H_local: n x W(D) int32 words, y_local: n int32) on the GPU kernels,
    with one integer all-reduce (`exchange`, in place, over device tensors)
    of the bundle and of every epoch's delta.  Every rank ends with the same
    acc (C x D int32) and class words (C x W(D)), equal to single-process
    training on all samples; returns (acc, cls, per-epoch update counts)."""
    from . import hdc
    dev = H_local.device
    acc = torch.empty((C, D), dtype=torch.int32, device=dev)
    cls = torch.empty((C, hdc.words(D)), dtype=torch.int32, device=dev)
    ws = hdc.train_workspace(max(H_local.shape[0], 1), D, C, dev)
    hdc.train_epoch(H_local, y_local, D, C, 0, acc, cls, ws=ws, stream=stream)
    exchange(acc)
    hdc.train_apply(acc, cls, stream=stream)
    delta = torch.empty_like(acc)
    nu = torch.zeros(1, dtype=torch.int32, device=dev)
    ups = []
    for _ in range(epochs):
        hdc.train_epoch(H_local, y_local, D, C, 2, delta, cls, n_updates=nu, ws=ws, stream=stream)
        exchange(delta)
        exchange(nu)
        hdc.train_apply(acc, cls, delta=delta, stream=stream)
        ups.append(int(nu.item()))
    return acc, cls, ups
