"""World-size-2 gloo runs (CPU) of the multi-process logic: query sharding,
max-over-ranks timing, and sharded training whose accumulators equal the
single-process oracle's exactly."""
import os
import socket

import numpy as np
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2606_26547_gb300 import dist as hdist


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _data():
    rng = np.random.default_rng(21)
    C, D, N = 5, 200, 301
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = (np.arange(N) % C).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D)) < 0.35).astype(np.uint8)
    return bits, y, C


def _worker(rank, world, port, q):
    import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bits, y, C = _data()
        lo, hi = hdist.shard_range(len(y), rank, world)

        def retrain_delta(b, yy, cls):
            # this rank's perceptron delta: predict with the start-of-epoch
            # classes, +h to the true class and -h to the predicted one
            pred = orc.argmin(orc.hamming(b, cls))
            wrong = pred != yy
            h = 1 - 2 * b.astype(np.int64)
            delta = np.zeros((C, b.shape[1]), np.int64)
            np.add.at(delta, yy[wrong], h[wrong])
            np.subtract.at(delta, pred[wrong], h[wrong])
            return delta, int(wrong.sum())

        acc, ups = hdist.sharded_train(bits[lo:hi], y[lo:hi], C, 3, orc.bundle, retrain_delta,
                                       lambda a: orc.class_bits(a.numpy()))
        t = hdist.max_over_ranks(0.5 + rank)
        q.put((rank, acc.numpy(), ups, t, (lo, hi)))
    finally:
        dist.destroy_process_group()


def test_sharded_training_and_timing_world2():
    import oracle as orc
    orc.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    out.sort()
    bits, y, C = _data()
    ref_acc, ref_ups = orc.train(bits, y, C, 3)
    for rank, acc, ups, t, (lo, hi) in out:
        assert np.array_equal(acc, ref_acc)          # sharded == single process, exactly
        assert ups == ref_ups
        assert t == 1.5                              # the slowest rank's time
    assert out[0][4] == (0, 150) and out[1][4] == (150, 301)


def test_shard_range_covers_everything():
    for n in (0, 1, 7, 1000, 1 << 20):
        for w in (1, 2, 3, 8):
            parts = [hdist.shard_range(n, r, w) for r in range(w)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            assert all(parts[i][1] == parts[i + 1][0] for i in range(w - 1))
            assert max(h - l for l, h in parts) - min(h - l for l, h in parts) <= 1
    assert hdist.job_throughput(100, 10, 4, 2.0) == 2000.0
