"""Training over sharded samples through the C ABI (hdc_train_epoch modes 0
and 2, hdc_train_apply): shards trained one after the other on one GPU, their
bundles and deltas summed as the all-reduce would, equal single-process
hdc.train bit for bit (accumulators, class words, update counts), and the
oracle's training of all samples."""
import numpy as np
import pytest
import torch

import oracle as orc
from tests._helpers import pack, unpack

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import build, hdc as h
    build.build()
    h.load()
    orc.build()
    return h


def _samples(N, D, C, flip, seed):
    rng = np.random.default_rng(seed)
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D), dtype=np.float32) < flip).astype(np.uint8)
    return bits, y


def _train_shards(hdc, H, y, D, C, epochs, cuts):
    dev = H.device
    W = hdc.words(D)
    shards = [(H[a:b].contiguous(), y[a:b].contiguous()) for a, b in zip(cuts[:-1], cuts[1:])]
    wss = [hdc.train_workspace(max(h.shape[0], 1), D, C, dev) for h, _ in shards]
    acc = torch.zeros((C, D), dtype=torch.int32, device=dev)
    part = torch.empty_like(acc)
    scratch_cls = torch.empty((C, W), dtype=torch.int32, device=dev)
    for (h, yy), ws in zip(shards, wss):
        hdc.train_epoch(h, yy, D, C, 0, part, scratch_cls, ws=ws)
        acc += part                                   # the all-reduce of the bundles
    cls = torch.empty((C, W), dtype=torch.int32, device=dev)
    hdc.train_apply(acc, cls)
    ups = []
    delta = torch.zeros_like(acc)
    nu = torch.zeros(1, dtype=torch.int32, device=dev)
    for _ in range(epochs):
        delta.zero_()
        n = 0
        cls_before = cls.clone()
        for (h, yy), ws in zip(shards, wss):
            hdc.train_epoch(h, yy, D, C, 2, part, cls, n_updates=nu, ws=ws)
            assert torch.equal(cls, cls_before)       # mode 2 leaves the classes alone
            delta += part                             # the all-reduce of the deltas
            n += int(nu.item())
        hdc.train_apply(acc, cls, delta=delta)
        ups.append(n)
    return acc, cls, ups


@pytest.mark.parametrize("N,D,C,flip,cuts", [(3000, 1000, 7, 0.45, (0, 1400, 3000)),
                                             (5000, 2048, 26, 0.45, (0, 1, 2500, 2500, 5000)),   # 1-row, empty shard
                                             (20000, 10000, 10, 0.497, (0, 9000, 20000))])
def test_sharded_training_equals_single_process(hdc, N, D, C, flip, cuts):
    bits, y = _samples(N, D, C, flip, N + C)
    H = torch.from_numpy(pack(bits).view(np.int32)).cuda()
    yd = torch.from_numpy(y).cuda()
    epochs = 3
    acc1, cls1, ups1 = hdc.train(H, yd, D, C, epochs)
    acc_s, cls_s, ups_s = _train_shards(hdc, H, yd, D, C, epochs, list(cuts))
    assert torch.equal(acc_s, acc1) and torch.equal(cls_s, cls1) and ups_s == ups1
    assert sum(ups1) > 0                              # the epochs did update
    if N <= 5000:
        oacc, oups = orc.train(bits, y, C, epochs)
        assert np.array_equal(acc_s.cpu().numpy().astype(np.int64), oacc) and ups_s == oups
        assert np.array_equal(unpack(cls_s.cpu().numpy().view(np.uint32), D), orc.class_bits(oacc))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


def test_gpu_sharded_train_one_process_equals_train(hdc):
    """dist.gpu_sharded_train with the exchange a no-op (one process) is
    single-process training."""
    from paper_2606_26547_gb300 import dist as hdist
    bits, y = _samples(4000, 1500, 9, 0.45, 3)
    H = torch.from_numpy(pack(bits).view(np.int32)).cuda()
    yd = torch.from_numpy(y).cuda()
    acc, cls, ups = hdist.gpu_sharded_train(H, yd, 1500, 9, 4)
    acc1, cls1, ups1 = hdc.train(H, yd, 1500, 9, 4)
    assert torch.equal(acc, acc1) and torch.equal(cls, cls1) and ups == ups1


def test_train_apply_without_delta_is_binarise(hdc):
    rng = np.random.default_rng(9)
    acc = torch.from_numpy(rng.integers(-3, 3, (5, 333)).astype(np.int32)).cuda()
    cls = torch.full((5, hdc.words(333)), -1, dtype=torch.int32, device="cuda")
    before = acc.clone()
    hdc.train_apply(acc, cls)
    assert torch.equal(acc, before)
    want = pack(orc.class_bits(before.cpu().numpy().astype(np.int64)))
    assert np.array_equal(cls.cpu().numpy().view(np.uint32), want)     # pad bits zero
    delta = torch.from_numpy(rng.integers(-4, 4, (5, 333)).astype(np.int32)).cuda()
    hdc.train_apply(acc, cls, delta=delta)
    assert torch.equal(acc, before + delta)
    want = pack(orc.class_bits((before + delta).cpu().numpy().astype(np.int64)))
    assert np.array_equal(cls.cpu().numpy().view(np.uint32), want)
