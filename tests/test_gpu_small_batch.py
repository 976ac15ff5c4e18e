"""Fused classify of batches with fewer 128-query tiles than SMs.

Such a batch splits each query tile's dim tiles over several CTAs (as many
as fill the SMs, each range non-empty); every CTA adds its partial Hamming
distances into a zero-filled scratch and the warp whose contribution
completes a tile takes the arg-min over all classes.  On integer features
with a +-1 base every projection is exact, so labels and distances must
equal the oracle's for every row, for every split count the batch size and
dimensionality produce, for one, two and four epilogue warpgroups, and with
ties that the lowest class index must win."""
import numpy as np
import pytest
import torch

import oracle as orc

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


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda:0"))


def sms() -> int:
    return torch.cuda.get_device_properties(0).multi_processor_count


def case(hdc, N, C, D, stride, enc, seed, acc=None):
    rng = np.random.default_rng(seed)
    F = 96
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    if acc is None:
        acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc, perf_stride=stride), acc=T(acc.astype(np.int32)))
    lab, dist = hdc.classify(T(X), model, sims=True)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    ol, od = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, stride, 1, integer=True, threads=8)
    assert np.array_equal(lab.cpu().numpy(), ol)
    assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)


@pytest.mark.parametrize("N", [1, 127, 128, 129, 300, 1000, 4173])
@pytest.mark.parametrize("C", [5, 26, 120])      # one, two and four epilogue warpgroups
def test_split_ranges_equal_oracle(hdc, N, C):
    """40 dim tiles (D' = 10,000) split 40, 40, 40, 40, 20, 20 and 5 ways."""
    case(hdc, N, C, 10000, 1, "fp8", N * 7 + C)


@pytest.mark.parametrize("D,stride", [(1000, 1), (2600, 2), (700, 3), (33, 1)])
@pytest.mark.parametrize("enc", ["fp8", "bf16"])
def test_split_dim_tile_counts(hdc, D, stride, enc):
    """Four, six, one and one dim tiles (ragged last tiles), BF16 and FP8."""
    case(hdc, 777, 11, D, stride, enc, D + stride)


def test_split_just_below_one_tile_per_sm(hdc):
    """sms - 1 query tiles: each tile's dim tiles in at most one range."""
    case(hdc, (sms() - 1) * 128 - 5, 7, 2048, 1, "fp8", 3)


def test_split_ties_take_lowest_class(hdc):
    """Equal class hypervectors spread over the class range: the distances
    of equal classes are equal after every range's contribution, and the
    lowest index among the nearest wins."""
    rng = np.random.default_rng(12)
    base = rng.integers(-50, 51, (3, 5000)).astype(np.int64)
    acc = base[rng.integers(0, 3, 30)]
    acc[-1] = base[0]
    case(hdc, 640, 30, 5000, 1, "fp8", 13, acc=acc)


def test_split_scratch_reused_across_calls(hdc):
    """Back-to-back calls with the same workspace (the scratch is zero-filled
    per call) and a larger batch in between."""
    rng = np.random.default_rng(21)
    F, D, C = 96, 4000, 9
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8"), acc=T(acc.astype(np.int32)))
    ws = model.workspace(4096)
    for N in (300, 4096, 300):
        X = rng.integers(-8, 8, (N, F)).astype(np.float32)
        lab, dist = hdc.classify(T(X), model, sims=True, ws=ws)
        torch.cuda.synchronize()
        ol, od = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, 1, integer=True, threads=8)
        assert np.array_equal(lab.cpu().numpy(), ol)
        assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)
    assert hdc.stream_status() == 0
