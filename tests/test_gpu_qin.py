"""The fused classify that quantises its own query tiles.

For binary classes on the tensor cores (up to 32 with the popcount
epilogue, 33..112 with the Hamming distances as a second MMA), hdc_classify
hands the FP32 rows to the fused kernel, which quantises each 128-query tile (BF16 by
round-to-nearest-even, E4M3 after the row's power-of-two scale: Sec. 4.2
"Element Type Representation") one tile ahead of its MMAs, whenever every
CTA has at least two tiles (N >= 2 x SMs x 128) and each tile carries at
least 0.15 * F MMA stages of 128 bytes (dim tiles x K blocks; below that the
separate quantiser pass is faster).  Smaller batches quantise all rows first
in a kernel of their own.  The shapes below (D = 10,000 at stride 2 or 3)
meet the stage rule.  Both routes feed the same
operands to the same MMAs, so labels and Hamming distances must agree bit
for bit: the checks below classify a batch above the threshold once and in
slices below it, compare with the Hamming distances of the hypervectors
hdc_encode produces, and, on integer data (every projection exact), with
the oracle."""
import numpy as np
import pytest
import torch

import oracle as orc
from tests._helpers import unpack

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


def dev():
    return torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def threshold() -> int:
    """Smallest batch on the in-kernel quantisation route: two 128-query
    tiles for each of the SMs' persistent CTAs."""
    return 2 * torch.cuda.get_device_properties(0).multi_processor_count * 128


def sliced(hdc, X, model):
    """The batch classified in slices below the threshold (rows quantised by
    the row-quantiser kernel first)."""
    n = threshold() - 1
    labs, dists = [], []
    for r0 in range(0, X.shape[0], n):
        lab, dist = hdc.classify(X[r0:r0 + n], model, sims=True)
        labs.append(lab)
        dists.append(dist)
    return torch.cat(labs), torch.cat(dists)


def gauss_rows(rng, N, F, octaves=True):
    """N(0, 1) rows, each scaled by 2^k, k uniform in [-30, 30]: the rows'
    power-of-two FP8 scales span 61 octaves."""
    X = rng.standard_normal((N, F)).astype(np.float32)
    if octaves:
        X *= np.exp2(rng.integers(-30, 31, (N, 1))).astype(np.float32)
    return X


@pytest.mark.parametrize("enc", ["fp8", "bf16"])
@pytest.mark.parametrize("C", [10, 26, 48, 112])        # one, two epilogue warpgroups; tensor-core Hamming
@pytest.mark.parametrize("F,extra", [(784, 77), (100, 0), (1024, 1)])
def test_qin_equals_row_quantiser_route(hdc, enc, C, F, extra):
    rng = np.random.default_rng(C * 1000 + F + extra)
    N = threshold() + (3 * 128 + 5 if extra else 0) + extra
    D = 10000
    X = gauss_rows(rng, N, F)
    Bt = rng.standard_normal((D, F)).astype(np.float32)
    acc = rng.integers(-500, 501, (C, D)).astype(np.int32)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc, perf_stride=2), acc=T(acc))
    Xd = T(X)
    lab, dist = hdc.classify(Xd, model, sims=True)
    l_ref, d_ref = sliced(hdc, Xd, model)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    assert torch.equal(lab, l_ref)
    assert torch.equal(dist, d_ref)
    # and the Hamming distances of hdc_encode's hypervectors, on sampled rows
    rows = np.unique(np.concatenate([rng.choice(N, 600, replace=False), [0, 127, 128, N - 129, N - 1]]))
    H = hdc.encode(Xd, model)
    kd = orc.kept_dims(D, 0.0, 1.0, 2)
    qb = unpack(H.cpu().numpy().view(np.uint32)[rows], kd.size)
    od = orc.hamming(qb, orc.gather_cols(orc.class_bits(acc.astype(np.int64)), kd))
    assert np.array_equal(dist.cpu().numpy()[rows].astype(np.int64), od)
    assert np.array_equal(lab.cpu().numpy()[rows], orc.argmin(od))


@pytest.mark.parametrize("enc", ["fp8", "bf16"])
@pytest.mark.parametrize("extra,C", [(0, 10), (1, 10), (128 * 152 + 77, 10), (77, 100)])
def test_qin_integer_data_equals_oracle(hdc, enc, extra, C):
    """Integer features and a +-1 base: every projection is exact in either
    encoding, so every label and distance equals the oracle's (all rows)."""
    from paper_2606_26547_gb300 import synth
    N = threshold() + extra
    F, D = 100, 8000
    X, _ = synth.int_mixture(N, F, C, 2.0, 401, 402)
    rng = np.random.default_rng(403)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc, perf_stride=2), acc=T(acc.astype(np.int32)))
    lab, dist = hdc.classify(T(X), model, sims=True)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    ol, od = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, 2, 1, integer=True, threads=8)
    assert np.array_equal(lab.cpu().numpy(), ol)
    assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)


@pytest.mark.parametrize("enc", ["fp8", "bf16"])
def test_qin_row_scale_edges(hdc, enc):
    """Rows of zeros, subnormal rows, rows far above 448 and rows
    whose maximum sits on either side of 448 * 2^k: the in-kernel scale and
    conversion equal the row quantiser's."""
    rng = np.random.default_rng(7)
    N, F, D, C = threshold() + 300, 128, 10000, 16
    X = gauss_rows(rng, N, F, octaves=False)
    X[0::7] = 0.0
    X[1::7] *= np.float32(2.0 ** -140)                        # subnormal
    X[2::7] *= np.float32(2.0 ** 100)                         # far above 448
    X[3::7, 0] = np.float32(448.0)                            # amax exactly 448 * 2^0
    X[4::7, 0] = np.nextafter(np.float32(448.0), np.float32(1e9))
    X[5::7] = -np.abs(X[5::7])                                # all negative
    Bt = rng.standard_normal((D, F)).astype(np.float32)
    acc = rng.integers(-50, 51, (C, D)).astype(np.int32)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc), acc=T(acc))
    Xd = T(X)
    lab, dist = hdc.classify(Xd, model, sims=True)
    l_ref, d_ref = sliced(hdc, Xd, model)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    assert torch.equal(lab, l_ref) and torch.equal(dist, d_ref)
    # a zero row encodes to all +1 (no set bit): distance = popcount of the class
    cb = orc.class_bits(acc.astype(np.int64))
    assert np.array_equal(dist.cpu().numpy()[0].astype(np.int64), cb.sum(1))


@pytest.mark.parametrize("delta", [-1, 0, 1])
def test_qin_threshold_edges(hdc, delta):
    """Either side of the route boundary, with ragged query tiles."""
    rng = np.random.default_rng(50 + delta)
    N, F, D, C = threshold() + delta, 64, 10000, 5
    X = gauss_rows(rng, N, F)
    Bt = rng.standard_normal((D, F)).astype(np.float32)
    acc = rng.integers(-50, 51, (C, D)).astype(np.int32)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8", perf_stride=3), acc=T(acc))
    Xd = T(X)
    lab, dist = hdc.classify(Xd, model, sims=True)
    n = N // 3 + 1
    ref = [hdc.classify(Xd[r0:r0 + n], model, sims=True) for r0 in range(0, N, n)]
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    assert torch.equal(lab, torch.cat([r[0] for r in ref]))
    assert torch.equal(dist, torch.cat([r[1] for r in ref]))


@pytest.mark.parametrize("enc", ["fp8", "bf16"])
@pytest.mark.parametrize("D", [512, 1536, 2560])
def test_qin_few_dim_tiles(hdc, enc, D):
    """Short rows (F = 8, one K block) and 2, 6 or 10 dim tiles per query
    tile: few MMA stages between consecutive query tiles, so the quantiser
    warps' tile-ahead hand-off is exercised at its tightest."""
    rng = np.random.default_rng(D)
    N, F, C = threshold() + 129, 8, 12
    X = gauss_rows(rng, N, F)
    Bt = rng.standard_normal((D, F)).astype(np.float32)
    acc = rng.integers(-50, 51, (C, D)).astype(np.int32)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc), acc=T(acc))
    Xd = T(X)
    lab, dist = hdc.classify(Xd, model, sims=True)
    l_ref, d_ref = sliced(hdc, Xd, model)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    assert torch.equal(lab, l_ref) and torch.equal(dist, d_ref)
