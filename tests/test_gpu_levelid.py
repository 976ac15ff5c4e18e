"""Level-ID encoding through the C ABI (hdc_levelid_prepare / encode)
against the oracle: packed hypervectors bit for bit (the quantisation takes
the same FP32 steps, the bundle is an exact count), across feature counts
around the 8-row carry-save groups, level counts, dims around word and
block edges, perforations, out-of-range / NaN / infinite features, and
training + classification on the encoded rows."""
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


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def run(hdc, F, D, L, N, perf, x_lo=-1.5, x_hi=2.0, seed=0, special=False):
    from paper_2606_26547_gb300 import synth
    ids, lo, hi, flip = synth.levelid_hvs(F, D, L, seed)
    rng = np.random.default_rng(seed + 1)
    X = rng.uniform(x_lo - 0.4, x_hi + 0.4, (N, F)).astype(np.float32)
    if special:
        X[0, : min(F, 4)] = [np.nan, np.inf, -np.inf, x_hi][: min(F, 4)]
        X[-1] = x_lo
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2])
    m = hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), L, x_lo, x_hi, cfg)
    H = hdc.levelid_encode(T(X), m)
    dims = orc.kept_dims(D, *perf)
    o_bits, _ = orc.levelid_encode(X, ids, lo, hi, flip, L, x_lo, x_hi, dims)
    got = unpack(H.cpu().numpy().view(np.uint32), len(dims))
    assert np.array_equal(got, o_bits)
    W = H.shape[1]
    full = H.cpu().numpy().view(np.uint32)
    tail = len(dims) % 32
    if tail:   # pad bits of the last kept word are zero
        assert not (full[:, len(dims) // 32] >> tail).any()
    assert not full[:, (len(dims) + 31) // 32:W].any()
    assert int(m.flip_error.item()) == 0
    return m, H, X, ids, lo, hi, flip, dims


@pytest.mark.parametrize("F,D,L,N,perf", [
    (1, 32, 2, 5, (0.0, 1.0, 1)),
    (7, 33, 16, 40, (0.0, 1.0, 1)),
    (8, 1000, 128, 70, (0.0, 0.5, 1)),
    (9, 1024, 3, 33, (0.1, 0.97, 3)),
    (617, 2048, 128, 100, (0.0, 1.0, 1)),
    (617, 10000, 64, 45, (0.0, 1.0, 2)),
    (300, 4096, 1024, 64, (0.25, 1.0, 1)),
    (1023, 700, 2, 31, (0.0, 1.0, 5)),
])
def test_levelid_encode_matches_oracle(hdc, F, D, L, N, perf):
    run(hdc, F, D, L, N, perf, seed=F + D + L, special=True)


def test_levelid_flip_check_and_limits(hdc):
    from paper_2606_26547_gb300 import synth
    ids, lo, hi, flip = synth.levelid_hvs(10, 100, 8, 5)
    flip[7] = 8                                       # outside 1..L-1
    m = hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), 8, 0.0, 1.0)
    torch.cuda.synchronize()
    assert int(m.flip_error.item()) == 1
    with pytest.raises(hdc.HdcError):                 # empty range
        hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), 8, 1.0, 1.0)
    big = synth.levelid_hvs(1200, 64, 600, 6)         # (F + L) * 128 B > 200 KB
    with pytest.raises(hdc.HdcError):
        hdc.LevelIdModel(*(T(a) for a in big), 600, 0.0, 1.0)


def test_levelid_train_and_classify(hdc):
    """Level-ID hypervectors of a labelled mixture, bundled and retrained on
    the GPU, classified by Hamming: all equal to the oracle's."""
    from paper_2606_26547_gb300 import synth
    w = synth.Workload("lid", 120, 2048, 8, 800, 300, "gauss", 1.0, 3, 9100)
    d = synth.make(w)
    ids, lo, hi, flip = synth.levelid_hvs(w.F, w.D, 32, w.seed)
    m = hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), 32, -4.0, 4.0)
    Htr = hdc.levelid_encode(T(d["Xtr"]), m)
    Hq = hdc.levelid_encode(T(d["Xq"]), m)
    acc, cls, ups = hdc.train(Htr, T(d["ytr"]), w.D, w.C, w.epochs)
    lab = hdc.hamming_argmin(Hq, cls, w.D)
    dims = orc.kept_dims(w.D)
    btr, _ = orc.levelid_encode(d["Xtr"], ids, lo, hi, flip, 32, -4.0, 4.0, dims)
    bq, _ = orc.levelid_encode(d["Xq"], ids, lo, hi, flip, 32, -4.0, 4.0, dims)
    o_acc, o_ups = orc.train(btr, d["ytr"], w.C, w.epochs)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), o_acc) and ups == o_ups
    o_lab = orc.argmin(orc.hamming(bq, orc.class_bits(o_acc)))
    assert np.array_equal(lab.cpu().numpy(), o_lab)
    assert (o_lab == d["yq"]).mean() > 0.5
