"""Perforation of the encoding's own reduction (the matmul over features;
the approximation the paper's no-approx hint rules out) through the C ABI,
against the oracle run on the kept features: bit-exact on integer data for
every encoder, within the FP32-accumulation bound on float data, and
consistent with the dimension perforation, the float-query path and the
host entry point."""
import numpy as np
import pytest
import torch

import oracle as orc
from tests._helpers import pack, unpack, words_for

pytestmark = pytest.mark.gpu
ENCS = {"fp32": orc.ENC_FP32, "bf16": orc.ENC_BF16, "fp8": orc.ENC_FP8}


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


@pytest.mark.parametrize("enc,simt", [("fp32", False), ("bf16", False), ("fp8", False), ("fp8", True)])
@pytest.mark.parametrize("fperf,dperf", [((0.0, 0.5, 1), (0.0, 1.0, 1)), ((0.1, 0.9, 3), (0.0, 1.0, 2)),
                                         ((0.0, 1.0, 2), (0.2, 0.8, 1)), ((0.37, 1.0, 1), (0.0, 0.5, 3))])
def test_encoding_perforation_integer_exact(hdc, enc, simt, fperf, dperf):
    rng = np.random.default_rng(int(fperf[2] * 10 + dperf[2]))
    F, D, C, N = 617, 1500, 26, 301
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    cfg = hdc.ApproxConfig(enc=enc, simt=simt, perf_start=dperf[0], perf_end=dperf[1], perf_stride=dperf[2],
                           enc_perf_start=fperf[0], enc_perf_end=fperf[1], enc_perf_stride=fperf[2])
    model = hdc.Model(T(Bt), cfg, acc=T(acc.astype(np.int32)))
    Xk, Btk = orc.perforate_features(X, Bt, *fperf)
    assert model.m.Fk == Xk.shape[1]
    dims = orc.kept_dims(D, *dperf)
    bits, _, _, _ = orc.encode_bits(Xk, Btk, orc.ENC_FP32, dims, integer=True)
    H = hdc.encode(T(X), model)
    assert np.array_equal(H.cpu().numpy().view(np.uint32), pack(bits, words_for(dims.size)))
    lab, dist = hdc.classify(T(X), model, sims=True)
    o_lab, o_dist = orc.classify(Xk, Btk, acc, orc.ENC_FP32, *dperf, 1, integer=True)
    assert np.array_equal(lab.cpu().numpy(), o_lab) and np.array_equal(dist.cpu().numpy().astype(np.int64), o_dist)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
def test_encoding_perforation_float_within_bound(hdc, enc):
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=200, n_query=4, D=1000)
    fperf = (0.05, 0.95, 2)
    X, Bt = d["Xtr"], d["Bt"]
    cfg = hdc.ApproxConfig(enc=enc, enc_perf_start=fperf[0], enc_perf_end=fperf[1], enc_perf_stride=fperf[2])
    model = hdc.Model(T(Bt), cfg)
    H, S = hdc.encode(T(X), model, scores=True)
    Xk, Btk = orc.perforate_features(X, Bt, *fperf)
    Fk = Xk.shape[1]
    dims = orc.kept_dims(1000)
    Xq, sx = orc.quantise_rows(Xk, ENCS[enc])
    Bq, sb = orc.quantise_rows(Btk, ENCS[enc])
    scale = sx[:, None] * sb[None, :]
    sq = orc.encode_f64(Xq, Bq, dims) * scale
    bound = 4 * Fk * 2.0 ** -24 * orc.encode_absdot(Xq, Bq, dims) * scale
    assert np.all(np.abs(S.cpu().numpy().astype(np.float64) - sq) <= bound)
    sure = np.abs(sq) > bound
    assert np.array_equal(unpack(H.cpu().numpy().view(np.uint32), 1000)[sure], (sq < 0)[sure])


def test_encoding_perforation_float_query_and_host(hdc):
    rng = np.random.default_rng(9)
    F, D, C, N = 300, 800, 12, 257
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-200, 201, (C, D)).astype(np.int64)
    fperf = (0.0, 0.7, 2)
    cfg = hdc.ApproxConfig(enc="fp8", class_bits=8, float_query=True, enc_perf_start=fperf[0],
                           enc_perf_end=fperf[1], enc_perf_stride=fperf[2])
    model = hdc.Model(T(Bt), cfg, acc=T(acc.astype(np.int32)))
    lab = hdc.classify(T(X), model).cpu().numpy()
    Xk, Btk = orc.perforate_features(X, Bt, *fperf)
    o_lab, o_sc, _ = orc.classify_float(Xk, Btk, acc, orc.ENC_FP32, 0.0, 1.0, 1, 8, integer=True)
    srt = np.sort(o_sc, axis=1)
    sure = srt[:, -1] - srt[:, -2] > 1e-3
    assert np.array_equal(lab[sure], o_lab[sure])
    # host rows of all F features through hdc_classify_host
    bmodel = hdc.Model(T(Bt), hdc.ApproxConfig(enc="bf16", enc_perf_start=0.2, enc_perf_end=1.0),
                       acc=T(acc.astype(np.int32)))
    want = hdc.classify(T(X), bmodel)
    parts = [torch.from_numpy(X[:100]).pin_memory(), torch.from_numpy(X[100:]).pin_memory()]
    Xd = torch.empty((N, F), dtype=torch.float32, device="cuda")
    ld = torch.empty(N, dtype=torch.int32, device="cuda")
    lh = torch.empty(N, dtype=torch.int32).pin_memory()
    hdc.classify_host(parts, bmodel, Xd, ld, lh, bmodel.workspace(N))
    torch.cuda.synchronize()
    assert torch.equal(lh, want.cpu())
