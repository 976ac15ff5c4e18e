"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Integer and binary results (packed hypervectors, Hamming distances, labels,
class accumulators, cosine scores of b-bit classes) must match bit for bit.
Float encodings are compared with the bound derived from FP32 accumulation:
|s_gpu - s_q| <= 4*F*2^-24 * sum_f |xq_f * bq_f|, where s_q is the FP64
projection of the same quantised inputs; packed bits must agree wherever the
oracle's |s_q| exceeds that bound.
"""
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


def dev():
    return torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(dev())


def words_np(t):
    return t.cpu().numpy().view(np.uint32)


def _model_bytes(model, ptr, nbytes):
    off = ptr - model.buf.data_ptr()
    return model.buf[off:off + nbytes].cpu().numpy()


def decode_bq(model, enc):
    m = model.m
    es = {"fp32": 4, "bf16": 2, "fp8": 1}[enc]
    raw = _model_bytes(model, m.Bq, m.Dk * m.ldb * es)
    t = torch.from_numpy(raw.copy())
    if enc == "fp32":
        v = t.view(torch.float32)
    elif enc == "bf16":
        v = t.view(torch.bfloat16)
    else:
        v = t.view(torch.float8_e4m3fn)
    return v.to(torch.float64).numpy().reshape(m.Dk, m.ldb)


# ------------------------------------------------------------------ quantise

@pytest.mark.parametrize("enc", ["bf16", "fp8", "fp32"])
@pytest.mark.parametrize("F", [617, 616])   # unaligned rows / 16-byte rows (streaming path)
def test_base_quantisation_bit_exact(hdc, enc, F):
    rng = np.random.default_rng(1)
    D = 700
    Bt = (rng.standard_normal((D, F)) * 10.0 ** rng.uniform(-3, 3, (D, 1))).astype(np.float32)
    Bt[5] = 0.0
    Bt[9] = (rng.standard_normal(F) * 1e-41).astype(np.float32)   # subnormal row: scale 2^k, k < -126
    Bt[11, 3] = 3.0e38                                               # huge entry
    cfg = hdc.ApproxConfig(enc=enc, perf_start=0.0, perf_end=1.0, perf_stride=3)
    model = hdc.Model(T(Bt), cfg)
    dims = orc.kept_dims(D, 0.0, 1.0, 3)
    q, sc = orc.quantise_rows(Bt[dims], ENCS[enc])
    got = decode_bq(model, enc)
    assert model.m.Dk == dims.size
    assert np.array_equal(got[:, :F], q)
    assert not got[:, F:].any()
    if enc == "fp8":
        gs = np.frombuffer(_model_bytes(model, model.m.b_scale, 4 * dims.size).tobytes(), dtype=np.float32)
        assert np.array_equal(gs.astype(np.float64), sc)


# -------------------------------------------------------------------- encode

def _int_data(n, D=2048):
    from paper_2606_26547_gb300 import synth
    return synth.make("int_exact_F617_D2048_C26", n_train=n, n_query=8, D=D)


@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("simt", [False, True])
@pytest.mark.parametrize("perf", [(0.0, 1.0, 1), (0.0, 0.5, 1), (0.1, 0.97, 3)])
def test_encode_integer_bit_exact(hdc, enc, simt, perf):
    d = _int_data(300)
    X, Bt = d["Xtr"], d["Bt"]
    cfg = hdc.ApproxConfig(enc=enc, perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2], simt=simt)
    model = hdc.Model(T(Bt), cfg)
    H, S = hdc.encode(T(X), model, scores=True)
    dims = orc.kept_dims(2048, *perf)
    bits, s, _, _ = orc.encode_bits(X, Bt, orc.ENC_FP32, dims, integer=True)
    assert np.array_equal(words_np(H), pack(bits, words_for(dims.size)))
    assert np.array_equal(S.cpu().numpy().astype(np.float64), s.astype(np.float64))


@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("simt", [False, True])
def test_encode_float_within_bound(hdc, enc, simt):
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=300, n_query=4, D=1000)
    X, Bt = d["Xtr"], d["Bt"]
    cfg = hdc.ApproxConfig(enc=enc, simt=simt)
    model = hdc.Model(T(Bt), cfg)
    H, S = hdc.encode(T(X), model, scores=True)
    dims = orc.kept_dims(1000)
    Xq, sx = orc.quantise_rows(X, ENCS[enc])
    Bq, sb = orc.quantise_rows(Bt, ENCS[enc])
    scale = sx[:, None] * sb[None, :]
    sq = orc.encode_f64(Xq, Bq, dims) * scale
    bound = 4 * 784 * 2.0 ** -24 * orc.encode_absdot(Xq, Bq, dims) * scale
    err = np.abs(S.cpu().numpy().astype(np.float64) - sq)
    assert np.all(err <= bound), float((err / np.maximum(bound, 1e-300)).max())
    gb = unpack(words_np(H), 1000)
    sure = np.abs(sq) > bound
    assert np.array_equal(gb[sure], (sq < 0)[sure])
    assert not unpack(words_np(H), words_for(1000) * 32)[:, 1000:].any()   # pad bits zero


# ------------------------------------------------------------ Hamming arg-min

@pytest.mark.parametrize("N,C,D", [(1, 1, 32), (300, 26, 2048), (257, 7, 1000), (129, 100, 16384), (50, 3, 33)])
@pytest.mark.parametrize("perf", [None, (0.0, 0.5, 1), (0.05, 0.95, 4), (0.0, 1.0, 8)])
def test_hamming_argmin_bit_exact(hdc, N, C, D, perf):
    rng = np.random.default_rng(N * 7 + C)
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    if C > 2:
        c[2] = c[1]                      # a guaranteed tie: lowest index wins
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2]) if perf else None
    if perf and orc.kept_dims(D, *perf).size == 0:
        pytest.skip("empty perforation")
    labels, dd = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D, cfg, dists=True)
    dims = orc.kept_dims(D, *perf) if perf else orc.kept_dims(D)
    od = orc.hamming(orc.gather_cols(q, dims), orc.gather_cols(c, dims))
    assert np.array_equal(dd.cpu().numpy().astype(np.int64), od)
    assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))


@pytest.mark.parametrize("C", [17, 33, 64, 100, 128, 200, 256, 257])
@pytest.mark.parametrize("D,perf", [(1000, None), (4096, (0.1, 0.9, 3)), (96, None), (2050, (0.0, 1.0, 2))])
def test_hamming_argmin_tensor_core_range(hdc, C, D, perf):
    """33..256 binary classes run as a tensor-core product of the rows
    expanded to +-1 (17..32 and 257 on the popcount paths): distances and
    labels equal the oracle's per-dim definition, with ties across the two
    epilogue warpgroups' class chunks and exact matches."""
    rng = np.random.default_rng(C * 31 + D)
    N = 300
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[C - 1] = c[0]                      # ties: classes in different 32-class chunks
    c[C // 2] = c[1]
    q[:5] = c[:5]                        # distance 0
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2]) if perf else None
    labels, dd = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D, cfg, dists=True)
    dims = orc.kept_dims(D, *perf) if perf else orc.kept_dims(D)
    od = orc.hamming(orc.gather_cols(q, dims), orc.gather_cols(c, dims))
    assert np.array_equal(dd.cpu().numpy().astype(np.int64), od)
    assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))


@pytest.mark.parametrize("N", [1, 127, 129])
@pytest.mark.parametrize("C", [32, 33, 48, 112, 113])
def test_hamming_argmin_class_count_edges(hdc, N, C):
    """Partial and single-row tiles at the class counts where the routes and
    the 16-class padding change (32 / 33, 112 / 113)."""
    rng = np.random.default_rng(N * 1000 + C)
    D = 700
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[C - 1] = c[0]
    labels, dd = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D, dists=True)
    od = orc.hamming(q, c)
    assert np.array_equal(dd.cpu().numpy().astype(np.int64), od)
    assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))


@pytest.mark.parametrize("N", [233471, 240037])   # either side of twelve 128-row blocks per SM on 152 SMs
@pytest.mark.parametrize("C", [10, 32, 257])
def test_hamming_argmin_popcount_batch_sizes(hdc, N, C):
    """The popcount kernel with one and with four threads per query (short
    batches split each row's words): distances and labels, the 257-class
    case on a sample of rows."""
    rng = np.random.default_rng(N + C)
    D = 96
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[2] = c[1]
    labels, dd = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D, dists=True)
    rows = np.arange(N) if C <= 32 else np.unique(np.r_[rng.integers(0, N, 3000), 0, N - 1])
    od = orc.hamming(q[rows], c)
    assert np.array_equal(dd.cpu().numpy()[rows].astype(np.int64), od)
    assert np.array_equal(labels.cpu().numpy()[rows], orc.argmin(od))


def test_hamming_argmin_tensor_core_many_tiles(hdc):
    """More 128-row tiles than SMs (the persistent loop), labels only."""
    rng = np.random.default_rng(11)
    N, C, D = 20000, 40, 512
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N)
    q = c[y] ^ (rng.random((N, D)) < 0.3).astype(np.uint8)
    labels = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D)
    od = orc.hamming(q, c)
    assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))


@pytest.mark.parametrize("C,D,perf", [(100, 1000, None), (200, 2048, (0.1, 0.9, 3)), (40, 4096, None), (26, 1024, None)])
def test_hamming_argmin_workspace_form_and_plain_form(hdc, C, D, perf):
    """hdc_hamming_argmin_ws (the classes expanded once into the caller's
    workspace, reused across calls) and hdc_hamming_argmin (expanded per
    tile) both give the oracle's distances and labels; 26 classes need no
    workspace."""
    rng = np.random.default_rng(C * 7 + D)
    N = 3000
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[C - 1] = c[1]
    q[:3] = c[:3]
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2]) if perf else None
    Qt, Ct = T(pack(q).view(np.int32)), T(pack(c).view(np.int32))
    dims = orc.kept_dims(D, *perf) if perf else orc.kept_dims(D)
    od = orc.hamming(orc.gather_cols(q, dims), orc.gather_cols(c, dims))
    ws = hdc.hamming_workspace(C, D, Qt.device)
    assert (ws is None) == (C <= 32)
    outs = [hdc.hamming_argmin(Qt, Ct, D, cfg, dists=True, ws=ws) for _ in range(2)]
    outs.append(hdc.hamming_argmin(Qt, Ct, D, cfg, dists=True, use_ws=False))
    for labels, dd in outs:
        assert np.array_equal(dd.cpu().numpy().astype(np.int64), od)
        assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("D,C,perf", [(131072, 256, None), (131072, 40, (0.02, 0.99, 5)), (131073, 256, None)])
def test_hamming_argmin_largest_rows(hdc, D, C, perf):
    """The tensor-core route's largest rows (4,096 words: the whole kept-dim
    mask in shared memory), with 256 classes (one CTA per SM, all 512 TMEM
    columns) and 40 (two CTAs), and one dim past it (4,100 words: the
    popcount route, which needs no workspace); two 128-row tiles, the second
    ragged.  Rows 0-2, 64 and 127-129 against the oracle."""
    rng = np.random.default_rng(D + C)
    N = 130
    q = rng.integers(0, 2, (N, D)).astype(np.uint8)
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[C - 1] = c[0]
    q[:2] = c[:2]
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2]) if perf else None
    assert (hdc.hamming_workspace(C, D, torch.device("cuda:0")) is None) == (D > 131072)
    Qt, Ct = T(pack(q).view(np.int32)), T(pack(c).view(np.int32))
    rows = np.array([0, 1, 2, 64, 127, 128, 129])
    dims = orc.kept_dims(D, *perf) if perf else orc.kept_dims(D)
    od = orc.hamming(orc.gather_cols(q[rows], dims), orc.gather_cols(c, dims))
    for use_ws in (True, False):
        labels, dd = hdc.hamming_argmin(Qt, Ct, D, cfg, dists=True, use_ws=use_ws)
        assert np.array_equal(dd.cpu().numpy()[rows].astype(np.int64), od)
        assert np.array_equal(labels.cpu().numpy()[rows], orc.argmin(od))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("N,C,perf", [(41000, 100, None), (40077, 128, (0.1, 0.9, 3))])
def test_hamming_argmin_tensor_core_more_tiles_than_ctas(hdc, N, C, perf):
    """More 128-row tiles than the two CTAs per SM hold, so CTAs take several
    and the query words stream through the copy ring across m-tiles; a ragged
    last tile, 100 and 128 classes, with and without perforation."""
    rng = np.random.default_rng(N + C)
    D = 1024
    c = rng.integers(0, 2, (C, D)).astype(np.uint8)
    c[C - 1] = c[3]
    y = rng.integers(0, C, N)
    q = c[y] ^ (rng.random((N, D)) < 0.4).astype(np.uint8)
    cfg = hdc.ApproxConfig(perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2]) if perf else None
    labels, dd = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), D, cfg, dists=True)
    dims = orc.kept_dims(D, *perf) if perf else orc.kept_dims(D)
    od = orc.hamming(orc.gather_cols(q, dims), orc.gather_cols(c, dims))
    assert np.array_equal(dd.cpu().numpy().astype(np.int64), od)
    assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))


@pytest.mark.parametrize("N,D,C", [(40000, 1024, 120), (39000, 1000, 33)])
def test_train_tensor_route_many_tiles_bit_exact(hdc, N, D, C):
    """Retraining whose predictions run on the tensor-core route with the
    classes expanded once: more 256-row tiles than SMs (CTAs take several,
    the class-atom ring running on across them), a ragged last tile, 128 and
    48 padded classes, and D = 1000 (a masked last word).  Accumulators and
    update counts equal the oracle's."""
    rng = np.random.default_rng(N + C)
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D)) < 0.46).astype(np.uint8)
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), D, C, epochs=1)
    oacc, oups = orc.train(bits, y, C, 1)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc)
    assert ups == oups and oups[0] > 0


def test_train_many_classes_bit_exact(hdc):
    """Retraining with 100 classes: its predictions run on the tensor-core
    Hamming kernel; accumulators and update counts equal the oracle's."""
    rng = np.random.default_rng(100)
    N, D, C = 1500, 2048, 100
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D)) < 0.45).astype(np.uint8)
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), D, C, epochs=3)
    oacc, oups = orc.train(bits, y, C, 3)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc)
    assert ups == oups


@pytest.mark.parametrize("N,D,C", [(3000, 256, 3),      # ~1,000 samples a class: several counting items per group
                                   (2400, 128, 600),    # retraining: 1,200 groups, offsets read from device memory
                                   (2000, 64, 7000)])   # retraining: 14,000 groups, histogram in device memory
def test_train_group_layouts_bit_exact(hdc, N, D, C):
    """Bundling and retraining epochs across the grouping layouts: multi-chunk
    groups, more groups than the counting kernel stages, more than the
    histogram kernel counts in shared memory."""
    rng = np.random.default_rng(N + C)
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D)) < 0.45).astype(np.uint8)
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), D, C, epochs=2)
    oacc, oups = orc.train(bits, y, C, 2)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc)
    assert ups == oups
    assert min(oups) > 0


@pytest.mark.parametrize("fill", [1, 0])
def test_train_saturated_chunks_bit_exact(hdc, fill):
    """Every row of a class identical (all bits set, or none): a 252-sample
    counting chunk reaches the largest per-dim count (16 carries of the
    carry-save tree less one, plus a full residue: 252), and a class of 520
    samples spans two full chunks and a partial one."""
    rng = np.random.default_rng(520 + fill)
    N, D, C = 600, 64, 2
    y = np.r_[np.zeros(520, np.int32), np.ones(80, np.int32)]
    rng.shuffle(y)
    bits = rng.integers(0, 2, (N, D)).astype(np.uint8)
    bits[y == 0] = fill
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), D, C, epochs=2)
    oacc, oups = orc.train(bits, y, C, 2)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc)
    assert ups == oups


def test_hamming_all_ties(hdc):
    q = np.zeros((40, 64), np.uint8)
    c = np.ones((5, 64), np.uint8)
    labels = hdc.hamming_argmin(T(pack(q).view(np.int32)), T(pack(c).view(np.int32)), 64)
    assert not labels.cpu().numpy().any()


# -------------------------------------------------------------------- train

@pytest.mark.parametrize("N,D,C", [(500, 2048, 26), (333, 1000, 10), (1, 64, 1), (700, 10000, 6)])
def test_train_bit_exact(hdc, N, D, C):
    rng = np.random.default_rng(D + C)
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    bits = protos[y] ^ (rng.random((N, D)) < 0.4).astype(np.uint8)
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), D, C, epochs=4)
    oacc, oups = orc.train(bits, y, C, 4)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc)
    assert ups == oups
    assert np.array_equal(words_np(cls), pack(orc.class_bits(oacc)))


def test_train_skips_out_of_range_labels(hdc):
    rng = np.random.default_rng(3)
    bits = rng.integers(0, 2, (64, 96)).astype(np.uint8)
    y = rng.integers(-1, 5, 64).astype(np.int32)            # -1 and 4 are skipped with C = 4
    acc, cls, ups = hdc.train(T(pack(bits).view(np.int32)), T(y), 96, 4, epochs=1)
    keep = (y >= 0) & (y < 4)
    oacc, oups = orc.train(bits[keep], y[keep], 4, 1)
    assert np.array_equal(acc.cpu().numpy().astype(np.int64), oacc) and ups == oups


# ----------------------------------------------------------------- classify

@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("bits_", [1, 4, 8])
@pytest.mark.parametrize("perf", [(0.0, 1.0, 1), (0.0, 0.5, 1), (0.0, 1.0, 2)])
def test_classify_integer_end_to_end(hdc, enc, bits_, perf):
    d = _int_data(600)
    dims_full = orc.kept_dims(2048)
    tb, _, _, _ = orc.encode_bits(d["Xtr"], d["Bt"], orc.ENC_FP32, dims_full, integer=True)
    oacc, _ = orc.train(tb, d["ytr"], 26, 2)
    from paper_2606_26547_gb300 import synth
    Xq, _ = synth.int_mixture(333, 617, 26, 2.0, 77, 1000)
    cfg = hdc.ApproxConfig(enc=enc, class_bits=bits_, perf_start=perf[0], perf_end=perf[1], perf_stride=perf[2])
    model = hdc.Model(T(d["Bt"]), cfg, acc=T(oacc.astype(np.int32)))
    labels, sims = hdc.classify(T(Xq), model, sims=True)
    ol, osim = orc.classify(Xq, d["Bt"], oacc, orc.ENC_FP32, *perf, bits_, integer=True)
    assert np.array_equal(labels.cpu().numpy(), ol)
    if bits_ == 1:
        assert np.array_equal(sims.cpu().numpy().astype(np.int64), osim)
    else:
        assert np.array_equal(sims.cpu().numpy(), osim)      # IEEE FP64 on both sides


@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
@pytest.mark.parametrize("bits_", [1, 8])
def test_classify_float_consistent_with_encode(hdc, enc, bits_):
    """Float encodings: the fused classify equals Hamming/cosine of the
    hypervectors hdc_encode produces with the same model, and those agree
    with the FP64 oracle wherever the projection's sign is certain."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=400, n_query=300, D=1000)
    dims = orc.kept_dims(1000)
    tb, _, _, _ = orc.encode_bits(d["Xtr"], d["Bt"], orc.ENC_FP32, dims)
    oacc, _ = orc.train(tb, d["ytr"], 10, 2)
    cfg = hdc.ApproxConfig(enc=enc, class_bits=bits_, perf_stride=2)
    model = hdc.Model(T(d["Bt"]), cfg, acc=T(oacc.astype(np.int32)))
    labels, sims = hdc.classify(T(d["Xq"]), model, sims=True)
    H = hdc.encode(T(d["Xq"]), model)
    kd = orc.kept_dims(1000, 0.0, 1.0, 2)
    qb = unpack(words_np(H), kd.size)
    if bits_ == 1:
        od = orc.hamming(qb, orc.gather_cols(orc.class_bits(oacc), kd))
        assert np.array_equal(sims.cpu().numpy().astype(np.int64), od)
        assert np.array_equal(labels.cpu().numpy(), orc.argmin(od))
    else:
        sc = orc.cosine_scores(qb, orc.gather_cols(orc.class_quantise(oacc, bits_), kd))
        assert np.array_equal(sims.cpu().numpy(), sc)
        assert np.array_equal(labels.cpu().numpy(), orc.argmax(sc))
    ol, _ = orc.classify(d["Xq"], d["Bt"], oacc, ENCS[enc], 0.0, 1.0, 2, bits_)
    agree = (labels.cpu().numpy() == ol).mean()
    assert agree >= 0.99, agree


def test_classify_edge_cases(hdc):
    rng = np.random.default_rng(5)
    F, D = 33, 100
    Bt = rng.standard_normal((D, F)).astype(np.float32)
    acc = np.zeros((1, D), np.int32)                       # C = 1, all classes +1
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="bf16"), acc=T(acc))
    lab = hdc.classify(T(np.zeros((1, F), np.float32)), model)
    assert lab.cpu().numpy().tolist() == [0]
    lab0 = hdc.classify(torch.empty((0, F), dtype=torch.float32, device=dev()), model)
    assert lab0.numel() == 0
    H = hdc.encode(T(np.zeros((3, F), np.float32)), model)   # x = 0 -> all +1 -> all bits 0
    assert not words_np(H).any()
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


# ------------------------------------------- tensor-core path specifics

@pytest.mark.parametrize("enc", ["bf16", "fp8"])
@pytest.mark.parametrize("C,bits_", [(1, 1), (16, 1), (17, 1), (32, 1), (33, 1), (64, 1), (65, 1), (100, 1),
                                      (128, 1), (65, 4), (128, 8), (33, 8)])
def test_tc_classify_matches_oracle_many_classes(hdc, enc, C, bits_):
    """Class counts across every register block of the fused epilogue."""
    rng = np.random.default_rng(C * 10 + bits_)
    F, D, N = 200, 1300, 260
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    cfg = hdc.ApproxConfig(enc=enc, class_bits=bits_, perf_stride=1)
    model = hdc.Model(T(Bt), cfg, acc=T(acc.astype(np.int32)))
    labels, sims = hdc.classify(T(X), model, sims=True)
    ol, osim = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, bits_, integer=True)
    assert np.array_equal(labels.cpu().numpy(), ol)
    if bits_ == 1:
        assert np.array_equal(sims.cpu().numpy().astype(np.int64), osim)
    else:
        assert np.array_equal(sims.cpu().numpy(), osim)


@pytest.mark.parametrize("enc", ["bf16", "fp8"])
@pytest.mark.parametrize("C", [129, 200, 256, 257])
def test_classify_binary_classes_past_the_fused_kernels(hdc, enc, C):
    """129..256 binary classes: encode, then the classes expanded once into
    the workspace and the tensor-core Hamming (257: the popcount route);
    labels and distances equal the oracle's, ties across class chunks."""
    rng = np.random.default_rng(C * 3 + len(enc))
    F, D, N = 200, 1300, 300
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    acc[C - 1] = acc[2]
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc), acc=T(acc.astype(np.int32)))
    labels, dist = hdc.classify(T(X), model, sims=True)
    ol, od = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, 1, integer=True)
    assert np.array_equal(labels.cpu().numpy(), ol)
    assert np.array_equal(dist.cpu().numpy().astype(np.int64), od)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("C", [20, 50, 100])
def test_tc_classify_ties_across_warpgroups(hdc, C):
    """Equal class hypervectors in every warpgroup's class range: each query
    takes the lowest class index among its nearest."""
    rng = np.random.default_rng(C)
    F, D, N = 128, 777, 300
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    base = rng.integers(-50, 51, (3, D))
    acc = base[rng.integers(0, 3, C)]          # only three distinct classes
    acc[-1] = base[0]
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8"), acc=T(acc.astype(np.int32)))
    labels, dists = hdc.classify(T(X), model, sims=True)
    ol, od = orc.classify(X, Bt, acc.astype(np.int64), orc.ENC_FP32, 0.0, 1.0, 1, 1, integer=True)
    assert np.array_equal(labels.cpu().numpy(), ol)
    assert np.array_equal(dists.cpu().numpy().astype(np.int64), od)


@pytest.mark.parametrize("C", [10, 30, 60, 100])
def test_tc_classify_many_tiles_matches_simt(hdc, C):
    """Persistent fused classify over more query tiles than SMs, every
    epilogue width, against the FFMA encoder + similarity kernel."""
    rng = np.random.default_rng(C + 5)
    F, D, N = 96, 1000, 152 * 128 * 2 + 77
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-200, 201, (C, D)).astype(np.int32)
    m_tc = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8"), acc=T(acc))
    m_si = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8", simt=True), acc=T(acc))
    Xd = T(X)
    l_tc, d_tc = hdc.classify(Xd, m_tc, sims=True)
    l_si, d_si = hdc.classify(Xd, m_si, sims=True)
    assert torch.equal(l_tc, l_si) and torch.equal(d_tc, d_si)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["bf16", "fp8"])
def test_tc_persistent_many_tiles_matches_simt(hdc, enc):
    """More query tiles than SMs: every CTA loops over several tiles and
    both TMEM accumulators; integer data make both encoders exact."""
    rng = np.random.default_rng(11)
    F, D, N = 96, 520, 152 * 128 * 2 + 77
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    m_tc = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc))
    m_si = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc, simt=True))
    Xd = T(X)
    h_tc, h_si = hdc.encode(Xd, m_tc), hdc.encode(Xd, m_si)
    assert torch.equal(h_tc, h_si)
    sub = rng.choice(N, 300, replace=False)
    bits, _, _, _ = orc.encode_bits(X[sub], Bt, orc.ENC_FP32, orc.kept_dims(D), integer=True)
    assert np.array_equal(words_np(h_tc)[sub], pack(bits, words_for(D)))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["fp32", "fp8"])
def test_classify_host_blocks_equal_classify(hdc, enc):
    """hdc_classify_host: host row blocks copied in order, classified, labels
    copied back -- equal to hdc_classify on the concatenated rows."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=200, n_query=700, D=900)
    acc = np.random.default_rng(2).integers(-50, 50, (10, 900)).astype(np.int32)
    model = hdc.Model(T(d["Bt"]), hdc.ApproxConfig(enc=enc, perf_stride=3), acc=T(acc))
    Xh = torch.from_numpy(d["Xq"]).pin_memory()
    cuts = [0, 1, 1, 250, 699, 700]                      # includes an empty block
    parts = [Xh[cuts[i]:cuts[i + 1]] for i in range(len(cuts) - 1)]
    Xd = torch.empty((700, 784), device=dev())
    Ld = torch.empty(700, dtype=torch.int32, device=dev())
    Lh = torch.full((700,), -1, dtype=torch.int32).pin_memory()
    hdc.classify_host(parts, model, Xd, Ld, Lh, model.workspace(700))
    torch.cuda.synchronize()
    ref = hdc.classify(T(d["Xq"]), model).cpu()
    assert torch.equal(Lh, ref)
