"""Float query hypervectors (HDC_FLAG_FLOAT_QUERY): BF16 projections and
cosine against b-bit class values on the tensor cores, through the C ABI,
against the oracle's FP64 definition.

Tolerance: integer data make the projections exact integers, so their BF16
values equal the oracle's; the remaining difference is the FP32 dot product
and the FP32 squared norm of the query, bounded (as for the projections of
the binary path) by gamma * sum_k |q_k c_k| with gamma = 4 Dk 2^-24, and
gamma |dot| for the norm.  Labels must agree wherever the oracle's best score
beats the runner-up by more than twice the bound; elsewhere the GPU's label
must be within twice the bound of the best."""
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
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def bound(q, chat):
    Dk = q.shape[1]
    g = 4.0 * Dk * 2.0 ** -24
    A = np.abs(q) @ np.abs(chat.astype(np.float64)).T
    dot = q @ chat.astype(np.float64).T
    nq = np.sqrt((q * q).sum(1))[:, None]
    nc = np.sqrt((chat.astype(np.float64) ** 2).sum(1))[None, :]
    den = nq * nc
    with np.errstate(divide="ignore", invalid="ignore"):
        b = np.where(den > 0, (g * A + g * np.abs(dot)) / den, 0.0)
    return b + 1e-12


def check(labels, scores, o_lab, o_sc, b):
    assert np.all(np.abs(scores - o_sc) <= b), float(np.max(np.abs(scores - o_sc) - b))
    srt = np.sort(o_sc, axis=1)
    margin = srt[:, -1] - (srt[:, -2] if o_sc.shape[1] > 1 else -np.inf)
    bmax = b.max(axis=1)
    sure = margin > 2 * bmax
    assert np.array_equal(labels[sure], o_lab[sure])
    rows = np.arange(len(labels))
    assert np.all(o_sc[rows, labels] >= srt[:, -1] - 2 * bmax)


@pytest.mark.parametrize("enc,simt", [("bf16", False), ("fp8", False), ("fp32", False), ("fp8", True)])
@pytest.mark.parametrize("C,bits_,perf", [(10, 8, (0.0, 1.0, 1)), (26, 4, (0.0, 0.5, 1)), (100, 8, (0.1, 0.97, 3)),
                                          (1, 8, (0.0, 1.0, 2)), (256, 4, (0.0, 1.0, 1)), (17, 8, (0.3, 1.0, 2)),
                                          (113, 8, (0.0, 1.0, 2)), (128, 4, (0.05, 0.95, 1))])
def test_float_query_integer_data(hdc, enc, simt, C, bits_, perf):
    rng = np.random.default_rng(C * 31 + bits_)
    F, D, N = 300, 1000, 333
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-400, 401, (C, D)).astype(np.int64)
    cfg = hdc.ApproxConfig(enc=enc, simt=simt, class_bits=bits_, perf_start=perf[0], perf_end=perf[1],
                           perf_stride=perf[2], float_query=True)
    model = hdc.Model(T(Bt), cfg, acc=T(acc.astype(np.int32)))
    labels, scores = hdc.classify(T(X), model, sims=True)
    o_lab, o_sc, q = orc.classify_float(X, Bt, acc, orc.ENC_FP32, *perf, bits_, integer=True)
    dims = orc.kept_dims(D, *perf)
    chat = orc.gather_cols(orc.class_quantise(acc, bits_), dims)
    check(labels.cpu().numpy(), scores.cpu().numpy(), o_lab, o_sc, bound(q, chat))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["fp8", "bf16"])
@pytest.mark.parametrize("D,C", [(100, 3), (240, 16), (480, 7), (481, 16), (1213, 11)])
def test_float_query_16_class_tiles(hdc, enc, D, C):
    """The fused kernel for up to 16 classes (240-dim encode tiles, the
    cosine partials beside each accumulator): kept dims below one tile,
    exactly one and two tiles, one past, and ragged; more 128-query blocks
    than SMs.  Sampled rows against the oracle on integer data."""
    rng = np.random.default_rng(D * 17 + C)
    F, N = 64, 152 * 128 + 77
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    m = hdc.Model(T(Bt), hdc.ApproxConfig(enc=enc, class_bits=8, float_query=True), acc=T(acc.astype(np.int32)))
    lab, sc = hdc.classify(T(X), m, sims=True)
    lab, sc = lab.cpu().numpy(), sc.cpu().numpy()
    rows = np.sort(np.concatenate([rng.choice(N - 200, 300, replace=False), np.arange(N - 200, N)]))
    o_lab, o_sc, q = orc.classify_float(X[rows], Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, 8, integer=True)
    chat = orc.gather_cols(orc.class_quantise(acc, 8), orc.kept_dims(D))
    check(lab[rows], sc[rows], o_lab, o_sc, bound(q, chat))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


def test_float_query_tensor_path_and_ffma_path_on_integers(hdc):
    """More query tiles than SMs through the fused tensor-core kernel and
    through the FFMA encoder + cosine kernel: on sampled rows both agree
    with the oracle within the bound (exact BF16 projections on integers;
    the FP32 dot products and norms are summed in different orders), and
    their labels agree wherever the oracle's margin exceeds the bound."""
    rng = np.random.default_rng(2)
    F, D, C, N = 128, 700, 40, 152 * 128 * 2 + 99
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    Xd = T(X)
    out = []
    for simt in (False, True):
        m = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8", simt=simt, class_bits=8, float_query=True),
                      acc=T(acc.astype(np.int32)))
        lab, sc = hdc.classify(Xd, m, sims=True)
        out.append((lab.cpu().numpy(), sc.cpu().numpy()))
    rows = np.sort(rng.choice(N, 400, replace=False))
    o_lab, o_sc, q = orc.classify_float(X[rows], Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, 8, integer=True)
    chat = orc.gather_cols(orc.class_quantise(acc, 8), orc.kept_dims(D))
    b = bound(q, chat)
    for lab, sc in out:
        check(lab[rows], sc[rows], o_lab, o_sc, b)
    assert (out[0][0] == out[1][0]).mean() > 0.999
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


def test_float_query_gauss_data(hdc):
    """Float features: FP32 accumulation can move a projection across a BF16
    rounding boundary, so the scores are held to one BF16 step of every
    projection plus the accumulation bound, and labels agree >= 99 %."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=10, n_query=600, D=2048)
    acc = np.random.default_rng(1).integers(-500, 501, (10, 2048)).astype(np.int64)
    for enc in ("bf16", "fp8", "fp32"):
        cfg = hdc.ApproxConfig(enc=enc, class_bits=8, perf_stride=2, float_query=True)
        model = hdc.Model(T(d["Bt"]), cfg, acc=T(acc.astype(np.int32)))
        labels, scores = hdc.classify(T(d["Xq"]), model, sims=True)
        e = {"bf16": orc.ENC_BF16, "fp8": orc.ENC_FP8, "fp32": orc.ENC_FP32}[enc]
        o_lab, o_sc, q = orc.classify_float(d["Xq"], d["Bt"], acc, e, 0.0, 1.0, 2, 8)
        dims = orc.kept_dims(2048, 0.0, 1.0, 2)
        chat = orc.gather_cols(orc.class_quantise(acc, 8), dims).astype(np.float64)
        step = (2.0 ** -8 * np.abs(q)) @ np.abs(chat).T / (np.sqrt((q * q).sum(1))[:, None] *
                                                            np.sqrt((chat ** 2).sum(1))[None, :])
        b = bound(q, chat) + 2 * step
        assert np.all(np.abs(scores.cpu().numpy() - o_sc) <= b)
        assert (labels.cpu().numpy() == o_lab).mean() >= 0.99


def test_float_query_edge_cases(hdc):
    rng = np.random.default_rng(4)
    F, D, C = 64, 300, 5
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-50, 51, (C, D)).astype(np.int32)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="bf16", class_bits=4, float_query=True), acc=T(acc))
    X = np.zeros((3, F), np.float32)                       # q = 0: every score 0, label 0
    lab, sc = hdc.classify(T(X), model, sims=True)
    assert lab.cpu().numpy().tolist() == [0, 0, 0] and not sc.cpu().numpy().any()
    assert hdc.classify(torch.empty((0, F), dtype=torch.float32, device="cuda"), model).numel() == 0
    X1 = rng.integers(-8, 8, (1, F)).astype(np.float32)
    l1 = hdc.classify(T(X1), model).cpu().numpy()
    o1, _, _ = orc.classify_float(X1, Bt, acc.astype(np.int64), orc.ENC_FP32, 0.0, 1.0, 1, 4, integer=True)
    assert l1.tolist() == o1.tolist()
    ls = hdc.classify_static(T(X1), model).cpu().numpy()
    assert ls.tolist() == o1.tolist()
    with pytest.raises(hdc.HdcError):   # float queries need b-bit classes
        hdc.Model(T(Bt), hdc.ApproxConfig(enc="bf16", class_bits=1, float_query=True), acc=T(acc))
    with pytest.raises(hdc.HdcError):   # at most 256 classes
        hdc.Model(T(Bt), hdc.ApproxConfig(enc="bf16", class_bits=8, float_query=True),
                  acc=T(rng.integers(-5, 5, (257, D)).astype(np.int32)))
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
