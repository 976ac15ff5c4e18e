"""Score error of the reduced-precision encodings against FP64 on the
ORIGINAL FP32 inputs (Sec. 4.2 Element Type Representation), through the C
ABI.

Projections (hdc_encode's de-scaled FP32 scores).  The quality gate is, per
element, |s_gpu - s| <= tol * sum_f |x_f b_f| with s the FP64 projection of
the unquantised inputs, tol = 1e-2 for BF16 operands and 6e-2 for FP8 E4M3
operands.  For BF16 the gate holds by construction: each product carries at
most (2u + u^2) of its size (u = 2^-9) and the FP32 sum adds at most
4 F 2^-24 of the absolute sum, 3.96e-3 in all at F = 784.  For E4M3 the
worst case (2 * 2^-4 + 2^-8 = 0.129) exceeds 6e-2, so the gate is a
statistical property of the rounding errors, checked here on every element
of the sample.

Float query hypervectors (HDC_FLAG_FLOAT_QUERY) against the un-rounded
definition: cosine of the FP64 projections of the original inputs with the
b-bit class values.  With v the exact projections and e the error of the
BF16 query values, |cos(v + e, c) - cos(v, c)| <= 2 ||e|| / ||v||.
  * Integer data (exact encoding): e is the BF16 rounding alone,
    ||e|| <= 2^-9 ||v||, so the scores are within 2^-8 plus the FP32
    dot-product bound.
  * FP32 operands on float data: ||e|| <= 2^-9 (||v|| + ||g||) + ||g||
    with g_k = 4 F 2^-24 sum_f |x_f b_fk| (FP32 accumulation).
  * BF16 / E4M3 operands on float data: a statistical tolerance.  Each
    operand's rounding error is modelled as independent, zero-mean, with
    variance spacing^2 / 12 (spacing of the format at the value); the first
    order change of the cosine, grad . e, then has a variance computed
    exactly from the inputs, and the tolerance is 6 of its standard
    deviations plus 3 E||e||^2 / ||v||^2 for the second-order term plus the
    FP32 dot-product bound.
"""
import os

import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu

TOL = {"bf16": 1e-2, "fp8": 6e-2}
THREADS = os.cpu_count() or 1


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


def stats(S, s, A):
    """Gate ratio |S - s| / A and the summary reported with it."""
    err = np.abs(S - s)
    r = err / A
    return {"max": float(r.max()), "p99": float(np.percentile(r, 99)),
            "frob_rel": float(np.linalg.norm(S - s) / np.linalg.norm(s)),
            "sign_flip_rate": float(((S < 0) != (s < 0)).mean())}


@pytest.fixture(scope="module")
def cfg2_rows():
    """2,000 query rows at the precision workload's shapes (F = 784,
    D = 10,000) with the FP64 projections of the original inputs and their
    absolute-product sums over all D (the strides below take columns)."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=1, n_query=2000)
    dims = orc.kept_dims(10000)
    s = orc.encode_f64(d["Xq"], d["Bt"], dims, threads=THREADS)
    A = orc.encode_absdot(d["Xq"], d["Bt"], dims, threads=THREADS)
    return d, s, A


@pytest.mark.parametrize("enc", ["bf16", "fp8"])
@pytest.mark.parametrize("stride", [1, 2])
def test_projection_score_error_gate(hdc, cfg2_rows, enc, stride):
    d, s_full, A_full = cfg2_rows
    model = hdc.Model(T(d["Bt"]), hdc.ApproxConfig(enc=enc, perf_stride=stride))
    H, S = hdc.encode(T(d["Xq"]), model, scores=True)
    dims = orc.kept_dims(10000, 0.0, 1.0, stride)
    s, A = s_full[:, dims], A_full[:, dims]
    S = S.cpu().numpy().astype(np.float64)
    st = stats(S, s, A)
    print("score error %s stride %d: %s" % (enc, stride, st))
    assert st["max"] <= TOL[enc], st
    if enc == "bf16":
        assert st["max"] <= 2 ** -8 + 2 ** -18 + 4 * 784 * 2.0 ** -24, st     # the worst case above
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["bf16", "fp8"])
def test_projection_score_error_gate_full_launch_sampled(hdc, enc):
    """One hdc_encode launch over 2^20 query rows (stride 2, the benchmarked
    perforation), the gate checked on a sample of rows recomputed by the
    oracle one by one, first and last row included."""
    from paper_2606_26547_gb300 import synth
    w = synth.WORKLOADS["precision_F784_D10000_C10"]
    d = synth.make(w, n_train=1, n_query=1)
    B = 1 << 20
    X, _ = synth.device_gauss_queries(B, w, seed=31, device=torch.device("cuda"))
    model = hdc.Model(T(d["Bt"]), hdc.ApproxConfig(enc=enc, perf_stride=2))
    H, S = hdc.encode(X, model, scores=True)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    rows = np.unique(np.concatenate([np.random.default_rng(5).choice(B, 150, replace=False), [0, B - 1]]))
    ri = torch.as_tensor(rows, device="cuda")
    Xs, Ss = X[ri].cpu().numpy(), S[ri].cpu().numpy().astype(np.float64)
    del S, H
    dims = orc.kept_dims(w.D, 0.0, 1.0, 2)
    s = orc.encode_f64(Xs, d["Bt"], dims, threads=THREADS)
    A = orc.encode_absdot(Xs, d["Bt"], dims, threads=THREADS)
    st = stats(Ss, s, A)
    print("score error %s stride 2, 2^20-row launch, %d sampled rows: %s" % (enc, rows.size, st))
    assert st["max"] <= TOL[enc], st


# ------------------------------------------------- float query hypervectors

def cos_exact(v, chat):
    """cos(v_i, chat_j) of FP64 projections v against integer class values."""
    return orc.cosine_float(v, chat)


def dot_bound(v, chat):
    """FP32 dot-product and squared-norm bound of the cosine kernels
    (gamma = 4 Dk 2^-24 of sum_k |q c| and of |dot|), relative to the norms."""
    Dk = v.shape[1]
    g = 4.0 * Dk * 2.0 ** -24
    c = chat.astype(np.float64)
    A = np.abs(v) @ np.abs(c).T
    dot = v @ c.T
    den = np.sqrt((v * v).sum(1))[:, None] * np.sqrt((c * c).sum(1))[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(den > 0, 1.01 * g * (A + np.abs(dot)) / den, 0.0) + 1e-12


def check_labels(lab, sc, o_sc, tol):
    srt = np.sort(o_sc, axis=1)
    margin = srt[:, -1] - srt[:, -2]
    tmax = tol.max(axis=1)
    sure = margin > 2 * tmax
    best = np.argmax(o_sc, axis=1)
    assert np.array_equal(lab[sure], best[sure])
    rows = np.arange(len(lab))
    assert np.all(o_sc[rows, lab] >= srt[:, -1] - 2 * tmax)
    return float(sure.mean())


def test_float_query_vs_unrounded_cosine_integer_data(hdc):
    """Exact encodings (integers, +-1 base): the BF16 rounding of the query
    values is the only departure from the un-rounded definition."""
    rng = np.random.default_rng(12)
    F, D, N, C = 617, 2048, 400, 26
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-600, 601, (C, D)).astype(np.int64)
    for enc, perf, bits_ in (("bf16", (0.0, 1.0, 1), 8), ("fp8", (0.0, 1.0, 2), 8), ("fp8", (0.0, 0.5, 1), 4)):
        cfg = hdc.ApproxConfig(enc=enc, class_bits=bits_, perf_start=perf[0], perf_end=perf[1],
                               perf_stride=perf[2], float_query=True)
        model = hdc.Model(T(Bt), cfg, acc=T(acc.astype(np.int32)))
        lab, sc = hdc.classify(T(X), model, sims=True)
        dims = orc.kept_dims(D, *perf)
        v = orc.encode_i64(X, Bt, dims).astype(np.float64)
        chat = orc.gather_cols(orc.class_quantise(acc, bits_), dims)
        o_sc = cos_exact(v, chat)
        tol = 2.0 ** -8 * 1.001 + dot_bound(v, chat)
        sc = sc.cpu().numpy()
        assert np.all(np.abs(sc - o_sc) <= tol), float((np.abs(sc - o_sc) - tol).max())
        check_labels(lab.cpu().numpy(), sc, o_sc, tol)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0


def _spacing_bf16(a):
    """Spacing of BF16 values at |a| (8 significant bits, FP32's exponent range)."""
    e = np.floor(np.log2(np.maximum(np.abs(a), 2.0 ** -126)))
    return 2.0 ** (e - 7)


def _spacing_e4m3(a):
    """Spacing of E4M3 values at |a| (4 significant bits; 2^-9 below 2^-6)."""
    e = np.floor(np.log2(np.maximum(np.abs(a), 2.0 ** -6)))
    return 2.0 ** (e - 3)


def _operand_var(M, enc):
    """Variance of each element's rounding error (original units) under the
    uniform model: spacing^2 / 12, with E4M3 spacing taken in the row's
    power-of-two scale."""
    if enc == "bf16":
        return _spacing_bf16(M) ** 2 / 12.0
    s = np.array([orc.pow2_scale(float(a)) for a in np.abs(M).max(1)])
    return (_spacing_e4m3(M / s[:, None]) * s[:, None]) ** 2 / 12.0


def statistical_tolerance(X, Bk, v, chat, enc):
    """6 sigma of the first-order change of every cosine score, plus the
    second-order term and the FP32 dot-product bound (module docstring)."""
    X = X.astype(np.float64)
    vx, vb = _operand_var(X, enc), _operand_var(Bk, enc)          # N x F, Dk x F
    c = chat.astype(np.float64)
    nv = np.linalg.norm(v, axis=1)
    chn = c / np.linalg.norm(c, axis=1)[:, None]                     # C x Dk
    cosv = (v / nv[:, None]) @ chn.T                                 # N x C
    var_r = _spacing_bf16(v) ** 2 / 12.0                             # BF16 rounding of the query value
    N, C = cosv.shape
    sig2 = np.empty((N, C))
    Ee2 = np.empty(N)
    for i in range(N):
        g = (chn - cosv[i][:, None] * (v[i] / nv[i])[None, :]) / nv[i]     # C x Dk gradients
        t1 = (g @ Bk) ** 2 @ vx[i]                                  # x rounding, shared by all dims
        t2 = (g ** 2) @ (vb @ (X[i] ** 2 + vx[i]))                   # base rounding (and its product with x's)
        t3 = (g ** 2) @ var_r[i]
        sig2[i] = t1 + t2 + t3
        Ee2[i] = (Bk ** 2 @ vx[i]).sum() + (vb @ (X[i] ** 2 + vx[i])).sum() + var_r[i].sum()
    return 6.0 * np.sqrt(sig2) + 3.0 * (Ee2 / nv ** 2)[:, None] + dot_bound(v, chat)


@pytest.mark.parametrize("enc", ["fp32", "bf16", "fp8"])
def test_float_query_vs_unrounded_cosine_gauss(hdc, enc):
    """Float features at the precision workload's shapes (F = 784,
    D = 10,000, stride 2, 8-bit classes) through the fused float-query
    kernel (FP32 operands: the CUDA-core encoder and the cosine kernel)."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=600, n_query=300)
    full = orc.kept_dims(10000)
    tb, _, _, _ = orc.encode_bits(d["Xtr"], d["Bt"], orc.ENC_FP32, full, threads=THREADS)
    acc, _ = orc.train(tb, d["ytr"], 10, 1)
    cfg = hdc.ApproxConfig(enc=enc, class_bits=8, perf_stride=2, float_query=True)
    model = hdc.Model(T(d["Bt"]), cfg, acc=T(acc.astype(np.int32)))
    lab, sc = hdc.classify(T(d["Xq"]), model, sims=True)
    sc = sc.cpu().numpy()
    dims = orc.kept_dims(10000, 0.0, 1.0, 2)
    v = orc.encode_f64(d["Xq"], d["Bt"], dims, threads=THREADS)
    chat = orc.gather_cols(orc.class_quantise(acc, 8), dims)
    o_sc = cos_exact(v, chat)
    if enc == "fp32":
        g = 4 * 784 * 2.0 ** -24 * orc.encode_absdot(d["Xq"], d["Bt"], dims, threads=THREADS)
        nv, ng = np.linalg.norm(v, axis=1), np.linalg.norm(g, axis=1)
        tol = (2 * (2.0 ** -9 * (nv + ng) + ng) / nv)[:, None] * 1.001 + dot_bound(v, chat)
    else:
        tol = statistical_tolerance(d["Xq"], d["Bt"][dims].astype(np.float64), v, chat, enc)
    err = np.abs(sc - o_sc)
    print("float query %s: max |cos error| %.3g, max tolerance used %.3g, median ratio %.3g"
          % (enc, err.max(), tol.max(), float(np.median(err / tol))))
    assert np.all(err <= tol), float((err - tol).max())
    sure = check_labels(lab.cpu().numpy(), sc, o_sc, tol)
    assert sure > 0.5
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
