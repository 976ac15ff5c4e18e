"""Pins of the CPU oracle against things other than itself.

Each test checks an oracle step against a value the paper prints, a closed
form, an invariant of the mathematics, a library routine (numpy, scipy,
torch CPU casts, Python fractions) or brute force on tiny inputs, chosen so
that a dropped term, a wrong sign or index, or a transposed operand fails.
No GPU is needed.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
import torch
from scipy.spatial import distance as sdist

from tests._helpers import pack, unpack, words_for

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# ----------------------------------------------------------- perforation

def test_kept_dims_listing1_golden(orc):
    # Listing 1 / Sec. 2.2: red_perf(dists, 0.0, 0.5, 1) on D = 2048 keeps
    # the first 1024 elements.
    with open(os.path.join(GOLDEN, "red_perf_listing1.txt")) as f:
        rows = [l.split() for l in f if l.strip() and not l.startswith("#")]
    for D, s, e, st, first, last, cnt in rows:
        dims = orc.kept_dims(int(D), float(s), float(e), int(st))
        assert dims.size == int(cnt)
        assert dims[0] == int(first) and dims[-1] == int(last)
        assert np.array_equal(dims, np.arange(int(first), int(last) + 1))


@pytest.mark.parametrize("D", [1, 31, 2048, 10000, 16384])
def test_kept_dims_properties(orc, D):
    full = orc.kept_dims(D)
    assert np.array_equal(full, np.arange(D))
    prev = set(full.tolist())
    for stride in (2, 4, 8):                      # nested strides
        k = orc.kept_dims(D, 0.0, 1.0, stride)
        assert k.size == (D + stride - 1) // stride
        assert set(k.tolist()) <= prev
        assert np.all(np.diff(k) == stride) or k.size <= 1
        prev = set(k.tolist())
    k = orc.kept_dims(D, 0.25, 0.75, 3) if D >= 4 else None
    if k is not None:
        lo = math.floor(Fraction(float(np.float32(0.25))) * D)
        hi = math.floor(Fraction(float(np.float32(0.75))) * D)
        assert k[0] == lo and k[-1] < hi and k[-1] + 3 >= hi


def test_kept_dims_invalid(orc):
    for args in [(0, 0.0, 1.0, 1), (10, 0.5, 0.5, 1), (10, 0.0, 1.0, 0), (10, -0.1, 1.0, 1),
                 (10, 0.0, 1.5, 1)]:
        with pytest.raises(ValueError):
            orc.kept_dims(*args)


# ------------------------------------------------------------ element types

def test_round_bf16_matches_torch(orc):
    rng = np.random.default_rng(1)
    v = np.concatenate([rng.standard_normal(4000) * 10.0 ** rng.integers(-30, 30, 4000),
                        np.array([0.0, -0.0, 1.0, -1.0, 3.0e38, 1e-40])]).astype(np.float32)
    ours = orc.round_bf16(v)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_round_bf16_ties_to_even(orc):
    # 1 + 2^-8 is halfway between 1 and 1 + 2^-7 -> even (1.0);
    # 1 + 3*2^-8 is halfway between 1 + 2^-7 and 1 + 2^-6 -> even (1 + 2^-6)
    assert orc.round_bf16(np.float32(1 + 2 ** -8)) == 1.0
    assert orc.round_bf16(np.float32(1 + 3 * 2 ** -8)) == 1 + 2 ** -6


def _e4m3_table():
    """All finite E4M3 values, decoded from the bit format in this test."""
    vals = set()
    for code in range(256):
        s, e, m = code >> 7, (code >> 3) & 15, code & 7
        if e == 15 and m == 7:
            continue                                   # NaN
        v = (m / 8.0) * 2.0 ** -6 if e == 0 else (1 + m / 8.0) * 2.0 ** (e - 7)
        vals.add(-v if s else v)
    return np.array(sorted(vals))


def test_e4m3_table_fixed_points(orc):
    t = _e4m3_table()
    assert t.max() == 448.0 and t.min() == -448.0 and t.size == 253  # +-0 merge
    assert np.array_equal(orc.round_e4m3(t), t)


def test_round_e4m3_nearest_even_bruteforce(orc):
    t = _e4m3_table()
    pos = t[t >= 0]
    rng = np.random.default_rng(2)
    v = np.concatenate([rng.uniform(-500, 500, 3000), rng.uniform(-1, 1, 3000),
                        rng.uniform(-0.02, 0.02, 2000),
                        (pos[:-1] + pos[1:]) / 2, -(pos[:-1] + pos[1:]) / 2])
    ours = orc.round_e4m3(v)
    for x, r in zip(v, ours):
        a = abs(x)
        if a >= 448:
            assert abs(r) == 448.0
            continue
        d = np.abs(pos - a)
        cand = pos[d == d.min()]
        if cand.size == 1:
            exp = cand[0]
        else:                                   # tie: even fraction code wins
            def code(val):
                if val < 2.0 ** -6:
                    return int(round(val / 2.0 ** -9))
                e = math.floor(math.log2(val))
                return int(round((val / 2.0 ** e - 1) * 8))
            exp = [c for c in cand if code(c) % 2 == 0][0]
        assert abs(r) == exp and (r == 0 or math.copysign(1, r) == math.copysign(1, x))


def test_round_e4m3_matches_torch_in_range(orc):
    rng = np.random.default_rng(3)
    v = (rng.standard_normal(5000) * 10.0 ** rng.uniform(-4, 2.6, 5000)).clip(-448, 448)
    ours = orc.round_e4m3(v)
    ref = torch.from_numpy(v.astype(np.float32)).to(torch.float8_e4m3fn).to(torch.float64).numpy()
    assert np.array_equal(ours, ref)


def test_pow2_scale_bruteforce(orc):
    rng = np.random.default_rng(4)
    for amax in list(rng.uniform(0, 1, 200) * 10.0 ** rng.integers(-20, 20, 200)) + [448.0, 896.0, 1.0, 3.5]:
        s = orc.pow2_scale(float(amax))
        m, e = math.frexp(s)
        assert m == 0.5                                   # power of two
        assert Fraction(amax) <= 448 * Fraction(s)
        assert Fraction(amax) > 224 * Fraction(s)        # s/2 would not do
    assert orc.pow2_scale(0.0) == 1.0


def test_quantise_rows_fp8_in_table(orc):
    rng = np.random.default_rng(5)
    X = (rng.standard_normal((16, 100)) * rng.uniform(0.01, 100, (16, 1))).astype(np.float32)
    X[3] = 0.0
    q, sc = orc.quantise_rows(X, orc.ENC_FP8)
    t = set(_e4m3_table().tolist())
    assert all(v in t for v in q.ravel())
    assert np.abs(q).max() <= 448
    assert sc[3] == 1.0 and np.all(q[3] == 0)
    # relative error of the e4m3 grid is at most 2^-4 for normal values
    rec = q * sc[:, None]
    big = np.abs(X) > 2.0 ** -6 * sc[:, None]
    assert np.all(np.abs(rec - X)[big] <= np.abs(X)[big] * 2.0 ** -4 + 1e-30)


def test_quantise_rows_dispatch_matches_torch_casts(orc):
    """Each element type of quantise_rows on FP32 rows that are not
    representable in BF16 or E4M3: BF16 = torch's CPU cast with scale 1, FP8 =
    torch's cast of x / s with s the row's power-of-two scale, FP32 = the
    input.  A swapped type code or a skipped rounding fails here."""
    rng = np.random.default_rng(55)
    X = (rng.standard_normal((24, 97)) * 10.0 ** rng.uniform(-6, 6, (24, 1))).astype(np.float32)
    X[:, 0] = np.float32(1 + 2 ** -9)                 # between BF16 neighbours, and E4M3 ones
    X[5] = 0.0
    t = torch.from_numpy(X)
    # most values are not representable in either format
    assert (t.to(torch.bfloat16).to(torch.float32) != t).float().mean() > 0.9
    q, sc = orc.quantise_rows(X, orc.ENC_BF16)
    assert np.array_equal(q, t.to(torch.bfloat16).to(torch.float64).numpy()) and np.all(sc == 1.0)
    q, sc = orc.quantise_rows(X, orc.ENC_FP8)
    amax = np.abs(X.astype(np.float64)).max(1)
    assert all(sc[i] == orc.pow2_scale(amax[i]) for i in range(24))
    scaled = torch.from_numpy((X.astype(np.float64) / sc[:, None]).astype(np.float32))   # exact: s = 2^k
    assert np.array_equal(q, scaled.to(torch.float8_e4m3fn).to(torch.float64).numpy())
    q, sc = orc.quantise_rows(X, orc.ENC_FP32)
    assert np.array_equal(q, X.astype(np.float64)) and np.all(sc == 1.0)


# --------------------------------------------------------------- encoding

def test_encode_int_matches_numpy(orc):
    rng = np.random.default_rng(6)
    X = rng.integers(-8, 8, (37, 61))
    Bt = 1 - 2 * rng.integers(0, 2, (300, 61))
    dims = orc.kept_dims(300, 0.1, 0.9, 3)
    s = orc.encode_i64(X, Bt, dims)
    assert np.array_equal(s, (X @ Bt.T)[:, dims])


def test_encode_f64_matches_numpy(orc):
    rng = np.random.default_rng(7)
    X = rng.standard_normal((20, 50))
    Bt = rng.standard_normal((70, 50))
    dims = orc.kept_dims(70)
    s = orc.encode_f64(X, Bt, dims)
    ab = orc.encode_absdot(X, Bt, dims)
    assert np.all(np.abs(s - X @ Bt.T) <= 1e-13 * ab)
    assert np.allclose(ab, np.abs(X) @ np.abs(Bt).T, rtol=1e-13)


def test_encode_special_cases(orc):
    rng = np.random.default_rng(8)
    F, D = 17, 90
    Bt = rng.standard_normal((D, F))
    dims = orc.kept_dims(D)
    E = np.eye(F)                                   # x = e_f -> h = sign(B row f)
    bits = orc.binarise(orc.encode_f64(E, Bt, dims))
    assert np.array_equal(bits, (Bt.T < 0).astype(np.uint8))
    z = orc.binarise(orc.encode_f64(np.zeros((3, F)), Bt, dims))
    assert not z.any()                              # sign(0) = +1 -> bit 0
    x = rng.standard_normal((5, F))
    for a in (2.0, 0.25, 1024.0):                   # exact positive rescale
        assert np.array_equal(orc.binarise(orc.encode_f64(a * x, Bt, dims)),
                              orc.binarise(orc.encode_f64(x, Bt, dims)))
    assert np.array_equal(orc.binarise(orc.encode_f64(-x, Bt, dims)),
                          1 - orc.binarise(orc.encode_f64(x, Bt, dims)))


def test_encode_simhash_angle(orc):
    # Random hyperplane hashing: for Gaussian B, P[bit differs] = angle/pi,
    # so Hamming/D estimates theta/pi (check within 5 binomial sigmas).
    rng = np.random.default_rng(9)
    F, D = 40, 10000
    Bt = rng.standard_normal((D, F))
    dims = orc.kept_dims(D)
    for _ in range(6):
        x, y = rng.standard_normal(F), rng.standard_normal(F)
        y = x + rng.uniform(0.2, 3) * y
        bx = orc.binarise(orc.encode_f64(x[None], Bt, dims))
        by = orc.binarise(orc.encode_f64(y[None], Bt, dims))
        h = orc.hamming(bx, by)[0, 0]
        p = math.acos(np.dot(x, y) / np.linalg.norm(x) / np.linalg.norm(y)) / math.pi
        assert abs(h / D - p) <= 5 * math.sqrt(p * (1 - p) / D)


# ----------------------------------------------------------------- Hamming

def test_hamming_axioms_and_scipy(orc):
    rng = np.random.default_rng(10)
    Dk = 333
    a = rng.integers(0, 2, (12, Dk)).astype(np.uint8)
    d = orc.hamming(a, a)
    assert np.all(np.diag(d) == 0)
    assert np.array_equal(d, d.T)
    assert np.all(orc.hamming(a, 1 - a).diagonal() == Dk)
    assert d.min() >= 0 and d.max() <= Dk
    for i in range(12):                              # triangle inequality
        for j in range(12):
            assert np.all(d[i, j] <= d[i, :] + d[:, j])
    ref = sdist.cdist(a, a, "hamming") * Dk
    assert np.array_equal(d, np.rint(ref).astype(np.int64))
    pm = 1 - 2 * a.astype(np.int64)                  # (Dk - <q,c>)/2 on +-1
    assert np.array_equal(d, (Dk - pm @ pm.T) // 2)


def test_hamming_perforated_is_subset_distance(orc):
    rng = np.random.default_rng(11)
    D = 1000
    q = rng.integers(0, 2, (5, D)).astype(np.uint8)
    c = rng.integers(0, 2, (7, D)).astype(np.uint8)
    tot = np.zeros((5, 7), dtype=np.int64)
    for r in range(4):                               # residues of stride 4
        dims = orc.kept_dims(D - r, 0.0, 1.0, 4) + r if r else orc.kept_dims(D, 0.0, 1.0, 4)
        dq, dc = orc.gather_cols(q, dims), orc.gather_cols(c, dims)
        part = orc.hamming(dq, dc)
        assert np.array_equal(part, (q[:, None, dims] != c[None, :, dims]).sum(-1))
        tot += part
    assert np.array_equal(tot, orc.hamming(q, c))    # residues add up to stride 1


def test_pack_roundtrip():
    rng = np.random.default_rng(12)
    for D in (1, 31, 32, 33, 127, 128, 129, 10000):
        b = rng.integers(0, 2, (3, D)).astype(np.uint8)
        w = pack(b)
        assert w.shape[1] == words_for(D) and w.shape[1] % 4 == 0
        assert np.array_equal(unpack(w, D), b)
        tail = unpack(w, w.shape[1] * 32)[:, D:]
        assert not tail.any()


# ----------------------------------------------------------- arg-min / max

def test_argmin_argmax_bruteforce(orc):
    rng = np.random.default_rng(13)
    v = rng.integers(0, 4, (500, 9))
    assert np.array_equal(orc.argmin(v), np.argmin(v, axis=1))   # numpy: first minimum
    f = rng.integers(0, 4, (500, 9)).astype(np.float64)
    assert np.array_equal(orc.argmax(f), np.argmax(f, axis=1))
    assert np.all(orc.argmin(np.full((4, 6), 7)) == 0)
    assert np.all(orc.argmax(np.zeros((4, 6))) == 0)


# -------------------------------------------------------- bundle / retrain

def test_bundle_properties(orc):
    rng = np.random.default_rng(14)
    N, D, C = 90, 257, 5
    bits = rng.integers(0, 2, (N, D)).astype(np.uint8)
    y = rng.integers(0, C, N).astype(np.int32)
    acc = orc.bundle(bits, y, C)
    onehot = np.eye(C, dtype=np.int64)[y]
    assert np.array_equal(acc, onehot.T @ (1 - 2 * bits.astype(np.int64)))
    n_c = np.bincount(y, minlength=C)
    assert np.all((acc - n_c[:, None]) % 2 == 0)      # acc = n_c (mod 2)
    perm = rng.permutation(N)
    assert np.array_equal(orc.bundle(bits[perm], y[perm], C), acc)
    one = orc.bundle(bits[:1], np.zeros(1, np.int32), 1)
    assert np.array_equal(orc.class_bits(one), bits[:1])  # one sample reproduces it
    two = orc.bundle(np.stack([bits[0], 1 - bits[0]]), np.zeros(2, np.int32), 1)
    assert not two.any() and not orc.class_bits(two).any()  # h + not h = 0 -> +1


def _separable(rng, C=4, D=512, N=200, flip=0.2):
    protos = rng.integers(0, 2, (C, D)).astype(np.uint8)
    y = (np.arange(N) % C).astype(np.int32)
    noise = (rng.random((N, D)) < flip).astype(np.uint8)
    return protos[y] ^ noise, y


def test_retrain_invariants(orc):
    rng = np.random.default_rng(15)
    bits, y = _separable(rng, C=6, D=300, N=240, flip=0.42)
    acc = orc.bundle(bits, y, 6)
    col = acc.sum(0).copy()
    for _ in range(4):
        before = acc.copy()
        cb = orc.class_bits(before)
        pred = np.argmin(sdist.cdist(bits, cb, "hamming"), axis=1)
        wrong = pred != y
        n = orc.retrain_epoch(bits, y, acc)
        assert n == int(wrong.sum())
        assert np.array_equal(acc.sum(0), col)        # updates move mass between classes
        h = 1 - 2 * bits.astype(np.int64)
        delta = (np.eye(6, dtype=np.int64)[y[wrong]] - np.eye(6, dtype=np.int64)[pred[wrong]]).T @ h[wrong]
        assert np.array_equal(acc - before, delta)


def test_retrain_converges_on_separable(orc):
    rng = np.random.default_rng(16)
    bits, y = _separable(rng, C=4, D=512, N=200, flip=0.3)
    acc = orc.bundle(bits, y, 4)
    ups = [orc.retrain_epoch(bits, y, acc) for _ in range(10)]
    assert ups[-1] == 0
    frozen = acc.copy()
    assert orc.retrain_epoch(bits, y, acc) == 0 and np.array_equal(acc, frozen)


def test_accumulators_checked_against_int32(orc):
    """The library keeps class accumulators in int32: the oracle (int64)
    refuses an epoch whose result int32 cannot hold, and accepts one that
    ends exactly at the int32 limits."""
    # class bits: class 0 = 0,1,0,0,0 and class 1 = 0,0,1,1,1.  Sample 0
    # (class 0, bits 0,1,1,1,1) is 3 from class 0 and 1 from class 1, so it
    # is misclassified and adds h = +1,-1,-1,-1,-1 to class 0; sample 1 equals
    # class 1 and is right
    bits = np.array([[0, 1, 1, 1, 1], [0, 0, 1, 1, 1]], np.uint8)
    y = np.array([0, 1], np.int32)
    over = np.array([[2 ** 31 - 1, -(2 ** 31), 5, 5, 5], [0, 0, -1, -1, -1]], np.int64)
    with pytest.raises(orc.AccumulatorOverflow):
        orc.retrain_epoch(bits, y, over)
    ok = np.array([[2 ** 31 - 2, -(2 ** 31) + 1, 5, 5, 5], [0, 0, -1, -1, -1]], np.int64)
    assert orc.retrain_epoch(bits, y, ok) == 1
    assert ok[0].tolist() == [2 ** 31 - 1, -(2 ** 31), 4, 4, 4] and ok[1].tolist() == [-1, 1, 0, 0, 0]
    assert orc._L().orc_acc_in_int32(orc._p(np.array([2 ** 31], np.int64)), 1) == 0
    assert orc._L().orc_acc_in_int32(orc._p(np.array([-(2 ** 31) - 1], np.int64)), 1) == 0
    assert orc._L().orc_acc_in_int32(orc._p(np.array([-(2 ** 31), 2 ** 31 - 1], np.int64)), 2) == 1


# --------------------------------------------------------- class quantise

def _round_half_away(fr: Fraction) -> int:
    s = -1 if fr < 0 else 1
    a = abs(fr)
    return s * math.floor(a + Fraction(1, 2))


@pytest.mark.parametrize("b", [2, 4, 8])
def test_class_quantise_exhaustive(orc, b):
    Q = 2 ** (b - 1) - 1
    for M in range(1, 40):
        acc = np.arange(-M, M + 1, dtype=np.int64)[None]
        chat = orc.class_quantise(acc, b)[0]
        exp = [_round_half_away(Fraction(int(a) * Q, M)) for a in acc[0]]
        assert chat.tolist() == exp
        assert np.abs(chat).max() == Q


def test_class_quantise_identity_and_sign(orc):
    rng = np.random.default_rng(17)
    acc = rng.integers(-127, 128, (3, 500))
    acc[:, 0] = 127
    assert np.array_equal(orc.class_quantise(acc, 8), acc)
    acc2 = rng.integers(-50, 51, (3, 500))
    c1 = orc.class_quantise(acc2, 1)
    assert np.array_equal(c1, np.where(acc2 >= 0, 1, -1))
    assert not orc.class_quantise(np.zeros((2, 9), np.int64), 4).any()


def test_cosine_scores_vs_scipy(orc):
    rng = np.random.default_rng(18)
    Dk = 400
    q = rng.integers(0, 2, (6, Dk)).astype(np.uint8)
    chat = rng.integers(-7, 8, (5, Dk))
    chat[2] = 0
    sc = orc.cosine_scores(q, chat)
    qpm = 1 - 2 * q.astype(np.float64)
    for i in range(6):
        for j in range(5):
            if j == 2:
                assert sc[i, j] == 0.0
                continue
            cos = 1.0 - sdist.cosine(qpm[i], chat[j].astype(np.float64))
            assert abs(sc[i, j] - cos * math.sqrt(Dk)) < 1e-9


def test_cosine_binary_classes_equals_hamming(orc):
    # with +-1 classes the score is (Dk - 2*Hamming)/sqrt(Dk): same winner
    rng = np.random.default_rng(19)
    Dk = 257
    q = rng.integers(0, 2, (300, Dk)).astype(np.uint8)
    cb = rng.integers(0, 2, (9, Dk)).astype(np.uint8)
    chat = 1 - 2 * cb.astype(np.int64)
    sc = orc.cosine_scores(q, chat)
    hd = orc.hamming(q, cb)
    assert np.allclose(sc, (Dk - 2 * hd) / math.sqrt(Dk), rtol=0, atol=1e-12)
    assert np.array_equal(orc.argmax(sc), orc.argmin(hd))


# ---------------------------------------------------------- end to end

def test_integer_data_three_routes_agree(orc):
    """Integer features and +-1 base: int64, FP64 of the FP32 values and
    FP64 of the E4M3-quantised values (pow2 row scales) give the same bits,
    because every product and partial sum is exact in all three."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("int_exact_F617_D2048_C26", n_train=50, n_query=40)
    dims = orc.kept_dims(2048)
    b_int, s_int, _, _ = orc.encode_bits(d["Xq"], d["Bt"], orc.ENC_FP32, dims, integer=True)
    b_f32, s_f32, _, _ = orc.encode_bits(d["Xq"], d["Bt"], orc.ENC_FP32, dims)
    b_fp8, s_fp8, sx, sb = orc.encode_bits(d["Xq"], d["Bt"], orc.ENC_FP8, dims)
    b_bf, _, _, _ = orc.encode_bits(d["Xq"], d["Bt"], orc.ENC_BF16, dims)
    assert np.array_equal(s_int, s_f32)
    assert np.array_equal(s_fp8 * sx[:, None] * sb[None, :], s_f32)
    assert np.array_equal(b_int, b_f32) and np.array_equal(b_int, b_fp8) and np.array_equal(b_int, b_bf)
    assert np.abs(s_int).max() <= 617 * 8


def test_classify_threads_invariant(orc):
    from paper_2606_26547_gb300 import synth
    d = synth.make("precision_F784_D10000_C10", n_train=40, n_query=30, D=512)
    bits, _, _, _ = orc.encode_bits(d["Xtr"], d["Bt"], orc.ENC_FP32, orc.kept_dims(512))
    acc, _ = orc.train(bits, d["ytr"], 10, 2)
    l1, s1 = orc.classify(d["Xq"], d["Bt"], acc, orc.ENC_BF16, 0.0, 1.0, 2, 1)
    l4, s4 = orc.classify(d["Xq"], d["Bt"], acc, orc.ENC_BF16, 0.0, 1.0, 2, 1, threads=4)
    assert np.array_equal(l1, l4) and np.array_equal(s1, s4)


# ------------------------------------------------- HD-Clustering (K-means)

def _planted(rng, K=5, D=400, per=40, flip=0.12):
    """K random centres; each point flips each bit of its centre w.p. flip."""
    centres = rng.integers(0, 2, (K, D)).astype(np.uint8)
    y = np.repeat(np.arange(K), per)
    bits = centres[y] ^ (rng.random((K * per, D)) < flip).astype(np.uint8)
    return bits, y, centres


def _brute_assign(bits, cb, dims):
    d = (bits[:, None, dims] != cb[None, :, dims]).sum(-1)
    return d.argmin(1)      # numpy: first index on ties


def test_kmeans_steps_are_assignment_and_majority(orc):
    """Every iteration: labels = brute-force nearest (perforated dims), and
    each cluster = per-dim majority of its members over all D (a tie, or no
    member, gives bit 0)."""
    rng = np.random.default_rng(21)
    bits, _, _ = _planted(rng, K=4, D=300, per=30, flip=0.3)
    init = bits[[0, 31, 62, 93]]
    D = bits.shape[1]
    tdims = orc.kept_dims(D, 0.1, 0.8, 3)
    cb = init.copy()
    for it in range(1, 5):
        lab, cb_o, acc, _ = orc.kmeans(bits, init, it, train_perf=(0.1, 0.8, 3))
        want_lab = _brute_assign(bits, cb, tdims)
        ones = np.stack([bits[want_lab == k].sum(0) for k in range(4)])
        cnt = np.bincount(want_lab, minlength=4)[:, None]
        want_cb = (2 * ones > cnt).astype(np.uint8)           # more -1s than +1s
        assert np.array_equal(cb_o, want_cb), it
        assert np.array_equal(acc, cnt - 2 * ones)             # sum of (1 - 2 bit)
        cb = want_cb


def test_kmeans_objective_never_increases(orc):
    """Unperforated K-means: sum over points of the Hamming distance to the
    assigned cluster cannot increase (nearest assignment, then the majority
    that minimises each cluster's sum)."""
    rng = np.random.default_rng(5)
    bits, _, _ = _planted(rng, K=6, D=256, per=50, flip=0.35)
    init = bits[rng.choice(bits.shape[0], 6, replace=False)]
    J = []
    for it in range(0, 8):
        _, cb, _, _ = orc.kmeans(bits, init, it)
        J.append(int((bits[:, None, :] != cb[None]).sum(-1).min(1).sum()))
    assert all(b <= a for a, b in zip(J, J[1:])), J
    assert J[-1] < J[0]


def test_kmeans_recovers_planted_clusters(orc):
    from paper_2606_26547_gb300 import metrics
    rng = np.random.default_rng(9)
    bits, y, centres = _planted(rng, K=5, D=512, per=60, flip=0.1)
    init = bits[[0, 60, 120, 180, 240]]
    lab, cb, _, changes = orc.kmeans(bits, init, 3, infer_perf=(0.0, 0.5, 2))
    assert metrics.nmi(y, lab) == pytest.approx(1.0)
    assert np.array_equal(cb, centres)        # the majority of 60 noisy copies is the centre
    assert changes[0] == bits.shape[0] and changes[-1] == 0


def test_kmeans_zero_iterations_and_empty_cluster(orc):
    rng = np.random.default_rng(3)
    bits, _, _ = _planted(rng, K=3, D=128, per=10)
    init = bits[[0, 0, 15]]                   # clusters 0 and 1 equal: ties go to 0
    lab0, cb0, acc0, ch0 = orc.kmeans(bits, init, 0)
    assert acc0 is None and ch0 == [] and np.array_equal(cb0, init)
    assert np.array_equal(lab0, _brute_assign(bits, init, np.arange(128)))
    lab, cb, acc, _ = orc.kmeans(bits, init, 1)
    assert not (lab == 1).any() and not acc[1].any() and not cb[1].any()


def test_nmi_definition():
    from paper_2606_26547_gb300 import metrics
    assert metrics.nmi([0, 0, 1, 1], [1, 1, 0, 0]) == pytest.approx(1.0)
    assert metrics.nmi([0, 0, 1, 1], [0, 1, 0, 1]) == pytest.approx(0.0)
    assert metrics.nmi([0, 0, 0], [0, 0, 0]) == 1.0
    # hand computation: U = [0,0,1,1], V = [0,0,0,1]
    h_u = math.log(2)
    h_v = -(0.75 * math.log(0.75) + 0.25 * math.log(0.25))
    mi = 0.5 * math.log(0.5 / (0.5 * 0.75)) + 0.25 * math.log(0.25 / (0.5 * 0.75)) + \
        0.25 * math.log(0.25 / (0.5 * 0.25))
    assert metrics.nmi([0, 0, 1, 1], [0, 0, 0, 1]) == pytest.approx(mi / ((h_u + h_v) / 2))
    sk = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(0)
    for _ in range(20):
        a, b = rng.integers(0, 7, 300), rng.integers(0, 5, 300)
        assert metrics.nmi(a, b) == pytest.approx(sk.normalized_mutual_info_score(a, b), abs=1e-12)


# --------------------------------------------- float query hypervectors

def _bf16_table():
    """Every finite BF16 value, ascending, with its bit pattern's parity."""
    bits = np.arange(0, 1 << 16, dtype=np.uint32)
    with np.errstate(invalid="ignore"):                  # the NaN patterns, dropped just below
        vals = (bits << 16).view(np.float32).astype(np.float64)
    ok = np.isfinite(vals)
    v, b = vals[ok], bits[ok]
    order = np.argsort(v, kind="stable")
    v, b = v[order], b[order]
    keep = np.concatenate([[True], v[1:] != v[:-1]])      # +0 / -0 once
    return v[keep], b[keep]


def test_round_bf16_f64_nearest_even_brute_force(orc):
    table, tbits = _bf16_table()
    rng = np.random.default_rng(17)
    x = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.integers(-40, 38, 3000),
                        table[rng.integers(0, table.size - 1, 500)]])
    # exact ties between neighbours, and ties nudged by less than an FP32 ulp
    i = rng.integers(20000, 30000, 200)
    mids = (table[i] + table[i + 1]) / 2
    x = np.concatenate([x, mids, mids + np.abs(mids) * 2.0 ** -40, mids - np.abs(mids) * 2.0 ** -40])
    x = x[np.abs(x) < table[-1]]
    got = orc.round_bf16_f64(x)
    for v, g in zip(x, got):
        j = np.searchsorted(table, v)
        lo, hi = table[max(j - 1, 0)], table[min(j, table.size - 1)]
        if v - lo < hi - v:
            want = lo
        elif hi - v < v - lo:
            want = hi
        else:   # tie: even bit pattern
            want = lo if tbits[max(j - 1, 0)] % 2 == 0 else hi
        assert g == want, (v, g, want)
    # an FP32 intermediate would round twice here: 1 + 2^-8 + 2^-40 -> 1 + 2^-7
    assert orc.round_bf16_f64(np.array([1 + 2.0 ** -8 + 2.0 ** -40]))[0] == 1 + 2.0 ** -7


def test_cosine_float_definition(orc):
    rng = np.random.default_rng(8)
    q = rng.standard_normal((40, 300))
    chat = rng.integers(-127, 128, (7, 300))
    sc = orc.cosine_float(q, chat)
    want = 1.0 - sdist.cdist(q, chat.astype(np.float64), "cosine")
    assert np.allclose(sc, want, rtol=0, atol=1e-12)
    assert np.allclose(orc.cosine_float(q * 2.5e7, chat), sc, rtol=0, atol=1e-12)    # scale invariance
    # +-1 queries: the binary-query cosine (which leaves out ||q|| = sqrt(Dk))
    bits = rng.integers(0, 2, (40, 300)).astype(np.uint8)
    pm = 1.0 - 2.0 * bits
    assert np.allclose(orc.cosine_float(pm, chat) * math.sqrt(300), orc.cosine_scores(bits, chat),
                       rtol=1e-13, atol=1e-12)
    z = orc.cosine_float(np.zeros((2, 300)), chat)
    assert not z.any()
    chat[3] = 0
    assert not orc.cosine_float(q, chat)[:, 3].any()


def test_float_queries_integer_data(orc):
    """Integer features, +-1 base: the projections are exact integers and
    their BF16 rounding is the cast of those integers."""
    from paper_2606_26547_gb300 import synth
    d = synth.make("int_exact_F617_D2048_C26", n_train=10, n_query=30)
    dims = orc.kept_dims(2048, 0.0, 1.0, 3)
    q = orc.float_queries(d["Xq"], d["Bt"], orc.ENC_FP32, dims, integer=True)
    s = d["Xq"].astype(np.int64) @ d["Bt"].astype(np.int64)[dims].T
    want = torch.from_numpy(s.astype(np.float32)).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(q, want)
    # E4M3 is exact on this data; sb undoes the base-row scale, and the query
    # row's power-of-two scale (dropped by the definition) scales BF16 exactly
    q8 = orc.float_queries(d["Xq"], d["Bt"], orc.ENC_FP8, dims)
    _, sx = orc.quantise_rows(d["Xq"], orc.ENC_FP8)
    assert np.array_equal(q8 * sx[:, None], want)


# ------------------------------------------------------ Level-ID encoding

def test_levelid_quantise_bins(orc):
    """lo = -8, hi = 8, L = 16: scale 1, so the level of an exactly
    representable x is floor(x + 8), clamped; out-of-range values clamp,
    NaN gives 0; levels never decrease with x; uniform x fills the bins
    evenly."""
    sc = orc.levelid_scale(16, -8.0, 8.0)
    assert sc == 1.0
    x = np.array([-100, -8, -7.5, -0.25, 0, 3.999, 7.75, 8, 1e30, np.nan, -np.inf, np.inf], np.float32)
    want = [0, 0, 0, 7, 8, 11, 15, 15, 15, 0, 0, 15]
    assert orc.levelid_quantise(x, -8.0, sc, 16).tolist() == want
    rng = np.random.default_rng(2)
    for L, lo, hi in ((128, -1.3, 2.9), (2, 0.0, 1.0), (1000, -5.0, 5.0)):
        s = orc.levelid_scale(L, lo, hi)
        xs = np.sort(rng.uniform(lo - 0.5, hi + 0.5, 20000).astype(np.float32))
        lv = orc.levelid_quantise(xs, lo, s, L)
        assert lv.min() >= 0 and lv.max() <= L - 1 and np.all(np.diff(lv) >= 0)
        inside = (xs > lo + 1e-3) & (xs < hi - 1e-3)
        # each level covers (hi - lo) / L of the range, up to FP32 rounding at the edges
        assert np.all(np.abs(lv[inside] - (xs[inside] - lo) * L / (hi - lo)) <= 1.0 + 1e-3)
        if L <= 128:
            cnt = np.bincount(lv[inside], minlength=L)
            assert cnt.min() > 0.6 * cnt.mean() and cnt.max() < 1.4 * cnt.mean()


def test_levelid_levels_interpolate(orc):
    rng = np.random.default_rng(3)
    D, L = 500, 9
    lo, hi = rng.integers(0, 2, D).astype(np.uint8), rng.integers(0, 2, D).astype(np.uint8)
    flip = rng.integers(1, L, D).astype(np.int32)
    lv = orc.levelid_levels(lo, hi, flip, L)
    assert np.array_equal(lv[0], lo) and np.array_equal(lv[L - 1], hi)
    for i in range(L):
        for j in range(i, L):
            want = int(((lo != hi) & (flip > i) & (flip <= j)).sum())
            assert int((lv[i] != lv[j]).sum()) == want
    d = [int((lv[0] != lv[j]).sum()) for j in range(L)]
    assert d == sorted(d)


def test_levelid_encode_bind_bundle(orc):
    """s = sum_f (+-1 id_f) * (+-1 level row of x_f), checked with a dense
    +-1 einsum; F = 1 is the XOR of the ID and level bits; the sign bit is the
    majority of the XORs (more than floor(F/2) differ)."""
    rng = np.random.default_rng(4)
    for F, D, L in ((1, 64, 4), (7, 100, 16), (8, 33, 2), (61, 257, 128)):
        ids = rng.integers(0, 2, (F, D)).astype(np.uint8)
        lo, hi = rng.integers(0, 2, D).astype(np.uint8), rng.integers(0, 2, D).astype(np.uint8)
        flip = rng.integers(1, L, D).astype(np.int32)
        X = rng.uniform(-1.2, 1.2, (25, F)).astype(np.float32)
        dims = orc.kept_dims(D, 0.0, 1.0, 1)
        bits, s = orc.levelid_encode(X, ids, lo, hi, flip, L, -1.0, 1.0, dims)
        lev = orc.levelid_quantise(X, -1.0, orc.levelid_scale(L, -1.0, 1.0), L)
        LV = 1 - 2 * orc.levelid_levels(lo, hi, flip, L).astype(np.int64)
        ID = 1 - 2 * ids.astype(np.int64)
        want = np.einsum("fd,nfd->nd", ID, LV[lev])
        assert np.array_equal(s, want)
        xor_cnt = (ids[None, :, :] ^ orc.levelid_levels(lo, hi, flip, L)[lev]).sum(1)
        assert np.array_equal(bits, (xor_cnt > F // 2).astype(np.uint8))
        if F == 1:
            assert np.array_equal(bits, ids[0][None, :] ^ orc.levelid_levels(lo, hi, flip, L)[lev[:, 0]])
    # perforation keeps the same dims of s
    dims = orc.kept_dims(257, 0.1, 0.9, 3)
    b2, s2 = orc.levelid_encode(X, ids, lo, hi, flip, L, -1.0, 1.0, dims)
    assert np.array_equal(s2, s[:, dims]) and np.array_equal(b2, bits[:, dims])
