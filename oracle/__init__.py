"""CPU oracle for the HDC classification path -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this package.  The product library never loads it and
shares no code with it.

The arithmetic lives in ``hdc_oracle.c`` (plain C, FP64/int64, compiled with
gcc ``-O2 -ffp-contract=off`` so that FP64 sums are evaluated exactly as
written on every host).  This module only marshals numpy arrays and strings
the C steps together in the paper's order (Sec. 2.1: encode -> bundle/retrain
-> similarity -> nearest class; Listing 1; Sec. 4.2 approximations).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "hdc_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")

ENC_FP32, ENC_BF16, ENC_FP8 = 0, 1, 2

_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile the oracle with gcc into oracle/_build/liboracle.so."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared",
                               "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            i64, f32, i32, f64 = ctypes.c_int64, ctypes.c_float, ctypes.c_int32, ctypes.c_double
            P = ctypes.c_void_p
            sig = {
                "orc_kept_dims": (i64, [i64, f32, f32, i64, P]),
                "orc_gather_cols_u8": (None, [P, i64, i64, P, i64, P]),
                "orc_gather_cols_i64": (None, [P, i64, i64, P, i64, P]),
                "orc_round_bf16": (f64, [f32]),
                "orc_round_e4m3": (f64, [f64]),
                "orc_pow2_scale": (f64, [f64]),
                "orc_quantise_rows": (None, [P, i64, i64, i32, P, P]),
                "orc_encode_f64": (None, [P, i64, i64, P, P, i64, P]),
                "orc_encode_i64": (None, [P, i64, i64, P, P, i64, P]),
                "orc_encode_absdot_f64": (None, [P, i64, i64, P, P, i64, P]),
                "orc_binarise_f64": (None, [P, i64, P]),
                "orc_binarise_i64": (None, [P, i64, P]),
                "orc_hamming": (None, [P, i64, P, i64, i64, P]),
                "orc_argmin_i64": (None, [P, i64, i64, P]),
                "orc_argmax_f64": (None, [P, i64, i64, P]),
                "orc_bundle": (i64, [P, P, i64, i64, i64, P]),
                "orc_acc_in_int32": (i32, [P, i64]),
                "orc_class_bits": (None, [P, i64, i64, P]),
                "orc_retrain_epoch": (i64, [P, P, i64, i64, i64, P]),
                "orc_class_quantise": (None, [P, i64, i64, i32, P]),
                "orc_cosine_scores": (None, [P, i64, P, i64, i64, P]),
                "orc_round_bf16_f64": (f64, [f64]),
                "orc_round_bf16_f64_array": (None, [P, i64, P]),
                "orc_cosine_float": (None, [P, i64, P, i64, i64, P]),
                "orc_levelid_scale": (f32, [i32, f32, f32]),
                "orc_levelid_quantise": (None, [P, i64, f32, f32, i32, P]),
                "orc_levelid_levels": (None, [P, P, P, i64, i32, P]),
                "orc_levelid_encode": (None, [P, i64, i64, P, P, i64, P]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    assert a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


# --------------------------------------------------------------------- steps

def kept_dims(D: int, start: float = 0.0, end: float = 1.0, stride: int = 1) -> np.ndarray:
    """Reduction-perforation index set (Sec. 4.2; Listing 1)."""
    n = _L().orc_kept_dims(D, start, end, stride, None)
    if n < 0:
        raise ValueError("invalid perforation (D=%d start=%r end=%r stride=%d)" % (D, start, end, stride))
    dims = np.empty(max(n, 1), dtype=np.int64)
    _L().orc_kept_dims(D, start, end, stride, _p(dims))
    return dims[:n]


def gather_cols(a: np.ndarray, dims: np.ndarray) -> np.ndarray:
    dims = _c(dims, np.int64)
    if a.dtype == np.uint8:
        a = _c(a, np.uint8)
        out = np.empty((a.shape[0], dims.size), dtype=np.uint8)
        _L().orc_gather_cols_u8(_p(a), a.shape[0], a.shape[1], _p(dims), dims.size, _p(out))
    else:
        a = _c(a, np.int64)
        out = np.empty((a.shape[0], dims.size), dtype=np.int64)
        _L().orc_gather_cols_i64(_p(a), a.shape[0], a.shape[1], _p(dims), dims.size, _p(out))
    return out


def round_bf16(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float32)
    f = _L().orc_round_bf16
    return np.array([f(float(v)) for v in x.ravel()], dtype=np.float64).reshape(x.shape)


def round_e4m3(x) -> np.ndarray:
    x = np.asarray(x, dtype=np.float64)
    f = _L().orc_round_e4m3
    return np.array([f(float(v)) for v in x.ravel()], dtype=np.float64).reshape(x.shape)


def pow2_scale(amax: float) -> float:
    return _L().orc_pow2_scale(float(amax))


def quantise_rows(X: np.ndarray, enc: int):
    """(values in scaled units as FP64, per-row scales) for ENC_FP32/BF16/FP8."""
    X = _c(X, np.float32)
    n, F = X.shape
    out = np.empty((n, F), dtype=np.float64)
    sc = np.empty(n, dtype=np.float64)
    _L().orc_quantise_rows(_p(X), n, F, enc, _p(out), _p(sc))
    return out, sc


def _row_blocks(fn, X: np.ndarray, threads: int, *args) -> np.ndarray:
    """fn(X[rows], *args) over a thread pool of row blocks, concatenated
    (the C steps run without the GIL; the result does not depend on it)."""
    if threads <= 1 or X.shape[0] <= 1:
        return fn(X, *args)
    idx = np.array_split(np.arange(X.shape[0]), min(threads, X.shape[0]))
    with ThreadPoolExecutor(len(idx)) as ex:
        return np.concatenate(list(ex.map(lambda r: fn(X[r], *args), idx)))


def encode_f64(X: np.ndarray, Bt: np.ndarray, dims: np.ndarray, threads: int = 1) -> np.ndarray:
    X = _c(X, np.float64); Bt = _c(Bt, np.float64); dims = _c(dims, np.int64)
    assert X.shape[1] == Bt.shape[1]
    if threads > 1:
        return _row_blocks(encode_f64, X, threads, Bt, dims)
    s = np.empty((X.shape[0], dims.size), dtype=np.float64)
    _L().orc_encode_f64(_p(X), X.shape[0], X.shape[1], _p(Bt), _p(dims), dims.size, _p(s))
    return s


def encode_i64(X: np.ndarray, Bt: np.ndarray, dims: np.ndarray) -> np.ndarray:
    X = _c(X, np.int64); Bt = _c(Bt, np.int64); dims = _c(dims, np.int64)
    assert X.shape[1] == Bt.shape[1]
    s = np.empty((X.shape[0], dims.size), dtype=np.int64)
    _L().orc_encode_i64(_p(X), X.shape[0], X.shape[1], _p(Bt), _p(dims), dims.size, _p(s))
    return s


def encode_absdot(X: np.ndarray, Bt: np.ndarray, dims: np.ndarray, threads: int = 1) -> np.ndarray:
    X = _c(X, np.float64); Bt = _c(Bt, np.float64); dims = _c(dims, np.int64)
    if threads > 1:
        return _row_blocks(encode_absdot, X, threads, Bt, dims)
    s = np.empty((X.shape[0], dims.size), dtype=np.float64)
    _L().orc_encode_absdot_f64(_p(X), X.shape[0], X.shape[1], _p(Bt), _p(dims), dims.size, _p(s))
    return s


def binarise(s: np.ndarray) -> np.ndarray:
    out = np.empty(s.shape, dtype=np.uint8)
    if s.dtype.kind == "i":
        s = _c(s, np.int64)
        _L().orc_binarise_i64(_p(s), s.size, _p(out))
    else:
        s = _c(s, np.float64)
        _L().orc_binarise_f64(_p(s), s.size, _p(out))
    return out


def hamming(q: np.ndarray, c: np.ndarray) -> np.ndarray:
    q = _c(q, np.uint8); c = _c(c, np.uint8)
    assert q.shape[1] == c.shape[1]
    d = np.empty((q.shape[0], c.shape[0]), dtype=np.int64)
    _L().orc_hamming(_p(q), q.shape[0], _p(c), c.shape[0], q.shape[1], _p(d))
    return d


def argmin(v: np.ndarray) -> np.ndarray:
    v = _c(v, np.int64)
    out = np.empty(v.shape[0], dtype=np.int32)
    _L().orc_argmin_i64(_p(v), v.shape[0], v.shape[1], _p(out))
    return out


def argmax(v: np.ndarray) -> np.ndarray:
    v = _c(v, np.float64)
    out = np.empty(v.shape[0], dtype=np.int32)
    _L().orc_argmax_f64(_p(v), v.shape[0], v.shape[1], _p(out))
    return out


class AccumulatorOverflow(OverflowError):
    """A class accumulator left the int32 range the library stores it in."""


def bundle(bits: np.ndarray, y: np.ndarray, C: int) -> np.ndarray:
    bits = _c(bits, np.uint8); y = _c(y, np.int32)
    acc = np.empty((C, bits.shape[1]), dtype=np.int64)
    if _L().orc_bundle(_p(bits), _p(y), bits.shape[0], bits.shape[1], C, _p(acc)) == -2:
        raise AccumulatorOverflow("oracle bundling: an accumulator leaves the int32 range")
    return acc


def class_bits(acc: np.ndarray) -> np.ndarray:
    acc = _c(acc, np.int64)
    out = np.empty(acc.shape, dtype=np.uint8)
    _L().orc_class_bits(_p(acc), acc.shape[0], acc.shape[1], _p(out))
    return out


def retrain_epoch(bits: np.ndarray, y: np.ndarray, acc: np.ndarray) -> int:
    """One epoch; updates acc (int64, C x D) in place, returns #updates."""
    bits = _c(bits, np.uint8); y = _c(y, np.int32)
    assert acc.dtype == np.int64 and acc.flags["C_CONTIGUOUS"]
    n = _L().orc_retrain_epoch(_p(bits), _p(y), bits.shape[0], bits.shape[1], acc.shape[0], _p(acc))
    if n == -2:
        raise AccumulatorOverflow("oracle retrain epoch: an accumulator leaves the int32 range")
    if n < 0:
        raise MemoryError("oracle retrain epoch: out of memory")
    return int(n)


def class_quantise(acc: np.ndarray, b: int) -> np.ndarray:
    acc = _c(acc, np.int64)
    out = np.empty(acc.shape, dtype=np.int64)
    _L().orc_class_quantise(_p(acc), acc.shape[0], acc.shape[1], b, _p(out))
    return out


def cosine_scores(q: np.ndarray, chat: np.ndarray) -> np.ndarray:
    q = _c(q, np.uint8); chat = _c(chat, np.int64)
    assert q.shape[1] == chat.shape[1]
    s = np.empty((q.shape[0], chat.shape[0]), dtype=np.float64)
    _L().orc_cosine_scores(_p(q), q.shape[0], _p(chat), chat.shape[0], q.shape[1], _p(s))
    return s


# ---------------------------------------------------------------- pipelines

def perforate_features(X: np.ndarray, Bt: np.ndarray, start: float = 0.0, end: float = 1.0,
                       stride: int = 1):
    """Reduction perforation of the encoding itself (Sec. 4.2 red_perf on the
    matmul over features): keep features s0 + k*stride < e0 of both the
    query rows and the base rows (the rule of kept_dims over F)."""
    f = kept_dims(X.shape[1], start, end, stride)
    return X[:, f], Bt[:, f]


def encode_bits(X: np.ndarray, Bt: np.ndarray, enc: int, dims: np.ndarray,
                integer: bool = False, threads: int = 1):
    """Quantise -> encode over the kept dims -> binarise.

    Returns (bits N x Dk, scores in units of the row scales, scale_x, scale_b).
    ``integer=True`` encodes integer-valued inputs exactly in int64.
    ``threads`` > 1 splits the rows over a thread pool (same result).
    """
    if threads > 1 and X.shape[0] > 1:
        chunks = np.array_split(np.arange(X.shape[0]), threads)
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda idx: encode_bits(X[idx], Bt, enc, dims, integer, 1), chunks))
        return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]),
                np.concatenate([p[2] for p in parts]), parts[0][3])
    if integer:
        s = encode_i64(np.rint(X).astype(np.int64), np.rint(Bt).astype(np.int64), dims)
        return binarise(s), s, np.ones(X.shape[0]), np.ones(Bt.shape[0])
    Xq, sx = quantise_rows(X, enc)
    Bq, sb = quantise_rows(Bt, enc)
    s = encode_f64(Xq, Bq, dims)
    return binarise(s), s, sx, sb


def train(bits: np.ndarray, y: np.ndarray, C: int, epochs: int):
    """Bundle (epoch 0) then ``epochs`` retraining epochs; returns (acc, updates)."""
    acc = bundle(bits, y, C)
    ups = []
    for _ in range(epochs):
        ups.append(retrain_epoch(bits, y, acc))
    return acc, ups


def kmeans(bits: np.ndarray, init: np.ndarray, iters: int, train_perf=(0.0, 1.0, 1),
           infer_perf=(0.0, 1.0, 1)):
    """HD-Clustering (Sec. 5.1): K-means over binary hypervectors.

    bits: N x D unpacked point bits; init: K x D initial cluster bits.  Each
    of ``iters`` iterations assigns every point to the nearest cluster
    (Hamming over the kept dims of ``train_perf`` = (start, end, stride),
    arg-min, lowest index on ties), then re-forms each cluster as the bundle
    of its members over all D (sign of the sum; no members -> zero sum -> all
    +1, bit 0).  The final labels use the kept dims of ``infer_perf``.
    Returns (labels, cluster bits, acc of the last update or None, changes).
    """
    bits = _c(bits, np.uint8)
    cb = _c(init, np.uint8).copy()
    K, D = cb.shape
    tdims = kept_dims(D, *train_perf)
    idims = kept_dims(D, *infer_perf)
    prev, acc, changes = None, None, []
    for _ in range(iters):
        lab = argmin(hamming(gather_cols(bits, tdims), gather_cols(cb, tdims)))
        changes.append(bits.shape[0] if prev is None else int((lab != prev).sum()))
        prev = lab
        acc = bundle(bits, lab, K)
        cb = class_bits(acc)
    labels = argmin(hamming(gather_cols(bits, idims), gather_cols(cb, idims)))
    return labels, cb, acc, changes


def round_bf16_f64(x: np.ndarray) -> np.ndarray:
    """BF16 rounding (nearest, ties to even) of FP64 values."""
    x = _c(x, np.float64)
    out = np.empty_like(x)
    _L().orc_round_bf16_f64_array(_p(x), x.size, _p(out))
    return out


def cosine_float(q: np.ndarray, chat: np.ndarray) -> np.ndarray:
    q = _c(q, np.float64); chat = _c(chat, np.int64)
    assert q.shape[1] == chat.shape[1]
    out = np.empty((q.shape[0], chat.shape[0]), dtype=np.float64)
    _L().orc_cosine_float(_p(q), q.shape[0], _p(chat), chat.shape[0], q.shape[1], _p(out))
    return out


def float_queries(X: np.ndarray, Bt: np.ndarray, enc: int, dims: np.ndarray, integer: bool = False):
    """Float query hypervectors (the flag HDC_FLAG_FLOAT_QUERY of the C ABI):
    q[i][k] = bf16(s[i][k] * sb[k]) with s the projection of the quantised
    inputs over the kept dims and sb the base row's scale (1 unless FP8)."""
    _, s, _, sb = encode_bits(X, Bt, enc, dims, integer)
    scale = np.ones(len(dims)) if integer else np.asarray(sb, np.float64)[dims]
    return round_bf16_f64(s.astype(np.float64) * scale[None, :])


def classify_float(X: np.ndarray, Bt: np.ndarray, acc: np.ndarray, enc: int = ENC_FP32,
                   start: float = 0.0, end: float = 1.0, stride: int = 1, class_bits_: int = 8,
                   integer: bool = False):
    """Cosine of float query hypervectors against the b-bit class values over
    the kept dims, arg-max.  Returns (labels, scores, q)."""
    D = Bt.shape[0]
    dims = kept_dims(D, start, end, stride)
    q = float_queries(X, Bt, enc, dims, integer)
    chat = gather_cols(class_quantise(acc, class_bits_), dims)
    sc = cosine_float(q, chat)
    return argmax(sc), sc, q


def levelid_scale(L: int, x_lo: float, x_hi: float) -> float:
    return float(_L().orc_levelid_scale(L, x_lo, x_hi))


def levelid_quantise(X: np.ndarray, x_lo: float, scale: float, L: int) -> np.ndarray:
    X = _c(X, np.float32)
    out = np.empty(X.shape, dtype=np.int32)
    _L().orc_levelid_quantise(_p(X), X.size, x_lo, scale, L, _p(out))
    return out


def levelid_levels(lo_bits: np.ndarray, hi_bits: np.ndarray, flip: np.ndarray, L: int) -> np.ndarray:
    lo_bits = _c(lo_bits, np.uint8); hi_bits = _c(hi_bits, np.uint8); flip = _c(flip, np.int32)
    out = np.empty((L, lo_bits.size), dtype=np.uint8)
    _L().orc_levelid_levels(_p(lo_bits), _p(hi_bits), _p(flip), lo_bits.size, L, _p(out))
    return out


def levelid_encode(X: np.ndarray, id_bits: np.ndarray, lo_bits: np.ndarray, hi_bits: np.ndarray,
                   flip: np.ndarray, L: int, x_lo: float, x_hi: float, dims: np.ndarray):
    """Level-ID encoding over the kept dims (Sec. 4.2 ID-based encoding):
    quantise each feature to a level, bind its ID hypervector with that
    level's hypervector, bundle over features, binarise.  Returns (bits, s)."""
    lev = levelid_quantise(X, x_lo, levelid_scale(L, x_lo, x_hi), L)
    levels = levelid_levels(lo_bits, hi_bits, flip, L)
    idk = gather_cols(_c(id_bits, np.uint8), dims)
    lvk = gather_cols(levels, dims)
    s = np.empty((X.shape[0], len(dims)), dtype=np.int64)
    _L().orc_levelid_encode(_p(lev), X.shape[0], X.shape[1], _p(idk), _p(lvk), len(dims), _p(s))
    return binarise(s), s


def classify(X: np.ndarray, Bt: np.ndarray, acc: np.ndarray, enc: int = ENC_FP32,
             start: float = 0.0, end: float = 1.0, stride: int = 1, class_bits_: int = 1,
             integer: bool = False, threads: int = 1):
    """End-to-end classification of query rows X (Listing 1 + Sec. 4.2 knobs).

    Returns (labels, similarity N x C) where similarity is the Hamming distance
    (class_bits_ = 1, arg-min) or the cosine score (class_bits_ > 1, arg-max).
    ``threads`` > 1 splits the queries over a thread pool (the C steps run
    without the GIL); the result does not depend on it.
    """
    D = Bt.shape[0]
    dims = kept_dims(D, start, end, stride)
    if threads > 1 and X.shape[0] > 1:
        chunks = np.array_split(np.arange(X.shape[0]), threads)
        with ThreadPoolExecutor(threads) as ex:
            parts = list(ex.map(lambda idx: classify(X[idx], Bt, acc, enc, start, end, stride,
                                                     class_bits_, integer, 1), chunks))
        return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))
    bits, _, _, _ = encode_bits(X, Bt, enc, dims, integer)
    if class_bits_ == 1:
        cb = gather_cols(class_bits(acc), dims)
        dist = hamming(bits, cb)
        return argmin(dist), dist
    chat = gather_cols(class_quantise(acc, class_bits_), dims)
    sc = cosine_scores(bits, chat)
    return argmax(sc), sc
