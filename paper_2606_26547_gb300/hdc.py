"""Thin Python binding of libhdc (include/hdc.h) over torch CUDA tensors.

Argument marshalling only: every step of the path runs in the library's CUDA
kernels.  PyTorch supplies device memory and the current stream.  If the
shared library has not been built the import fails loudly; there is no CPU
fallback.
"""
from __future__ import annotations

import ctypes
import dataclasses
import os

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libhdc.so")

ENC = {"fp32": 0, "bf16": 1, "fp8": 2}
FLAG_SIMT_ENCODE = 0x1
FLAG_FLOAT_QUERY = 0x2
STATIC_SCRATCH_BYTES = 64 << 20  # HDC_STATIC_SCRATCH_BYTES

STATUS = {0: "ok", 1: "invalid argument", 2: "unsupported configuration", 3: "buffer or workspace too small",
          4: "CUDA error", 5: "device wait timed out", 6: "device-side check failed"}


class HdcError(RuntimeError):
    def __init__(self, fn: str, code: int):
        super().__init__("%s failed: %s (%d)" % (fn, STATUS.get(code, "?"), code))
        self.code = code


class ApproxConfigC(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("perf_start", ctypes.c_float), ("perf_end", ctypes.c_float),
                ("perf_stride", ctypes.c_uint32), ("enc", ctypes.c_int32), ("class_bits", ctypes.c_uint32),
                ("flags", ctypes.c_uint32), ("enc_perf_start", ctypes.c_float), ("enc_perf_end", ctypes.c_float),
                ("enc_perf_stride", ctypes.c_uint32)]


class ModelC(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("F", ctypes.c_int32), ("D", ctypes.c_int32),
                ("Dk", ctypes.c_int32), ("C", ctypes.c_int32), ("enc", ctypes.c_int32), ("ldb", ctypes.c_int32),
                ("class_bits", ctypes.c_int32), ("W", ctypes.c_int32), ("flags", ctypes.c_uint32),
                ("Bq", ctypes.c_void_p), ("b_scale", ctypes.c_void_p), ("cls", ctypes.c_void_p),
                ("cls_sum", ctypes.c_void_p), ("cls_norm", ctypes.c_void_p), ("cls_sign", ctypes.c_void_p),
                ("ldcs", ctypes.c_int32), ("Fk", ctypes.c_int32), ("fs0", ctypes.c_int32), ("fstride", ctypes.c_int32)]


_P, _I32, _I64, _SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_size_t
_SIGS = {
    "hdc_default_config": (None, [_P]),
    "hdc_kept_dims": (_I64, [_I32, _P]),
    "hdc_words": (_I32, [_I32]),
    "hdc_model_bytes": (_I32, [_I32, _I32, _I32, _P, _P]),
    "hdc_model_prepare": (_I32, [_P, _I32, _I32, _P, _I32, _P, _P, _SZ, _P, _P]),
    "hdc_workspace_bytes": (_I32, [_I64, _P, _P]),
    "hdc_encode": (_I32, [_P, _I64, _P, _P, _P, _P, _SZ, _P]),
    "hdc_hamming_argmin": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _P]),
    "hdc_hamming_argmin_workspace_bytes": (_I32, [_I32, _I32, _P]),
    "hdc_hamming_argmin_ws": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    "hdc_train_workspace_bytes": (_I32, [_I64, _I32, _I32, _P]),
    "hdc_train_epoch": (_I32, [_P, _P, _I64, _I32, _I32, _I32, _P, _P, _P, _P, _SZ, _P]),
    "hdc_train_apply": (_I32, [_P, _I32, _I32, _P, _P, _P]),
    "hdc_classify": (_I32, [_P, _I64, _P, _P, _P, _P, _P, _SZ, _P]),
    "hdc_classify_static": (_I32, [_P, _I64, _P, _P, _P, _P, _P]),
    "hdc_classify_host": (_I32, [_P, _P, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "hdc_sweep_workspace_bytes": (_I32, [_I32, _I32, _P, _P]),
    "hdc_sweep_eval": (_I32, [_P, _P, _I64, _I32, _I32, _P, _P, _P, _P, _P, _SZ, _P]),
    "hdc_cluster_workspace_bytes": (_I32, [_I64, _I32, _I32, _P]),
    "hdc_levelid_model_bytes": (_I32, [_I32, _I32, _I32, _P, _P]),
    "hdc_levelid_prepare": (_I32, [_P, _P, _P, _P, _I32, _I32, _I32, ctypes.c_float, ctypes.c_float, _P, _P, _SZ,
                                   _P, _P, _P]),
    "hdc_levelid_encode": (_I32, [_P, _I64, _P, _P, _P]),
    "hdc_cluster": (_I32, [_P, _I64, _I32, _I32, _I32, _P, _P, _P, _P, _P, _P, _P, _SZ, _P]),
    "hdc_stream_status": (_I32, [_P]),
    "hdc_selftest_wait": (_I32, [ctypes.c_uint32, _P]),
    "hdc_profile_events": (None, [_P, _P]),
    "hdc_status_string": (ctypes.c_char_p, [_I32]),
}
EXPORTED = tuple(_SIGS)

_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load libhdc.so (raises if it is missing: build it with build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(path):
            raise ImportError("libhdc.so not built at %s; run paper_2606_26547_gb300.build.build()" % path)
        lib = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def _call(name: str, *args) -> None:
    rc = getattr(load(), name)(*args)
    if rc != 0:
        raise HdcError(name, rc)


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = torch.cuda.current_stream() if stream is None else stream
    return ctypes.c_void_p(s.cuda_stream)


@dataclasses.dataclass(frozen=True)
class ApproxConfig:
    """Approximation knobs (Sec. 4.2): perforation, encoding type, class bits."""
    perf_start: float = 0.0
    perf_end: float = 1.0
    perf_stride: int = 1
    enc: str = "fp32"
    class_bits: int = 1
    simt: bool = False  # force the CUDA-core encoder
    float_query: bool = False  # cosine on non-binarised query hypervectors (class_bits 4 / 8)
    # perforation of the encoding's own reduction over the F features
    enc_perf_start: float = 0.0
    enc_perf_end: float = 1.0
    enc_perf_stride: int = 1

    def c(self) -> ApproxConfigC:
        cfg = ApproxConfigC()
        load().hdc_default_config(ctypes.byref(cfg))
        cfg.perf_start = self.perf_start
        cfg.perf_end = self.perf_end
        cfg.perf_stride = self.perf_stride
        cfg.enc = ENC[self.enc]
        cfg.class_bits = self.class_bits
        cfg.flags = (FLAG_SIMT_ENCODE if self.simt else 0) | (FLAG_FLOAT_QUERY if self.float_query else 0)
        cfg.enc_perf_start = self.enc_perf_start
        cfg.enc_perf_end = self.enc_perf_end
        cfg.enc_perf_stride = self.enc_perf_stride
        return cfg


def kept_dims(D: int, cfg: ApproxConfig | None = None) -> int:
    c = cfg.c() if cfg else None
    return int(load().hdc_kept_dims(D, ctypes.byref(c) if c else None))


def words(L: int) -> int:
    return int(load().hdc_words(L))


def _empty_bytes(n: int, device) -> torch.Tensor:
    # 256-byte aligned device buffer (the caching allocator aligns to 512)
    return torch.empty(max(int(n), 1), dtype=torch.uint8, device=device)


class Model:
    """A prepared model (hdc_model_prepare): its device buffer and views."""

    def __init__(self, Bt: torch.Tensor, cfg: ApproxConfig, acc: torch.Tensor | None = None,
                 stream=None):
        assert Bt.dtype == torch.float32 and Bt.dim() == 2
        D, F = Bt.shape
        C = 0 if acc is None else acc.shape[0]
        if acc is not None:
            assert acc.dtype == torch.int32 and acc.shape == (C, D)
        self.cfg = cfg
        c = cfg.c()
        nbytes = ctypes.c_size_t()
        _call("hdc_model_bytes", F, D, C, ctypes.byref(c), ctypes.byref(nbytes))
        self.buf = _empty_bytes(nbytes.value, Bt.device)
        self.m = ModelC()
        _call("hdc_model_prepare", _ptr(Bt), F, D, _ptr(acc), C, ctypes.byref(c), _ptr(self.buf),
              nbytes.value, ctypes.byref(self.m), _stream(stream))
        self.device = Bt.device

    @property
    def W(self) -> int:
        return self.m.W

    @property
    def Dk(self) -> int:
        return self.m.Dk

    @property
    def C(self) -> int:
        return self.m.C

    def workspace_bytes(self, N: int) -> int:
        n = ctypes.c_size_t()
        _call("hdc_workspace_bytes", N, ctypes.byref(self.m), ctypes.byref(n))
        return n.value

    def workspace(self, N: int) -> torch.Tensor:
        return _empty_bytes(self.workspace_bytes(N), self.device)


def encode(X: torch.Tensor, model: Model, scores: bool = False, ws: torch.Tensor | None = None,
           stream=None, out: torch.Tensor | None = None):
    """Packed hypervectors (N x W int32 view of uint32 words), [projections]."""
    assert X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == model.m.F
    N = X.shape[0]
    H = torch.empty((N, model.W), dtype=torch.int32, device=X.device) if out is None else out
    assert H.shape == (N, model.W) and H.dtype == torch.int32
    S = torch.empty((N, model.Dk), dtype=torch.float32, device=X.device) if scores else None
    ws = model.workspace(N) if ws is None else ws
    _call("hdc_encode", _ptr(X), N, ctypes.byref(model.m), _ptr(H), _ptr(S), _ptr(ws), ws.numel(),
          _stream(stream))
    return (H, S) if scores else H


def hamming_workspace(C: int, D: int, device) -> torch.Tensor | None:
    """Device workspace for hdc_hamming_argmin_ws (None when it needs none)."""
    n = ctypes.c_size_t()
    _call("hdc_hamming_argmin_workspace_bytes", C, D, ctypes.byref(n))
    return _empty_bytes(n.value, device) if n.value else None


def hamming_argmin(Q: torch.Tensor, Cls: torch.Tensor, D: int, cfg: ApproxConfig | None = None,
                   dists: bool = False, stream=None, ws: torch.Tensor | None = None, use_ws: bool = True):
    """Hamming arg-min of packed rows: hdc_hamming_argmin_ws with a workspace
    (allocated here unless given), or hdc_hamming_argmin with use_ws=False."""
    N, C = Q.shape[0], Cls.shape[0]
    labels = torch.empty(N, dtype=torch.int32, device=Q.device)
    dd = torch.empty((N, C), dtype=torch.int32, device=Q.device) if dists else None
    c = cfg.c() if cfg else None
    if use_ws:
        if ws is None:
            ws = hamming_workspace(C, D, Q.device)
        _call("hdc_hamming_argmin_ws", _ptr(Q), _ptr(Cls), N, C, D, ctypes.byref(c) if c else None, _ptr(labels),
              _ptr(dd), _ptr(ws), ws.numel() if ws is not None else 0, _stream(stream))
    else:
        _call("hdc_hamming_argmin", _ptr(Q), _ptr(Cls), N, C, D, ctypes.byref(c) if c else None, _ptr(labels),
              _ptr(dd), _stream(stream))
    return (labels, dd) if dists else labels


def train_workspace(N: int, D: int, C: int, device) -> torch.Tensor:
    """Device workspace for hdc_train_epoch over N samples, D dims, C classes."""
    n = ctypes.c_size_t()
    _call("hdc_train_workspace_bytes", N, D, C, ctypes.byref(n))
    return _empty_bytes(n.value, device)


def train_epoch(H: torch.Tensor, y: torch.Tensor, D: int, C: int, mode: int, acc: torch.Tensor,
                cls: torch.Tensor, n_updates: torch.Tensor | None = None, ws: torch.Tensor | None = None,
                stream=None) -> None:
    """One bundling (mode 0) or retraining (mode 1) pass, updating acc and
    cls; mode 2 writes this shard's retraining delta to acc and leaves cls."""
    N = H.shape[0]
    if ws is None:
        ws = train_workspace(N, D, C, H.device)
    _call("hdc_train_epoch", _ptr(H), _ptr(y), N, D, C, mode, _ptr(acc), _ptr(cls), _ptr(n_updates),
          _ptr(ws), ws.numel(), _stream(stream))


def train_apply(acc: torch.Tensor, cls: torch.Tensor, delta: torch.Tensor | None = None, stream=None) -> None:
    """hdc_train_apply: acc += delta (if given), then cls = sign of acc."""
    C, D = acc.shape
    assert acc.dtype == torch.int32 and cls.shape == (C, words(D))
    assert delta is None or (delta.shape == acc.shape and delta.dtype == torch.int32)
    _call("hdc_train_apply", _ptr(delta), C, D, _ptr(acc), _ptr(cls), _stream(stream))


def train(H: torch.Tensor, y: torch.Tensor, D: int, C: int, epochs: int, stream=None):
    """Bundling then ``epochs`` retraining epochs; returns (acc, cls, updates)."""
    acc = torch.empty((C, D), dtype=torch.int32, device=H.device)
    cls = torch.empty((C, words(D)), dtype=torch.int32, device=H.device)
    train_epoch(H, y, D, C, 0, acc, cls, stream=stream)
    ups = []
    nu = torch.zeros(1, dtype=torch.int32, device=H.device)
    for _ in range(epochs):
        train_epoch(H, y, D, C, 1, acc, cls, n_updates=nu, stream=stream)
        ups.append(int(nu.item()))
    return acc, cls, ups


def classify(X: torch.Tensor, model: Model, sims: bool = False, ws: torch.Tensor | None = None,
             labels: torch.Tensor | None = None, stream=None):
    """Labels (N int32) and optionally the similarity (N x C int32 Hamming
    distances for binary classes, N x C float64 cosine scores otherwise)."""
    assert X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == model.m.F
    N, C = X.shape[0], model.C
    if labels is None:
        labels = torch.empty(N, dtype=torch.int32, device=X.device)
    dd = sc = None
    if sims:
        if model.m.class_bits == 1:
            dd = torch.empty((N, C), dtype=torch.int32, device=X.device)
        else:
            sc = torch.empty((N, C), dtype=torch.float64, device=X.device)
    ws = model.workspace(N) if ws is None else ws
    _call("hdc_classify", _ptr(X), N, ctypes.byref(model.m), _ptr(labels), _ptr(dd), _ptr(sc), _ptr(ws),
          ws.numel(), _stream(stream))
    if sims:
        return labels, (dd if dd is not None else sc)
    return labels


def profile_events(start=None, stop=None) -> None:
    """Record torch.cuda.Event pair around the encoding kernel of later calls
    from this thread (None, None turns it off)."""
    load().hdc_profile_events(ctypes.c_void_p(start.cuda_event) if start is not None else None,
                              ctypes.c_void_p(stop.cuda_event) if stop is not None else None)


def classify_static(X: torch.Tensor, model: Model, sims: bool = False, labels: torch.Tensor | None = None,
                    stream=None):
    """classify() through hdc_classify_static: no workspace argument; the
    scratch is the library's fixed device array (one call at a time per
    device, at most STATIC_SCRATCH_BYTES of workspace)."""
    assert X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == model.m.F
    N, C = X.shape[0], model.C
    if labels is None:
        labels = torch.empty(N, dtype=torch.int32, device=X.device)
    dd = sc = None
    if sims:
        if model.m.class_bits == 1:
            dd = torch.empty((N, C), dtype=torch.int32, device=X.device)
        else:
            sc = torch.empty((N, C), dtype=torch.float64, device=X.device)
    _call("hdc_classify_static", _ptr(X), N, ctypes.byref(model.m), _ptr(labels), _ptr(dd), _ptr(sc),
          _stream(stream))
    if sims:
        return labels, (dd if dd is not None else sc)
    return labels


def classify_host(parts, model: Model, X_dev: torch.Tensor, labels_dev: torch.Tensor,
                  labels_host: torch.Tensor, ws: torch.Tensor, stream=None) -> None:
    """hdc_classify_host: copy the host row blocks `parts` (CPU tensors,
    pinned for overlap) into X_dev, classify, copy labels to labels_host
    (CPU int32).  Asynchronous on the stream."""
    n = len(parts)
    ptrs = (ctypes.c_void_p * max(n, 1))(*[p.data_ptr() for p in parts])
    rows = (ctypes.c_int64 * max(n, 1))(*[p.shape[0] for p in parts])
    for p in parts:
        assert not p.is_cuda and p.dtype == torch.float32 and p.is_contiguous() and p.shape[1] == model.m.F
    assert not labels_host.is_cuda and labels_host.dtype == torch.int32
    _call("hdc_classify_host", ptrs, rows, n, ctypes.byref(model.m), _ptr(X_dev), _ptr(labels_dev),
          ctypes.c_void_p(labels_host.data_ptr()), _ptr(ws), ws.numel(), _stream(stream))


class SweepSpecC(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("n_strides", ctypes.c_int32), ("strides", ctypes.c_int32 * 6),
                ("starts", ctypes.c_float * 6), ("ends", ctypes.c_float * 6), ("n_bits", ctypes.c_int32), ("bits", ctypes.c_int32 * 4),
                ("block_threads", ctypes.c_int32), ("words_per_chunk", ctypes.c_int32)]


def sweep_spec(strides, bits, block_threads: int = 0, words_per_chunk: int = 0, ends=None,
               starts=None) -> SweepSpecC:
    """strides[i] with optional starts[i] (fraction of D, default 0.0) and
    ends[i] (default 1.0) form the perforation (starts[i], ends[i],
    strides[i]) of entry i."""
    s = SweepSpecC()
    s.struct_size = ctypes.sizeof(SweepSpecC)
    s.n_strides = len(strides)
    for i, v in enumerate(strides):
        s.strides[i] = v
        s.starts[i] = 0.0 if starts is None else starts[i]
        s.ends[i] = 1.0 if ends is None else ends[i]
    s.n_bits = len(bits)
    for i, v in enumerate(bits):
        s.bits[i] = v
    s.block_threads = block_threads
    s.words_per_chunk = words_per_chunk
    return s


class Sweep:
    """Batched scoring of (class width x perforation stride) configurations
    of one trained model (hdc_sweep_eval); buffers are allocated once so the
    call can be captured in a CUDA graph."""

    def __init__(self, D: int, C: int, strides, bits, N: int, device, block_threads: int = 0,
                 words_per_chunk: int = 0, keep_labels: bool = False, ends=None, starts=None):
        self.D, self.C, self.N = D, C, N
        self.strides, self.bits = list(strides), list(bits)
        self.ends = [1.0] * len(self.strides) if ends is None else list(ends)
        self.starts = [0.0] * len(self.strides) if starts is None else list(starts)
        self.spec = sweep_spec(self.strides, self.bits, block_threads, words_per_chunk, self.ends, self.starts)
        n = ctypes.c_size_t()
        _call("hdc_sweep_workspace_bytes", D, C, ctypes.byref(self.spec), ctypes.byref(n))
        self.ws = _empty_bytes(n.value, device)
        self.correct = torch.zeros((len(self.bits), len(self.strides)), dtype=torch.int32, device=device)
        self.labels = (torch.empty((len(self.bits), len(self.strides), N), dtype=torch.int32, device=device)
                       if keep_labels else None)

    def __call__(self, H: torch.Tensor, y: torch.Tensor, acc: torch.Tensor, stream=None) -> torch.Tensor:
        assert H.shape[0] == self.N and y.shape[0] == self.N and acc.shape == (self.C, self.D)
        _call("hdc_sweep_eval", _ptr(H), _ptr(y), self.N, self.D, self.C, _ptr(acc), ctypes.byref(self.spec),
              _ptr(self.correct), _ptr(self.labels), _ptr(self.ws), self.ws.numel(), _stream(stream))
        return self.correct


def cluster(H: torch.Tensor, D: int, init: torch.Tensor, iters: int, train_sim: ApproxConfig | None = None,
            infer_sim: ApproxConfig | None = None, stream=None):
    """HD-Clustering (hdc_cluster): K-means over the packed hypervectors H
    (N x W) from the packed initial cluster hypervectors ``init`` (K x W).
    Returns (labels N, cluster hypervectors K x W, acc K x D, changes[iters])."""
    N, K = H.shape[0], init.shape[0]
    assert H.dtype == torch.int32 and init.dtype == torch.int32 and init.shape[1] == H.shape[1]
    cls = init.clone()
    acc = torch.zeros((K, D), dtype=torch.int32, device=H.device)
    labels = torch.empty(N, dtype=torch.int32, device=H.device)
    changes = torch.zeros(max(iters, 1), dtype=torch.int32, device=H.device)
    n = ctypes.c_size_t()
    _call("hdc_cluster_workspace_bytes", N, D, K, ctypes.byref(n))
    ws = _empty_bytes(n.value, H.device)
    ts = train_sim.c() if train_sim else None
    isim = infer_sim.c() if infer_sim else None
    _call("hdc_cluster", _ptr(H), N, D, K, iters, ctypes.byref(ts) if ts else None,
          ctypes.byref(isim) if isim else None, _ptr(cls), _ptr(acc), _ptr(labels), _ptr(changes), _ptr(ws),
          ws.numel(), _stream(stream))
    return labels, cls, acc, changes[:iters]


class LevelIdModelC(ctypes.Structure):
    _fields_ = [("struct_size", ctypes.c_uint32), ("F", ctypes.c_int32), ("D", ctypes.c_int32),
                ("Dk", ctypes.c_int32), ("L", ctypes.c_int32), ("W", ctypes.c_int32), ("lo", ctypes.c_float),
                ("scale", ctypes.c_float), ("id", ctypes.c_void_p), ("level", ctypes.c_void_p)]


class LevelIdModel:
    """Level-ID encoder (hdc_levelid_prepare): ID hypervectors (F x D bits),
    level end points lo / hi (D bits each), one uint8 or bool element per
    dim (1 = the element -1), and flip levels (D, in 1..L-1), all device
    tensors of the caller's draws."""

    def __init__(self, id_bits: torch.Tensor, lo_bits: torch.Tensor, hi_bits: torch.Tensor, flip: torch.Tensor,
                 L: int, x_lo: float, x_hi: float, cfg: ApproxConfig | None = None, stream=None):
        F, D = id_bits.shape
        assert lo_bits.numel() == D and hi_bits.numel() == D and flip.numel() == D
        self.idb = id_bits.to(torch.uint8).contiguous()
        self.lob = lo_bits.to(torch.uint8).contiguous()
        self.hib = hi_bits.to(torch.uint8).contiguous()
        self.flip = flip.to(torch.int32).contiguous()
        c = cfg.c() if cfg else None
        n = ctypes.c_size_t()
        _call("hdc_levelid_model_bytes", F, D, L, ctypes.byref(c) if c else None, ctypes.byref(n))
        self.buf = _empty_bytes(n.value, id_bits.device)
        self.flip_error = torch.zeros(1, dtype=torch.int32, device=id_bits.device)
        self.m = LevelIdModelC()
        _call("hdc_levelid_prepare", _ptr(self.idb), _ptr(self.lob), _ptr(self.hib), _ptr(self.flip), F, D, L,
              x_lo, x_hi, ctypes.byref(c) if c else None, _ptr(self.buf), n.value, _ptr(self.flip_error),
              ctypes.byref(self.m), _stream(stream))

    @property
    def W(self) -> int:
        return self.m.W

    @property
    def Dk(self) -> int:
        return self.m.Dk


def levelid_encode(X: torch.Tensor, model: LevelIdModel, out: torch.Tensor | None = None, stream=None):
    """Packed Level-ID hypervectors (N x W int32 view of uint32 words)."""
    assert X.dtype == torch.float32 and X.dim() == 2 and X.shape[1] == model.m.F
    N = X.shape[0]
    H = torch.empty((N, model.W), dtype=torch.int32, device=X.device) if out is None else out
    _call("hdc_levelid_encode", _ptr(X), N, ctypes.byref(model.m), _ptr(H), _stream(stream))
    return H


def stream_status(stream=None) -> int:
    """Synchronise the stream and return (and clear) the device status."""
    return int(load().hdc_stream_status(_stream(stream)))


def selftest_wait(limit_us: int = 1000, stream=None) -> int:
    """Enqueue the failure-detection self-test (a bounded wait that runs out
    after limit_us microseconds); returns the launch status.  The expiry shows
    up in the next stream_status()."""
    return int(load().hdc_selftest_wait(int(limit_us), _stream(stream)))
