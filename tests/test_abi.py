"""Host-side checks of the C ABI: the library loads without a GPU, exports
every function include/hdc.h declares, and its host-only logic (perforation
index sets, word counts, argument checks) agrees with the oracle and the
header.  No kernel is launched."""
import ctypes
import os
import re

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_2606_26547_gb300 import build, hdc
    build.build()
    return hdc.load()


def _declared():
    src = open(os.path.join(ROOT, "include", "hdc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hdc_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol(lib):
    from paper_2606_26547_gb300 import hdc
    names = _declared()
    assert len(names) >= 12
    for n in names:
        assert hasattr(lib, n), n
    assert set(names) <= set(hdc.EXPORTED) | set()


def test_kept_dims_matches_oracle(lib, orc):
    from paper_2606_26547_gb300 import hdc
    rng = np.random.default_rng(0)
    cases = [(2048, 0.0, 0.5, 1), (10000, 0.0, 1.0, 2), (16384, 0.0, 1.0, 2), (10000, 0.1, 0.9, 3),
             (617, 0.3, 0.7, 5), (1, 0.0, 1.0, 1)]
    for _ in range(200):
        s, e = sorted(rng.uniform(0, 1, 2))
        cases.append((int(rng.integers(1, 20000)), float(np.float32(s)), float(np.float32(e)),
                      int(rng.integers(1, 9))))
    for D, s, e, st in cases:
        cfg = hdc.ApproxConfig(perf_start=s, perf_end=e, perf_stride=st)
        try:
            n = orc.kept_dims(D, s, e, st).size
        except ValueError:
            n = -1
        got = hdc.kept_dims(D, cfg)
        assert got == (n if n > 0 else -1), (D, s, e, st)


def test_words(lib):
    from paper_2606_26547_gb300 import hdc
    from tests._helpers import words_for
    for L in (1, 31, 32, 33, 128, 129, 1000, 10000, 16384):
        assert hdc.words(L) == words_for(L)


def test_status_strings(lib):
    for code in range(7):
        assert lib.hdc_status_string(code)


def test_hamming_workspace_without_gpu(lib):
    """The Hamming arg-min workspace holds bytes only on the tensor-core
    route (33..256 classes, D <= 131,072): C rounded up to 16 rows of 256
    bytes per 8 words (W(D) is padded to 4 words); a missing, short or
    misaligned workspace is rejected before anything is enqueued."""
    n = ctypes.c_size_t()

    def nbytes(C, D):
        assert lib.hdc_hamming_argmin_workspace_bytes(C, D, ctypes.byref(n)) == 0
        return n.value
    assert nbytes(10, 1000) == 0 and nbytes(32, 1024) == 0      # popcount routes
    assert nbytes(33, 1024) == 48 * 1024                       # 48 rows x 4 tiles of 256 bytes
    assert nbytes(33, 1000) == 48 * 1024                       # W(1000) = 32, as for 1,024 dims
    assert nbytes(100, 16384) == 112 * 16384
    assert nbytes(256, 2048) == 256 * 2048
    assert nbytes(257, 2048) == 0                              # past the tensor-core route
    assert nbytes(40, 700) == 48 * 768                         # W(700) = 24: three tiles
    assert nbytes(40, 33) == 48 * 256                          # W(33) = 4: one tile, half of it padding
    assert nbytes(40, 131072) == 48 * 131072 and nbytes(40, 131073) == 0   # W <= 4,096
    assert lib.hdc_hamming_argmin_workspace_bytes(0, 10, ctypes.byref(n)) == 1
    assert lib.hdc_hamming_argmin_workspace_bytes(40, 0, ctypes.byref(n)) == 1
    assert lib.hdc_hamming_argmin_workspace_bytes(40, 10, None) == 1
    fake = ctypes.c_void_p(1 << 20)                            # aligned, never dereferenced
    assert lib.hdc_hamming_argmin_ws(fake, fake, 5, 40, 1024, None, fake, None, None, 0, None) == 3
    assert lib.hdc_hamming_argmin_ws(fake, fake, 5, 40, 1024, None, fake, None, fake, 48 * 1024 - 1, None) == 3
    assert lib.hdc_hamming_argmin_ws(fake, fake, 5, 40, 1024, None, fake, None,
                                     ctypes.c_void_p((1 << 20) + 16), 1 << 20, None) == 3
    assert lib.hdc_hamming_argmin_ws(None, None, 5, 0, 10, None, None, None, None, 0, None) == 1


def test_classify_workspace_holds_expanded_classes_without_gpu(lib):
    """hdc_workspace_bytes of a binary model past the fused kernels (129..256
    classes) exceeds that of the same model with 8-bit classes by the
    classes expanded to E4M3 bytes (C rounded up to 16 rows of 256 bytes
    per 8 words); at 128 and 257 classes the two are equal.  A model
    descriptor with placeholder pointers: the size query reads its fields
    only."""
    from paper_2606_26547_gb300 import hdc
    words = lambda d: ((d + 31) // 32 + 3) // 4 * 4

    def ws(C, bits=1, D=10000, N=4096):
        m = hdc.ModelC()
        m.struct_size = ctypes.sizeof(m)
        m.F, m.D, m.Dk, m.C, m.enc, m.ldb, m.class_bits = 784, D, D, C, 1, 784, bits
        m.W, m.flags, m.Fk, m.fs0, m.fstride = words(D), 0, 784, 0, 1
        m.Bq = m.cls = m.cls_sum = m.cls_norm = 1 << 20
        n = ctypes.c_size_t()
        assert lib.hdc_workspace_bytes(N, ctypes.byref(m), ctypes.byref(n)) == 0
        return n.value
    ldcs = (words(10000) + 7) // 8 * 256
    for C, Cp in ((129, 144), (200, 208), (256, 256)):
        assert ws(C) - ws(C, bits=8) == Cp * ldcs
    assert ws(128) == ws(128, bits=8) and ws(257) == ws(257, bits=8)


def test_argument_checks_without_gpu(lib):
    """Invalid arguments are rejected before anything is enqueued."""
    from paper_2606_26547_gb300 import hdc
    cfg = hdc.ApproxConfig().c()
    n = ctypes.c_size_t()
    assert lib.hdc_model_bytes(0, 10, 2, ctypes.byref(cfg), ctypes.byref(n)) == 1
    assert lib.hdc_model_bytes(16, 10, 2, None, ctypes.byref(n)) == 1
    bad = hdc.ApproxConfig(class_bits=3).c()
    assert lib.hdc_model_bytes(16, 10, 2, ctypes.byref(bad), ctypes.byref(n)) == 2
    assert lib.hdc_model_bytes(784, 10000, 10, ctypes.byref(cfg), ctypes.byref(n)) == 0 and n.value > 0
    m = hdc.ModelC()
    assert lib.hdc_model_prepare(None, 16, 10, None, 0, ctypes.byref(cfg), None, 0, ctypes.byref(m), None) == 1
    assert lib.hdc_encode(None, 5, ctypes.byref(m), None, None, None, 0, None) == 1
    assert lib.hdc_hamming_argmin(None, None, 5, 0, 10, None, None, None, None) == 1
    assert lib.hdc_train_epoch(None, None, 5, 10, 2, 7, None, None, None, None, 0, None) == 1
    fake = ctypes.c_void_p(1 << 20)                      # aligned, never dereferenced: argument checks come first
    assert lib.hdc_train_epoch(fake, fake, 5, 10, 2, 3, fake, fake, None, fake, 1 << 20, None) == 1
    assert lib.hdc_train_apply(None, 0, 10, fake, fake, None) == 1         # C = 0
    assert lib.hdc_train_apply(None, 2, 10, None, fake, None) == 1         # no accumulators
    assert lib.hdc_train_apply(fake, 2, 10, fake, ctypes.c_void_p((1 << 20) + 4), None) == 1   # cls misaligned
    assert lib.hdc_classify(None, 5, ctypes.byref(m), None, None, None, None, 0, None) == 1
    assert lib.hdc_kept_dims(100, None) == 100
    assert lib.hdc_selftest_wait(0, None) == 1           # wait limit out of range: nothing enqueued
    assert lib.hdc_selftest_wait(2000001, None) == 1


@pytest.mark.parametrize("N,C", [(1, 1), (60000, 10), (100000, 100), (2000, 7000)])
def test_train_workspace_covers_retraining_groups(lib, N, C):
    """A retraining epoch groups each misclassified sample twice (true and
    predicted class, 2C groups): the workspace holds N predictions, 2N
    permutation entries and per-group histogram, offsets, first items and
    cursors; one byte less is refused before anything is enqueued."""
    n = ctypes.c_size_t()
    assert lib.hdc_train_workspace_bytes(N, 1024, C, ctypes.byref(n)) == 0
    G = 2 * C
    assert n.value >= 4 * N + 4 * 2 * N + 4 * G + 4 * (G + 1) + 4 * (G + 1) + 4 * G
    fake = ctypes.c_void_p(1 << 20)                      # aligned, never dereferenced: the size check comes first
    assert lib.hdc_train_epoch(fake, fake, N, 1024, C, 1, fake, fake, None, fake, n.value - 1, None) == 3
    assert lib.hdc_train_workspace_bytes(N, 0, C, ctypes.byref(n)) == 1


def test_training_size_limits_without_gpu(lib):
    """Training and clustering group samples with int32 offsets over up to
    2N entries: N > 2^30 - 1 or more than 2^28 classes is refused as
    unsupported before anything is enqueued."""
    n = ctypes.c_size_t()
    big = 1 << 30
    assert lib.hdc_train_workspace_bytes(big - 1, 64, 10, ctypes.byref(n)) == 0
    assert lib.hdc_train_workspace_bytes(big, 64, 10, ctypes.byref(n)) == 2
    assert lib.hdc_train_workspace_bytes(10, 64, (1 << 28) + 1, ctypes.byref(n)) == 2
    fake = ctypes.c_void_p(1 << 20)                      # aligned, never dereferenced
    assert lib.hdc_train_epoch(fake, fake, big, 64, 10, 1, fake, fake, None, fake, 1 << 40, None) == 2
    assert lib.hdc_cluster_workspace_bytes(big, 64, 10, ctypes.byref(n)) == 2
    assert lib.hdc_cluster(fake, big, 64, 10, 5, None, None, fake, fake, fake, None, fake, 1 << 40, None) == 2


def test_static_scratch_size_matches_header(lib):
    from paper_2606_26547_gb300 import hdc
    src = open(os.path.join(ROOT, "include", "hdc.h")).read()
    m = re.search(r"#define HDC_STATIC_SCRATCH_BYTES \(\(size_t\)(\d+) << (\d+)\)", src)
    assert m and int(m.group(1)) << int(m.group(2)) == hdc.STATIC_SCRATCH_BYTES


def test_sweep_spec_layout_matches_header(lib):
    """The binding's hdc_sweep_spec fields are the header's, in order."""
    from paper_2606_26547_gb300 import hdc
    src = open(os.path.join(ROOT, "include", "hdc.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} hdc_sweep_spec;", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = re.findall(r"\b([a-z_]+)\s*(?:\[[A-Z_]+\])?\s*;", body)
    assert names == [f[0] for f in hdc.SweepSpecC._fields_]


def test_sweep_spec_checks_without_gpu(lib):
    """Entry extents: start in [0, 1), end in (0, 1] (0 = 1.0), and at least
    one kept dim (floor(end*D) > floor(start*D)); strides powers of two <= 32."""
    from paper_2606_26547_gb300 import hdc
    n = ctypes.c_size_t()

    def ok(D, strides, bits=(1,), **kw):
        spec = hdc.sweep_spec(strides, bits, **kw)
        return lib.hdc_sweep_workspace_bytes(D, 10, ctypes.byref(spec), ctypes.byref(n)) == 0

    assert ok(10000, (1, 2, 4, 8, 16, 32))
    assert ok(10000, (1, 2), ends=(0.5, 0.0), starts=(0.25, 0.9))
    assert ok(100, (1,), starts=(0.0,), ends=(0.015,))          # e0 = 1: dim 0 only
    assert not ok(100, (1,), starts=(0.0,), ends=(0.001,))      # e0 = 0: nothing kept
    assert not ok(100, (1,), starts=(0.5,), ends=(0.505,))      # e0 == s0
    assert not ok(100, (1,), starts=(1.0,))
    assert not ok(100, (1,), starts=(-0.1,))
    assert not ok(100, (1,), ends=(1.5,))
    assert not ok(100, (3,))
    assert not ok(100, (64,))
    assert not ok(100, (1,), bits=(2,))
    spec = hdc.sweep_spec((1,) * 6, (1,))
    spec.n_strides = 7
    assert lib.hdc_sweep_workspace_bytes(100, 10, ctypes.byref(spec), ctypes.byref(n)) == 1


def _struct_fields(name):
    src = open(os.path.join(ROOT, "include", "hdc.h")).read()
    body = re.search(r"typedef struct \{([^}]*)\} " + name + ";", src).group(1)
    body = re.sub(r"/\*.*?\*/", "", body, flags=re.S)
    names = []
    for decl in body.split(";"):
        decl = decl.strip()
        if decl:
            names += [n.strip().lstrip("*") for n in re.sub(r"^(const\s+)?\w+\s*\**", "", decl).split(",")]
    return [n.strip("* ") for n in names]


@pytest.mark.parametrize("cname,pyname", [("hdc_approx_config", "ApproxConfigC"), ("hdc_model", "ModelC"),
                                          ("hdc_levelid_model", "LevelIdModelC")])
def test_struct_layouts_match_header(lib, cname, pyname):
    from paper_2606_26547_gb300 import hdc
    assert _struct_fields(cname) == [f[0] for f in getattr(hdc, pyname)._fields_]


def test_encoding_perforation_checks_without_gpu(lib):
    """Encoding perforation (start, end, stride over F) is validated like the
    dimension perforation; the model is sized for the kept features."""
    from paper_2606_26547_gb300 import hdc
    n0, n1 = ctypes.c_size_t(), ctypes.c_size_t()
    full = hdc.ApproxConfig(enc="fp8").c()
    half = hdc.ApproxConfig(enc="fp8", enc_perf_end=0.5).c()
    assert lib.hdc_model_bytes(784, 10000, 10, ctypes.byref(full), ctypes.byref(n0)) == 0
    assert lib.hdc_model_bytes(784, 10000, 10, ctypes.byref(half), ctypes.byref(n1)) == 0
    assert n1.value < n0.value
    for bad in (hdc.ApproxConfig(enc_perf_start=0.6, enc_perf_end=0.5), hdc.ApproxConfig(enc_perf_stride=0),
                hdc.ApproxConfig(enc_perf_end=0.001)):
        c = bad.c()
        assert lib.hdc_model_bytes(784, 10000, 10, ctypes.byref(c), ctypes.byref(n0)) == 1
