"""hdc_classify_static: classification for callers that cannot allocate.

A plugin inside a serving process whose device memory belongs to another
allocator, a process held to a device-memory budget fixed at start-up, or a
loop that may not call cudaMalloc can still classify: this entry point takes
no workspace and uses a fixed device array compiled into libhdc instead.
These tests call it through the C ABI and check that, on two calls in a
row, it returns exactly what hdc_classify returns with a caller-provided
workspace (labels and integer distances / FP64 cosine scores are exact, so
the tolerance is zero, as in the other integer-result parity tests), and
that a batch needing more scratch than the array holds is refused.

This file is collected last on purpose and must also pass on its own in a
fresh process.
"""
import ctypes

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import build, hdc as h
    build.build()
    h.load()
    return h


def _model(hdc, enc, bits, seed):
    g = torch.Generator(device="cuda")
    g.manual_seed(seed)
    F, D, C = 784, 2000, 10
    Bt = torch.randn(D, F, generator=g, device="cuda")
    acc = torch.randint(-500, 500, (C, D), generator=g, device="cuda", dtype=torch.int32)
    return hdc.Model(Bt, hdc.ApproxConfig(enc=enc, class_bits=bits, perf_stride=2), acc=acc)


@pytest.mark.parametrize("enc,bits", [("fp8", 1), ("bf16", 1), ("fp32", 1), ("fp8", 8)])
def test_static_scratch_matches_workspace_entry_point(hdc, enc, bits):
    lib = hdc.load()
    model = _model(hdc, enc, bits, 7)
    stream = torch.cuda.current_stream()
    g = torch.Generator(device="cuda")
    for call, seed in enumerate((11, 12)):       # two calls in a row, different inputs
        g.manual_seed(seed)
        N = 3000 + 517 * call
        X = torch.randn(N, 784, generator=g, device="cuda")
        ref_labels, ref_sims = hdc.classify(X, model, sims=True)
        labels = torch.full((N,), -1, dtype=torch.int32, device="cuda")
        sims = torch.zeros_like(ref_sims)
        d_ptr = ctypes.c_void_p(sims.data_ptr()) if bits == 1 else None
        s_ptr = ctypes.c_void_p(sims.data_ptr()) if bits > 1 else None
        rc = lib.hdc_classify_static(ctypes.c_void_p(X.data_ptr()), N, ctypes.byref(model.m),
                                     ctypes.c_void_p(labels.data_ptr()), d_ptr, s_ptr,
                                     ctypes.c_void_p(stream.cuda_stream))
        assert rc == 0, rc
        torch.cuda.synchronize()
        assert torch.equal(labels, ref_labels)
        assert torch.equal(sims, ref_sims)
    assert hdc.stream_status() == 0


def test_static_scratch_refuses_oversize_batch(hdc):
    lib = hdc.load()
    model = _model(hdc, "fp8", 1, 3)
    need = ctypes.c_size_t()
    N = 1
    while True:                                  # smallest batch that does not fit
        assert lib.hdc_workspace_bytes(N, ctypes.byref(model.m), ctypes.byref(need)) == 0
        if need.value > hdc.STATIC_SCRATCH_BYTES:
            break
        N *= 2
    X = torch.zeros((1, 784), device="cuda")     # never read: the call is refused first
    labels = torch.zeros(1, dtype=torch.int32, device="cuda")
    rc = lib.hdc_classify_static(ctypes.c_void_p(X.data_ptr()), N, ctypes.byref(model.m),
                                 ctypes.c_void_p(labels.data_ptr()), None, None, None)
    assert rc == 3                               # HDC_ERR_WORKSPACE
    torch.cuda.synchronize()
    assert labels.item() == 0
