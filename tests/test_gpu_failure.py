"""Failure detection on the GPU without a fault.

A bounded device wait that runs out is reported by hdc_stream_status as a
timeout, the read clears it, and the context keeps working: the self-test
block waits on a barrier nothing arrives on, through the same bounded-wait
routine as the tensor-core kernels, and returns when its limit expires.
"""
import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu

HDC_OK, HDC_ERR_INVALID_ARG, HDC_ERR_TIMEOUT = 0, 1, 5


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
    return torch.from_numpy(np.ascontiguousarray(a)).to(torch.device("cuda:0"))


def _classify_matches_oracle(hdc, seed):
    rng = np.random.default_rng(seed)
    F, D, N, C = 200, 1300, 300, 10
    X = rng.integers(-8, 8, (N, F)).astype(np.float32)
    Bt = (1 - 2 * rng.integers(0, 2, (D, F))).astype(np.float32)
    acc = rng.integers(-300, 301, (C, D)).astype(np.int64)
    model = hdc.Model(T(Bt), hdc.ApproxConfig(enc="fp8", perf_stride=1), acc=T(acc.astype(np.int32)))
    labels, sims = hdc.classify(T(X), model, sims=True)
    ol, osim = orc.classify(X, Bt, acc, orc.ENC_FP32, 0.0, 1.0, 1, 1, integer=True)
    return np.array_equal(labels.cpu().numpy(), ol) and np.array_equal(sims.cpu().numpy().astype(np.int64), osim)


def test_wait_expiry_is_reported_once(hdc):
    torch.cuda.synchronize()
    assert hdc.stream_status() == HDC_OK
    assert hdc.selftest_wait(2000) == HDC_OK
    assert hdc.stream_status() == HDC_ERR_TIMEOUT
    assert hdc.stream_status() == HDC_OK          # the read cleared it


def test_context_usable_after_expiry(hdc):
    assert hdc.selftest_wait(1000) == HDC_OK
    assert hdc.stream_status() == HDC_ERR_TIMEOUT
    assert _classify_matches_oracle(hdc, 5)        # the fused tensor-core path still runs, bit-exact
    assert hdc.stream_status() == HDC_OK


def test_expiry_on_a_side_stream(hdc):
    s = torch.cuda.Stream()
    assert hdc.selftest_wait(1000, stream=s) == HDC_OK
    assert hdc.stream_status(stream=s) == HDC_ERR_TIMEOUT
    assert hdc.stream_status(stream=s) == HDC_OK


def test_limit_out_of_range_enqueues_nothing(hdc):
    assert hdc.selftest_wait(0) == HDC_ERR_INVALID_ARG
    assert hdc.selftest_wait(2_000_001) == HDC_ERR_INVALID_ARG
    assert hdc.stream_status() == HDC_OK
