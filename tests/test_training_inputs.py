"""Host-side checks of bench_kernels.py (no GPU): the training samples'
packed Bernoulli rows use the library's packed layout, keep pad bits zero and
flip bits at the requested rate; the popcount and LOP3 roofline arithmetic."""
import numpy as np
import pytest
import torch

from tests._helpers import unpack, words_for


@pytest.mark.parametrize("n,D,p", [(5, 40, 0.5), (300, 1000, 0.48), (64, 64, 0.0), (64, 96, 1.0)])
def test_packed_bernoulli_layout_and_rate(n, D, p):
    from bench_kernels import packed_bernoulli
    W = words_for(D)
    g = torch.Generator()
    g.manual_seed(3)
    w = packed_bernoulli(n, D, W, p, g, torch.device("cpu"))
    assert w.shape == (n, W) and w.dtype == torch.int32
    words = w.numpy().view(np.uint32)
    bits = unpack(words, W * 32)
    assert not bits[:, D:].any()                       # pad bits zero
    rate = bits[:, :D].mean()
    assert abs(rate - p) <= 4 * np.sqrt(max(p * (1 - p), 1e-12) / (n * D)) + 1e-12


def test_packed_bernoulli_is_seeded():
    from bench_kernels import packed_bernoulli
    out = []
    for _ in range(2):
        g = torch.Generator()
        g.manual_seed(11)
        out.append(packed_bernoulli(100, 300, words_for(300), 0.3, g, torch.device("cpu")))
    assert torch.equal(out[0], out[1])


def test_popcount_roofline_arithmetic():
    """The popcount peak: 16 per clock per SM x SMs x clock; LOP3: 64."""
    from bench_kernels import lop3_roofline, popcount_roofline
    r = popcount_roofline(16 * 152 * 1e9, 152, 1000.0)
    assert r["peak_per_s"] == 16 * 152 * 1000.0 * 1e6
    assert abs(r["frac"] - 1.0) < 1e-12
    r = lop3_roofline(64 * 148 * 1.5e9 / 2, 148, 1500.0)
    assert r["peak_tlops"] == 64 * 148 * 1500.0 * 1e6 / 1e12 and abs(r["frac"] - 0.5) < 1e-12
