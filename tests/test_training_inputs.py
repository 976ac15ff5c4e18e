"""Host-side checks of the throughput modules (no GPU): the training
module's packed Bernoulli rows use the library's packed layout, keep pad
bits zero and flip bits at the requested rate; the Hamming module's popcount
roofline arithmetic."""
import numpy as np
import pytest
import torch

from tests._helpers import unpack, words_for


@pytest.mark.parametrize("n,D,p", [(5, 40, 0.5), (300, 1000, 0.48), (64, 64, 0.0), (64, 96, 1.0)])
def test_packed_bernoulli_layout_and_rate(n, D, p):
    from paper_2606_26547_gb300.training import packed_bernoulli
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
    from paper_2606_26547_gb300.training import packed_bernoulli
    out = []
    for _ in range(2):
        g = torch.Generator()
        g.manual_seed(11)
        out.append(packed_bernoulli(100, 300, words_for(300), 0.3, g, torch.device("cpu")))
    assert torch.equal(out[0], out[1])


def test_popcount_roofline_arithmetic():
    """The Hamming module's popcount peak: 16 per clock per SM x SMs x clock."""
    from paper_2606_26547_gb300.hamming import popcount_roofline
    r = popcount_roofline(16 * 152 * 1e9, 152, 1000.0)
    assert r["peak_per_s"] == 16 * 152 * 1000.0 * 1e6
    assert abs(r["frac"] - 1.0) < 1e-12
