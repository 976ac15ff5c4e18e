"""HD-Clustering through the C ABI (hdc_cluster) against the oracle's
K-means: labels, cluster hypervectors, accumulators and per-iteration
change counts bit for bit, under independent training / inference
perforations, with empty clusters, zero iterations and encoded inputs."""
import numpy as np
import pytest
import torch

import oracle as orc
from tests._helpers import pack, unpack, words_for

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


def planted(rng, K, D, per, flip):
    centres = rng.integers(0, 2, (K, D)).astype(np.uint8)
    y = np.repeat(np.arange(K), per)
    return centres[y] ^ (rng.random((K * per, D)) < flip).astype(np.uint8), y


def run_both(hdc, bits, init_idx, iters, tp, ip):
    D = bits.shape[1]
    W = words_for(D)
    H = T(pack(bits, W).view(np.int32))
    init = H[torch.as_tensor(init_idx, device=H.device)].contiguous()
    cfg = lambda p: hdc.ApproxConfig(perf_start=p[0], perf_end=p[1], perf_stride=p[2])
    lab, cls, acc, ch = hdc.cluster(H, D, init, iters, cfg(tp), cfg(ip))
    o_lab, o_cb, o_acc, o_ch = orc.kmeans(bits, bits[init_idx], iters, tp, ip)
    assert np.array_equal(lab.cpu().numpy(), o_lab)
    assert np.array_equal(unpack(cls.cpu().numpy().view(np.uint32), D), o_cb)
    if iters:
        assert np.array_equal(acc.cpu().numpy().astype(np.int64), o_acc)
        assert ch.cpu().numpy().tolist() == o_ch
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    return o_lab


@pytest.mark.parametrize("K,D,per,flip,iters,tp,ip", [
    (5, 512, 60, 0.1, 5, (0.0, 1.0, 1), (0.0, 1.0, 1)),
    (26, 1000, 40, 0.3, 4, (0.1, 0.9, 3), (0.0, 0.9, 1)),
    (3, 33, 7, 0.2, 3, (0.0, 0.5, 1), (0.2, 1.0, 2)),
    (100, 2048, 30, 0.35, 6, (0.0, 0.75, 1), (0.0, 1.0, 4)),
    # 60,000 rows: more 256-row tensor-core tiles than SMs, the class-atom
    # ring running on across tiles; perforated assignment (masked queries)
    (40, 512, 1500, 0.3, 2, (0.0, 1.0, 1), (0.1, 0.95, 3)),
])
def test_cluster_matches_oracle(hdc, K, D, per, flip, iters, tp, ip):
    rng = np.random.default_rng(K * 7 + D)
    bits, _ = planted(rng, K, D, per, flip)
    init_idx = rng.choice(bits.shape[0], K, replace=False)
    run_both(hdc, bits, init_idx, iters, tp, ip)


def test_cluster_empty_and_zero_iterations(hdc):
    rng = np.random.default_rng(1)
    bits, _ = planted(rng, 4, 256, 20, 0.2)
    run_both(hdc, bits, np.array([0, 0, 25, 61]), 3, (0.0, 1.0, 1), (0.0, 1.0, 1))   # cluster 1 stays empty
    run_both(hdc, bits, np.array([5, 30, 45, 70]), 0, (0.0, 1.0, 1), (0.0, 0.5, 1))
    run_both(hdc, bits[:1], np.array([0]), 2, (0.0, 1.0, 1), (0.0, 1.0, 1))


def test_cluster_of_encoded_features(hdc):
    """Encode integer features (exact on every encoder), then cluster."""
    from paper_2606_26547_gb300 import metrics, synth
    d = synth.make("int_exact_F617_D2048_C26", n_train=10, n_query=1040)
    X, y = d["Xq"], d["yq"]
    model = hdc.Model(T(d["Bt"]), hdc.ApproxConfig(enc="fp8"))
    H = hdc.encode(T(X), model)
    bits = unpack(H.cpu().numpy().view(np.uint32), 2048)
    o_bits, _, _, _ = orc.encode_bits(X, d["Bt"], orc.ENC_FP32, orc.kept_dims(2048), integer=True)
    assert np.array_equal(bits, o_bits)
    init_idx = np.array([np.flatnonzero(y == k)[0] for k in range(26)])
    lab = run_both(hdc, bits, init_idx, 5, (0.0, 1.0, 1), (0.0, 0.9, 1))
    assert metrics.nmi(y, lab) > 0.9


def test_cluster_argument_checks(hdc):
    H = torch.zeros((10, 4), dtype=torch.int32, device="cuda")
    with pytest.raises(hdc.HdcError):
        hdc.cluster(H, 100, H[:2].clone(), 2, hdc.ApproxConfig(class_bits=4))
    with pytest.raises(hdc.HdcError):
        hdc.cluster(H, 100, H[:2].clone(), 2, hdc.ApproxConfig(perf_start=0.5, perf_end=0.5))
