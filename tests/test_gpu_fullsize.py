"""Full-size parity: the benchmarked configurations at 1,048,576 queries in
one hdc_classify launch (the launch bench.py times), checked on a sample of
rows against the oracle, which recomputes those rows one by one.

Integer data (Listing 1 shapes): every projection is exact, so the sampled
distances and labels equal the oracle's.  Float data: a projection whose
FP64 value lies within the FP32-accumulation bound of zero may take either
sign, so a row's distance to a class may differ from the oracle's by at most
the row's count of such uncertain dims, and the label must agree wherever
the oracle's margin exceeds twice that count."""
import numpy as np
import pytest
import torch

import oracle as orc

pytestmark = pytest.mark.gpu
B = 1 << 20


@pytest.fixture(scope="module")
def hdc():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import build, hdc as h
    build.build()
    h.load()
    orc.build()
    return h


def run(hdc, workload, enc, stride, n_train, sample, seed):
    from paper_2606_26547_gb300 import synth
    w = synth.WORKLOADS[workload]
    d = synth.make(w, n_train=n_train, n_query=10)
    dev = torch.device("cuda")
    Bt = torch.from_numpy(d["Bt"]).to(dev)
    H = hdc.encode(torch.from_numpy(d["Xtr"]).to(dev), hdc.Model(Bt, hdc.ApproxConfig(enc="fp32")))
    acc, _, _ = hdc.train(H, torch.from_numpy(d["ytr"]).to(dev), w.D, w.C, 1)
    model = hdc.Model(Bt, hdc.ApproxConfig(enc=enc, perf_stride=stride), acc=acc)
    X, _ = synth.device_gauss_queries(B, w, seed=seed, device=dev)
    labels, dists = hdc.classify(X, model, sims=True)
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
    rows = np.sort(np.random.default_rng(seed).choice(B, sample, replace=False))
    rows = np.unique(np.concatenate([rows, [0, B - 1]]))
    Xs = X[torch.as_tensor(rows, device=dev)].cpu().numpy()
    return w, d, acc.cpu().numpy().astype(np.int64), rows, Xs, labels.cpu().numpy()[rows], \
        dists.cpu().numpy()[rows].astype(np.int64)


def test_fullsize_integer_F617_D2048_C26_exact(hdc):
    """cfg1 shapes, FP8 (exact on integers), stride 1: tensor-core Hamming path."""
    w, d, acc, rows, Xs, lab, dist = run(hdc, "int_exact_F617_D2048_C26", "fp8", 1, 3000, 400, 11)
    o_lab, o_dist = orc.classify(Xs, d["Bt"], acc, orc.ENC_FP8, 0.0, 1.0, 1, 1, integer=True)
    assert np.array_equal(dist, o_dist) and np.array_equal(lab, o_lab)


def _uncertain(Xs, Bt, enc, dims, F):
    Xq, sx = orc.quantise_rows(Xs, enc)
    Bq, sb = orc.quantise_rows(Bt, enc)
    s = orc.encode_f64(Xq, Bq, dims)
    bound = 4 * F * 2.0 ** -24 * orc.encode_absdot(Xq, Bq, dims)
    return (np.abs(s) <= bound).sum(1)


@pytest.mark.parametrize("workload,stride,n_train,sample", [("precision_F784_D10000_C10", 2, 4000, 150),
                                                            ("large_F1024_D16384_C100", 2, 2000, 60)])
def test_fullsize_float_sampled(hdc, workload, stride, n_train, sample):
    """The headline configuration (FP8, stride 2, one launch of 2^20 queries)
    and the 100-class one, sampled."""
    w, d, acc, rows, Xs, lab, dist = run(hdc, workload, "fp8", stride, n_train, sample, 23)
    o_lab, o_dist = orc.classify(Xs, d["Bt"], acc, orc.ENC_FP8, 0.0, 1.0, stride, 1, threads=8)
    dims = orc.kept_dims(w.D, 0.0, 1.0, stride)
    unc = _uncertain(Xs, d["Bt"], orc.ENC_FP8, dims, w.F)
    assert np.all(np.abs(dist - o_dist) <= unc[:, None])
    srt = np.sort(o_dist, axis=1)
    sure = srt[:, 1] - srt[:, 0] > 2 * unc
    assert sure.mean() > 0.9
    assert np.array_equal(lab[sure], o_lab[sure])
