"""Batched configuration sweep (hdc_sweep_eval) through the C ABI.

Every configuration's predictions must equal hdc_classify's with a model
prepared for that configuration (bit for bit: same encoder columns, same
class quantisation, same FP64 scores); the unquantised-accumulator control
must equal the oracle's cosine arg-max; the launch shape must not change
any result; the CUDA-graph replay must equal the eager run.
"""
import numpy as np
import pytest
import torch

import oracle as orc
from tests._helpers import unpack

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


@pytest.fixture(scope="module")
def trained(hdc):
    from paper_2606_26547_gb300 import synth
    w = synth.Workload("sweep_test", 561, 1000, 6, 600, 300, "gauss", 3.0, 3, 4242)
    d = synth.make(w)
    dev = torch.device("cuda")
    Bt = torch.from_numpy(d["Bt"]).to(dev)
    out = {}
    for enc in ("fp32", "fp8", "bf16"):
        base = hdc.Model(Bt, hdc.ApproxConfig(enc=enc))
        acc, _, _ = hdc.train(hdc.encode(torch.from_numpy(d["Xtr"]).to(dev), base),
                              torch.from_numpy(d["ytr"]).to(dev), w.D, w.C, w.epochs)
        Xv = torch.from_numpy(d["Xq"]).to(dev)
        out[enc] = dict(base=base, acc=acc, H=hdc.encode(Xv, base), Xv=Xv)
    return w, d, Bt, out


STRIDES = (1, 2, 4, 8, 16, 32)


@pytest.mark.parametrize("enc", ["fp32", "fp8", "bf16"])
def test_sweep_equals_classify_per_config(hdc, trained, enc):
    w, d, Bt, out = trained
    m = out[enc]
    yv = torch.from_numpy(d["yq"]).to(Bt.device)
    sw = hdc.Sweep(w.D, w.C, STRIDES, (1, 4, 8), d["Xq"].shape[0], Bt.device, keep_labels=True)
    correct = sw(m["H"], yv, m["acc"]).cpu().numpy()
    labels = sw.labels.cpu().numpy()
    for jb, b in enumerate((1, 4, 8)):
        for i, s in enumerate(STRIDES):
            model = hdc.Model(Bt, hdc.ApproxConfig(enc=enc, class_bits=b, perf_stride=s), acc=m["acc"])
            ref = hdc.classify(m["Xv"], model).cpu().numpy()
            assert np.array_equal(labels[jb, i], ref), (enc, b, s)
            assert correct[jb, i] == int((ref == d["yq"]).sum())


def test_sweep_unquantised_control_vs_oracle(hdc, trained):
    w, d, Bt, out = trained
    m = out["fp32"]
    yv = torch.from_numpy(d["yq"]).to(Bt.device)
    sw = hdc.Sweep(w.D, w.C, STRIDES, (0,), d["Xq"].shape[0], Bt.device, keep_labels=True)
    correct = sw(m["H"], yv, m["acc"]).cpu().numpy()
    qbits = unpack(m["H"].cpu().numpy().view(np.uint32), w.D)
    acc = m["acc"].cpu().numpy().astype(np.int64)
    for i, s in enumerate(STRIDES):
        dims = orc.kept_dims(w.D, 0.0, 1.0, s)
        ref = orc.argmax(orc.cosine_scores(orc.gather_cols(qbits, dims), orc.gather_cols(acc, dims)))
        assert np.array_equal(sw.labels[0, i].cpu().numpy(), ref), s
        assert correct[0, i] == int((ref == d["yq"]).sum())


def test_sweep_launch_shape_does_not_change_results(hdc, trained):
    from paper_2606_26547_gb300 import autotune
    w, d, Bt, out = trained
    m = out["fp8"]
    yv = torch.from_numpy(d["yq"]).to(Bt.device)
    ref = None
    for bt, wc in autotune.CANDIDATES:
        try:
            sw = hdc.Sweep(w.D, w.C, (1, 2, 4, 8), (1, 4, 8, 0), d["Xq"].shape[0], Bt.device, bt, wc,
                           keep_labels=True)
            sw(m["H"], yv, m["acc"])
        except hdc.HdcError:
            continue
        got = (sw.correct.cpu().numpy(), sw.labels.cpu().numpy())
        if ref is None:
            ref = got
        assert np.array_equal(got[0], ref[0]) and np.array_equal(got[1], ref[1]), (bt, wc)
    assert ref is not None


def test_batched_sweep_graph_equals_eager(hdc):
    from paper_2606_26547_gb300 import sweep
    dev = torch.device("cuda")
    models, Xv, yv, w = sweep.train_models("sweep_F561_D10000_C6", range(2), sweep.ENCS, 400, 500, 2, dev)
    bs = sweep.BatchedSweep(models, Xv, yv, w)
    bs.run()
    torch.cuda.synchronize()
    eager = bs.results()
    for sw in bs.sweeps:
        sw.correct.zero_()
    bs.capture()
    for sw in bs.sweeps:
        sw.correct.fill_(-7)
    bs.replay()
    torch.cuda.synchronize()
    assert bs.results() == eager
    assert len(eager) == 2 * 3 * 12 + 4
    assert hdc.stream_status() == 0


@pytest.mark.parametrize("enc", ["fp8", "fp32"])
def test_sweep_entries_with_extents_equal_classify(hdc, trained, enc):
    """Entries (start, end, stride): kept dims d = s0 + k*stride < e0, as
    hdc_classify's perforation (start, end, stride); odd starts shift the
    stride's bit pattern inside each word."""
    w, d, Bt, out = trained
    m = out[enc]
    yv = torch.from_numpy(d["yq"]).to(Bt.device)
    cases = [((1, 2, 4, 1, 8, 2), (0.0, 0.0, 0.0, 0.0, 0.0, 0.0), (0.5, 0.75, 1.0, 0.33, 0.9, 0.031)),
             ((8, 32, 2, 1, 16, 4), (0.013, 0.1, 0.25, 0.5, 0.0071, 0.9), (1.0, 0.95, 0.6, 0.52, 0.4, 1.0))]
    for strides, starts, ends in cases:
        sw = hdc.Sweep(w.D, w.C, strides, (1, 8), d["Xq"].shape[0], Bt.device, keep_labels=True, ends=ends,
                       starts=starts)
        correct = sw(m["H"], yv, m["acc"]).cpu().numpy()
        for jb, b in enumerate((1, 8)):
            for i, (s, a, e) in enumerate(zip(strides, starts, ends)):
                model = hdc.Model(Bt, hdc.ApproxConfig(enc=enc, class_bits=b, perf_start=a, perf_end=e,
                                                       perf_stride=s), acc=m["acc"])
                ref = hdc.classify(m["Xv"], model).cpu().numpy()
                assert np.array_equal(sw.labels[jb, i].cpu().numpy(), ref), (enc, b, s, a, e)
                assert correct[jb, i] == int((ref == d["yq"]).sum())


def test_sweep_extent_control_vs_oracle(hdc, trained):
    """Unquantised-accumulator cosine over (start, end, stride) entries
    against the oracle's kept dims and cosine arg-max."""
    w, d, Bt, out = trained
    m = out["bf16"]
    yv = torch.from_numpy(d["yq"]).to(Bt.device)
    strides, starts, ends = (1, 4, 32, 2), (0.2, 0.031, 0.0, 0.5), (0.7, 1.0, 1.0, 0.51)
    sw = hdc.Sweep(w.D, w.C, strides, (0,), d["Xq"].shape[0], Bt.device, keep_labels=True, ends=ends,
                   starts=starts)
    sw(m["H"], yv, m["acc"])
    qbits = unpack(m["H"].cpu().numpy().view(np.uint32), w.D)
    acc = m["acc"].cpu().numpy().astype(np.int64)
    for i, (s, a, e) in enumerate(zip(strides, starts, ends)):
        dims = orc.kept_dims(w.D, float(np.float32(a)), float(np.float32(e)), s)
        ref = orc.argmax(orc.cosine_scores(orc.gather_cols(qbits, dims), orc.gather_cols(acc, dims)))
        assert np.array_equal(sw.labels[0, i].cpu().numpy(), ref), (s, a, e)
