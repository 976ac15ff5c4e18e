"""Approximation tuner on the GPU: every accuracy the batched evaluator
reports equals the accuracy of the same configuration trained and
classified one by one through the C ABI, and the search returns a feasible
configuration at least as fast as the baseline."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ev():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import build, hdc, synth, tuner
    build.build()
    hdc.load()
    w = synth.Workload("tune_test", 561, 1024, 6, 2000, 1000, "gauss", 4.0, 4, 7100)
    return tuner.GpuEvaluator(w, 4, (1024, 512, 256), reps=2)


def one_by_one(ev, c):
    """Train at c.dim for c.epochs and classify under c through the ABI."""
    from paper_2606_26547_gb300 import hdc
    Bt = ev.Bt[:c.dim]
    H = hdc.encode(ev.Xtr, hdc.Model(Bt, hdc.ApproxConfig(enc=c.enc)))
    acc, _, _ = hdc.train(H, ev.ytr, c.dim, ev.w.C, c.epochs)
    m = hdc.Model(Bt, hdc.ApproxConfig(enc=c.enc, class_bits=c.bits, perf_start=c.start, perf_end=c.end,
                                       perf_stride=c.stride), acc=acc)
    lab = hdc.classify(ev.Xv, m)
    return float((lab == ev.yv).sum().item()) / ev.Xv.shape[0]


def test_tuner_accuracies_equal_one_by_one(ev):
    from paper_2606_26547_gb300 import tuner as T
    space = T.Space("full", 1024, 4, dim_levels=3)
    s = T.Search(space, ev, T.baseline_config(1024, 4), seed=5, batch=24)
    s.run(evaluations=150)
    rep = s.report()
    assert s.feasible(s.best) and rep["speedup"] >= 1.0
    rng = np.random.default_rng(0)
    cs = list(s.results)
    picks = [s.best, s.baseline] + [cs[i] for i in rng.choice(len(cs), 6, replace=False)]
    for c in picks:
        assert s.results[c].accuracy == one_by_one(ev, c), c
        assert s.results[c].ms > 0


def test_tuner_modes_respect_pruning(ev):
    from paper_2606_26547_gb300 import tuner as T
    for mode in ("none", "end_only"):
        space = T.Space(mode, 1024, 4, dim_levels=3)
        s = T.Search(space, ev, T.baseline_config(1024, 4), seed=1, batch=24)
        s.run(evaluations=80)
        b = s.best
        assert b.start == 0.0 and b.stride == 1 and (mode != "none" or b.end == 1.0)
