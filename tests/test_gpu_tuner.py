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
    from paper_2606_26547_gb300 import hdc, tuner as T
    if T.lid_levels(c.enc):
        m = ev._lid_model(c.enc, c.dim)
        acc, cls, _ = hdc.train(hdc.levelid_encode(ev.Xtr, m), ev.ytr, c.dim, ev.w.C, c.epochs)
        cfg = hdc.ApproxConfig(perf_start=c.start, perf_end=c.end, perf_stride=c.stride)
        lab = hdc.hamming_argmin(hdc.levelid_encode(ev.Xv, m), cls, c.dim, cfg)
        return float((lab == ev.yv).sum().item()) / ev.Xv.shape[0]
    Bt = ev.Bt[:c.dim]
    fp = dict(enc_perf_start=c.e_start, enc_perf_end=c.e_end, enc_perf_stride=c.e_stride)
    H = hdc.encode(ev.Xtr, hdc.Model(Bt, hdc.ApproxConfig(enc=c.enc, **fp)))
    acc, _, _ = hdc.train(H, ev.ytr, c.dim, ev.w.C, c.epochs)
    m = hdc.Model(Bt, hdc.ApproxConfig(enc=c.enc, class_bits=c.bits, perf_start=c.start, perf_end=c.end,
                                       perf_stride=c.stride, float_query=c.query == "float", **fp), acc=acc)
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
    fl = [c for c in cs if c.query == "float"]
    picks = [s.best, s.baseline] + [cs[i] for i in rng.choice(len(cs), 6, replace=False)] + fl[:3]
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


def test_cluster_tuner_nmi_equals_direct_run(ev):
    """Clustering candidates: the evaluator's NMI equals encoding and
    clustering the configuration directly through the ABI, and its graph
    replay gives the same labels as the eager run."""
    from paper_2606_26547_gb300 import cluster, hdc, metrics, synth, tuner as T
    w = synth.Workload("ctest", 300, 512, 8, 0, 1200, "gauss", 2.5, 6, 8100)
    cev = T.ClusterEvaluator(w)
    s = T.Search(T.ClusterSpace("full", 512, 6, dim_levels=3), cev, T.cluster_baseline(512, 6), seed=2, batch=12)
    s.run(evaluations=40)
    assert s.feasible(s.best) and s.report()["speedup"] >= 1.0
    run = cluster.ClusterRun(w)
    for c in list(s.results)[:6] + [s.best]:
        Bt = run.Bt[:c.dim]
        H = hdc.encode(run.X, hdc.Model(Bt, hdc.ApproxConfig(enc=c.enc)))
        sim = lambda a, e, st: hdc.ApproxConfig(perf_start=a, perf_end=e, perf_stride=st)
        lab, _, _, _ = hdc.cluster(H, c.dim, H[run.init_idx].contiguous(), c.iters,
                                   sim(c.t_start, c.t_end, c.t_stride), sim(c.i_start, c.i_end, c.i_stride))
        assert s.results[c].accuracy == metrics.nmi(run.y, lab.cpu().numpy()), c
    ms, nmi = run.graph_ms(cev._cc(s.best), reps=2)
    assert ms > 0 and nmi == s.results[s.best].accuracy


def test_tuner_levelid_candidates_equal_one_by_one():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import synth, tuner as T
    w = synth.Workload("tune_lid", 200, 1024, 6, 1500, 800, "gauss", 2.0, 3, 7300)
    ev = T.GpuEvaluator(w, 3, (1024, 512), reps=2, encs=("fp8", "lid16", "lid128"))
    space = T.Space("full", 1024, 3, dim_levels=2, levelid=True)
    space.values["enc"] = ("fp8", "lid16", "lid128")
    space.sizes = tuple(len(space.values[k]) for k in space.KNOBS)
    s = T.Search(space, ev, T.Config("fp8", 1024, 3, 0.0, 1.0, 1, 8, "float"), seed=3, batch=24)
    s.run(evaluations=120)
    lid = [c for c in s.results if T.lid_levels(c.enc)]
    assert all(space.contains(c) for c in lid)
    assert len(lid) >= 5
    for c in lid[:6]:
        assert s.results[c].accuracy == one_by_one(ev, c), c
        assert s.results[c].ms > 0


def test_tuner_full_nohint_perforates_the_encoding(ev):
    """Mode (1): candidates with a perforated encoding are trained on
    demand; their accuracies equal the same configurations run one by one."""
    from paper_2606_26547_gb300 import tuner as T
    space = T.Space("full_nohint", 1024, 4, dim_levels=3)
    s = T.Search(space, ev, T.baseline_config(1024, 4), seed=11, batch=24)
    s.run(evaluations=100)
    perf = [c for c in s.results if c.fperf() != T.NO_FPERF]
    assert len(perf) >= 10 and ev.families_built > 9
    for c in perf[:5]:
        assert s.results[c].accuracy == one_by_one(ev, c), c
