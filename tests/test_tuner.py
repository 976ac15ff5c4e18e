"""Approximation tuner (search-space pruning modes, techniques, the bandit
and the constrained search) on the CPU with a synthetic evaluator whose
optimum is known by enumeration."""
import math

import numpy as np
import pytest

from paper_2606_26547_gb300 import tuner as T


def fake_eval(c: T.Config):
    """Accuracy falls with fewer dims, fewer epochs, narrower classes and
    fewer kept dims; time grows with the kept dims and the epochs."""
    kept = (c.end - c.start) / c.stride
    acc = 0.9 - 0.02 * math.log2(10000 / c.dim) - 0.01 * (10 - c.epochs) - 0.015 * (c.bits == 1) \
        - 0.08 * (1 - kept) ** 2 - 0.005 * {"fp32": 0, "bf16": 1, "fp8": 2}[c.enc] \
        + 0.01 * (c.query == "float")
    ms = 5.0 * {"fp32": 3, "bf16": 1.5, "fp8": 1}[c.enc] * c.dim / 10000 + 0.3 * c.epochs \
        + 2.0 * kept * c.dim / 10000 * (0.5 if c.bits == 1 else 1.0) + 1.5 * (c.query == "float")
    return T.Result(acc, ms)


class Counting:
    def __init__(self):
        self.calls = 0
        self.configs = 0

    def __call__(self, configs):
        self.calls += 1
        self.configs += len(configs)
        return {c: fake_eval(c) for c in configs}


def brute_best(space, target):
    best = None
    for p in space.all_points():
        c = space.config(p)
        r = fake_eval(c)
        if r.accuracy >= target and (best is None or r.ms < fake_eval(best).ms):
            best = c
    return best


def test_space_sizes_and_round_trip():
    full, end, none = (T.Space(m, 10000, 10) for m in ("full", "end_only", "none"))
    assert none.values["dim"] == (10000, 5000, 2500, 1250, 625)
    assert none.sizes == (3, 5, 11, 1, 1, 1, 3, 2, 1, 1, 1)
    assert end.sizes[T.Space.KNOBS.index("end")] == 96 and end.sizes[T.Space.KNOBS.index("stride")] == 1
    assert full.log10_size() > end.log10_size() > none.log10_size()
    rng = np.random.default_rng(1)
    for _ in range(500):
        p = full.random(rng)
        c = full.config(p)
        assert full.valid(c) and full.point(c) == p and full.contains(c)
    assert not full.valid(T.Config("fp8", 10000, 0, 0.5, 0.52, 1, 1))
    assert not full.valid(T.Config("fp8", 10000, 0, 0.0, 1.0, 1, 1, "float"))   # float queries: cosine only
    assert full.config(full.repair(full.point(T.Config("fp8", 10000, 0, 0.0, 1.0, 1, 8, "float")))).bits == 8
    assert full.valid(full.config(full.repair(full.point(T.Config("fp8", 10000, 0, 0.95, 0.96, 1, 1)))))


@pytest.mark.parametrize("tech", [T.UniformRandom(), T.GreedyMutation(), T.NormalMutation(),
                                  T.DifferentialEvolution()])
def test_techniques_stay_in_space(tech):
    space = T.Space("full", 10000, 10)
    s = T.Search(space, Counting(), T.baseline_config(10000, 10), seed=3, batch=8)
    s.run(evaluations=120)
    rng = np.random.default_rng(0)
    for _ in range(300):
        p = tech.propose(space, s, rng)
        assert len(p) == len(space.sizes) and all(0 <= i < n for i, n in zip(p, space.sizes))
        assert space.valid(space.config(p))


def test_bandit_prefers_the_technique_that_succeeds():
    b = T.AUCBandit([T.UniformRandom(), T.GreedyMutation()])
    rng = np.random.default_rng(0)
    for _ in range(200):
        k = b.choose(rng)
        b.credit(k, k == 1)
    uses = [sum(1 for t, _ in b.history if t == k) for k in range(2)]
    assert uses[1] > 3 * uses[0]


def test_search_exhausts_small_space_and_finds_optimum():
    space = T.Space("none", 10000, 10)
    ev = Counting()
    s = T.Search(space, ev, T.baseline_config(10000, 10), qos_drop=0.05, seed=0, batch=16)
    s.run(evaluations=10_000)
    n_valid = sum(1 for _ in space.all_points())
    assert sum(1 for c in s.results if space.contains(c)) == n_valid
    want = brute_best(space, s.target)
    assert fake_eval(s.best).ms == pytest.approx(fake_eval(want).ms)
    assert s.feasible(s.best)


def test_running_best_is_monotone_and_feasible():
    space = T.Space("full", 10000, 10)
    s = T.Search(space, Counting(), T.baseline_config(10000, 10), seed=7)
    s.run(evaluations=1500)
    sp = [t[2] for t in s.trace]
    assert sp[0] == 1.0 and all(b >= a for a, b in zip(sp, sp[1:]))
    assert s.feasible(s.best) and s.results[s.best].accuracy >= s.target
    assert all(not (s.feasible(c) and s.results[c].ms < s.results[s.best].ms) for c in s.results)
    rep = s.report()
    assert rep["speedup"] == pytest.approx(sp[-1]) and rep["speedup"] > 1.5
    assert set(rep["techniques"]) == {"uniform_random", "greedy_mutation", "normal_mutation",
                                      "differential_evolution"}


def test_end_only_never_moves_start_or_stride():
    space = T.Space("end_only", 10000, 10)
    s = T.Search(space, Counting(), T.baseline_config(10000, 10), seed=2)
    s.run(evaluations=400)
    for c in s.results:
        if space.contains(c):
            assert c.start == 0.0 and c.stride == 1


def test_cluster_space_spans_and_modes():
    for mode, n_perf in (("none", 1), ("end_only", 96), ("full", None)):
        sp = T.ClusterSpace(mode, 1024, 20)
        assert sp.values["iters"] == tuple(range(1, 21))
        assert sp.values["dim"] == (1024, 512, 256, 128)
        if n_perf:
            assert len(sp.values["t_end"]) == len(sp.values["i_end"]) == n_perf
    sp = T.ClusterSpace("full", 1024, 20)
    rng = np.random.default_rng(4)
    for _ in range(300):
        c = sp.config(sp.random(rng))
        assert sp.valid(c) and c.t_end - c.t_start >= 0.049 and c.i_end - c.i_start >= 0.049
    base = T.cluster_baseline(1024, 20)
    assert sp.contains(base) and T.ClusterSpace("none", 1024, 20).contains(base)


def test_cluster_search_with_fake_evaluator():
    def ev(configs):
        out = {}
        for c in configs:
            kt = (c.t_end - c.t_start) / c.t_stride
            nmi = 0.8 - 0.03 * (20 - c.iters) / 20 - 0.1 * (1 - kt) ** 2 - 0.05 * (1 - c.i_end) \
                - 0.04 * math.log2(1024 / c.dim)
            ms = 0.1 * c.iters * kt * c.dim / 1024 + {"fp32": 0.3, "bf16": 0.1, "fp8": 0.08}[c.enc]
            out[c] = T.Result(nmi, ms)
        return out
    s = T.Search(T.ClusterSpace("end_only", 1024, 20), ev, T.cluster_baseline(1024, 20), seed=1)
    s.run(evaluations=800)
    assert s.feasible(s.best) and s.report()["speedup"] > 3


def test_levelid_encoders_are_binary_hamming_only():
    sp = T.Space("full", 2048, 10, levelid=True)
    assert set(T.LID_ENCS) <= set(sp.values["enc"]) and T.lid_levels("lid128") == 128 and T.lid_levels("fp8") == 0
    assert not sp.valid(T.Config("lid64", 2048, 3, 0.0, 1.0, 1, 8, "binary"))
    assert not sp.valid(T.Config("lid64", 2048, 3, 0.0, 1.0, 1, 1, "float"))
    rng = np.random.default_rng(6)
    seen = 0
    for _ in range(2000):
        c = sp.config(sp.random(rng))
        assert sp.valid(c)
        if T.lid_levels(c.enc):
            seen += 1
            assert c.bits == 1 and c.query == "binary"
    assert seen > 500
    assert "lid16" not in T.Space("full", 2048, 10).values["enc"]


def test_full_nohint_adds_encoding_perforation_knobs():
    full, nohint = T.Space("full", 2048, 10), T.Space("full_nohint", 2048, 10)
    assert full.values["e_start"] == (0.0,) and full.values["e_end"] == (1.0,) and full.values["e_stride"] == (1,)
    assert len(nohint.values["e_end"]) == 96 and nohint.log10_size() > full.log10_size()
    rng = np.random.default_rng(1)
    for _ in range(500):
        c = nohint.config(nohint.random(rng))
        assert nohint.valid(c) and c.e_end - c.e_start >= 0.049
    lid = T.Space("full_nohint", 2048, 10, levelid=True)
    for _ in range(500):
        c = lid.config(lid.random(rng))
        if T.lid_levels(c.enc):
            assert c.fperf() == T.NO_FPERF
