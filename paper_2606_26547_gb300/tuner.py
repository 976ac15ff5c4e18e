"""Approximation tuner over the batched evaluator (the paper's tuning loop,
Sec. 3 and Sec. 5.2), with every candidate scored on the GPU.

Knobs (Sec. 4.2, 4.3) as this library implements them:
  enc      the encoder: random projection with element type fp32, bf16 or
           fp8, or Level-ID with N_LEVELS levels ("lid<L>"; the encoder
           algorithmic choice and the N_LEVELS knob of Sec. 5.3)
  dim      encoding dimensionality D' in {D, D/2, D/4, ...} (global)
  epochs   TRAIN_ITERATIONS: retraining epochs after bundling (custom knob)
  start, end, stride
           red_perf of the inference similarity reduction
  bits     class hypervector width: 1 (Hamming) or 4 / 8 (cosine), the
           algorithmic choice and element type of the similarity
  query    binary (packed signs) or float (BF16 projections; cosine, so
           4 / 8-bit classes only): the algorithmic choice of Sec. 4.2
           between the float + cosine form and automatic binarization
The encoding's feature reduction is never perforated here: every space
carries the no-approx hint on the encoding.  The pruning modes of Sec. 5.2
therefore become: ``full`` (start, stride and end tunable; Full RedPerf
with the hint), ``end_only`` (start 0 and stride 1 fixed) and ``none``
(no perforation).

Search: an ensemble of techniques (uniform random, greedy uniform mutation,
normal mutation, differential evolution) chosen per proposal by an
area-under-curve bandit, the scheme OpenTuner's default meta-technique
follows; each run starts from the baseline configuration.  QoS is a
constraint: a configuration is feasible when its validation accuracy is
at least the baseline's minus ``qos_drop`` (0.05 in the paper's runs).
The objective is the application's time: training (encode the training
set, bundle, retrain) plus classifying the validation set, each part
measured with CUDA events.  Proposals are scored in batches: one
hdc_sweep_eval launch per trained snapshot (enc, dim, epochs) scores all
of the batch's perforation entries (up to six per launch) under every
class width at once.
"""
from __future__ import annotations

import collections
import ctypes
import dataclasses
import json
import math
import time

import numpy as np

ENCS = ("fp32", "bf16", "fp8")
LEVELS = (16, 32, 64, 128, 256, 512, 814)
LID_ENCS = tuple("lid%d" % L for L in LEVELS)


def lid_levels(enc: str) -> int:
    """N_LEVELS of a Level-ID encoder name, 0 for a random projection."""
    return int(enc[3:]) if enc.startswith("lid") else 0
STRIDES = (1, 2, 4, 8, 16, 32)
BITS = (1, 4, 8)
GRID = 100          # start / end fractions on a 1/GRID grid
MIN_SPAN = 5        # end - start >= MIN_SPAN / GRID
# Sec. 5.2's pruning modes: none = (3) No RedPerf, end_only = (2) End-only
# + hint, full = (4) Full RedPerf + hint, full_nohint = (1) Full RedPerf
# (the encoding's own reduction perforated too)
MODES = ("none", "end_only", "full", "full_nohint")


@dataclasses.dataclass(frozen=True, order=True)
class Config:
    enc: str
    dim: int
    epochs: int
    start: float
    end: float
    stride: int
    bits: int
    query: str = "binary"
    e_start: float = 0.0     # red_perf of the encoding's reduction over features
    e_end: float = 1.0
    e_stride: int = 1

    def fperf(self):
        return (self.e_start, self.e_end, self.e_stride)


NO_FPERF = (0.0, 1.0, 1)
QUERIES = ("binary", "float")


def perf_values(mode: str):
    """(starts, ends, strides) of one red_perf op under a pruning mode."""
    full = mode in ("full", "full_nohint")
    starts = tuple(i / GRID for i in range(GRID - MIN_SPAN + 1)) if full else (0.0,)
    ends = tuple(i / GRID for i in range(MIN_SPAN, GRID + 1)) if mode != "none" else (1.0,)
    strides = STRIDES if full else (1,)
    return starts, ends, strides


class Space:
    """The knobs of one pruning mode as index ranges; a point is a tuple of
    value indices in KNOBS order.  SPANS lists the (start, end) knob pairs of
    the red_perf ops, each of which must keep end - start >= MIN_SPAN/GRID."""
    KNOBS = ("enc", "dim", "epochs", "start", "end", "stride", "bits", "query", "e_start", "e_end", "e_stride")
    SPANS = (("start", "end"), ("e_start", "e_end"))
    CONFIG = Config

    def __init__(self, mode: str, D: int, max_epochs: int, dim_levels: int = 5, min_dim: int = 128,
                 levelid: bool = False):
        if mode not in MODES:
            raise ValueError(mode)
        self.mode = mode
        self.encs = ENCS + (LID_ENCS if levelid else ())
        self.values = self._values(mode, tuple(D >> k for k in range(dim_levels) if (D >> k) >= min_dim),
                                   max_epochs)
        self.sizes = tuple(len(self.values[k]) for k in self.KNOBS)

    def _values(self, mode, dims, max_epochs):
        starts, ends, strides = perf_values(mode)
        # the encoding's reduction is perforated only without the no-approx hint
        es, ee, est = perf_values("full") if mode == "full_nohint" else ((0.0,), (1.0,), (1,))
        return dict(enc=self.encs, dim=dims, epochs=tuple(range(max_epochs + 1)), start=starts, end=ends,
                    stride=strides, bits=BITS, query=QUERIES, e_start=es, e_end=ee, e_stride=est)

    def log10_size(self) -> float:
        return float(sum(math.log10(n) for n in self.sizes))

    def config(self, point):
        return self.CONFIG(*(self.values[k][i] for k, i in zip(self.KNOBS, point)))

    def point(self, c: Config):
        return tuple(self.values[k].index(getattr(c, k)) for k in self.KNOBS)

    def contains(self, c: Config) -> bool:
        try:
            self.point(c)
        except ValueError:
            return False
        return self.valid(c)

    def valid(self, c) -> bool:
        if getattr(c, "query", "binary") == "float" and c.bits == 1:
            return False     # a float query is compared by cosine only
        if lid_levels(c.enc) and (c.bits != 1 or getattr(c, "query", "binary") != "binary" or
                                  getattr(c, "e_start", 0.0) != 0.0 or getattr(c, "e_end", 1.0) != 1.0 or
                                  getattr(c, "e_stride", 1) != 1):
            return False     # Level-ID rows are binary, compared by Hamming, all features
        return all(round((getattr(c, e) - getattr(c, a)) * GRID) >= MIN_SPAN for a, e in self.SPANS)

    def repair(self, point):
        """Nearest valid point: per span, move end up (else start down)."""
        p = list(point)
        for a, e in self.SPANS:
            ks, ke = self.KNOBS.index(a), self.KNOBS.index(e)
            while round((self.values[e][p[ke]] - self.values[a][p[ks]]) * GRID) < MIN_SPAN:
                if p[ke] + 1 < self.sizes[ke]:
                    p[ke] += 1
                else:
                    p[ks] -= 1
        if "query" in self.KNOBS:
            kq, kb, ke = self.KNOBS.index("query"), self.KNOBS.index("bits"), self.KNOBS.index("enc")
            if lid_levels(self.values["enc"][p[ke]]):
                p[kq], p[kb] = self.values["query"].index("binary"), self.values["bits"].index(1)
                for k, v in (("e_start", 0.0), ("e_end", 1.0), ("e_stride", 1)):
                    p[self.KNOBS.index(k)] = self.values[k].index(v)
            elif self.values["query"][p[kq]] == "float" and self.values["bits"][p[kb]] == 1:
                p[kb] = self.values["bits"].index(8)
        return tuple(p)

    def random(self, rng):
        return self.repair(tuple(int(rng.integers(n)) for n in self.sizes))

    def all_points(self):
        for p in np.ndindex(*self.sizes):
            if self.valid(self.config(p)):
                yield tuple(int(i) for i in p)


@dataclasses.dataclass(frozen=True, order=True)
class ClusterCfg:
    enc: str
    dim: int
    iters: int
    t_start: float
    t_end: float
    t_stride: int
    i_start: float
    i_end: float
    i_stride: int


class ClusterSpace(Space):
    """HD-Clustering knobs: element type, D', TRAIN_ITERATIONS (K-means
    iterations, 1..max) and the red_perf of its two similarity ops, the
    assignment during training (t_*) and the final one (i_*)."""
    KNOBS = ("enc", "dim", "iters", "t_start", "t_end", "t_stride", "i_start", "i_end", "i_stride")
    SPANS = (("t_start", "t_end"), ("i_start", "i_end"))
    CONFIG = ClusterCfg

    def _values(self, mode, dims, max_epochs):
        starts, ends, strides = perf_values(mode)
        return dict(enc=ENCS, dim=dims, iters=tuple(range(1, max_epochs + 1)), t_start=starts, t_end=ends,
                    t_stride=strides, i_start=starts, i_end=ends, i_stride=strides)


# ------------------------------------------------------------ techniques
class Technique:
    name = "technique"

    def propose(self, space: Space, search: "Search", rng):
        raise NotImplementedError


class UniformRandom(Technique):
    name = "uniform_random"

    def propose(self, space, search, rng):
        return space.random(rng)


class GreedyMutation(Technique):
    """Copy the best point; each knob independently (at least one) takes a
    uniformly random value."""
    name = "greedy_mutation"

    def __init__(self, rate: float = 0.2):
        self.rate = rate

    def propose(self, space, search, rng):
        p = list(search.best_point)
        live = [k for k, n in enumerate(space.sizes) if n > 1]
        hit = [k for k in live if rng.random() < self.rate] or [live[int(rng.integers(len(live)))]]
        for k in hit:
            p[k] = int(rng.integers(space.sizes[k]))
        return space.repair(tuple(p))


class NormalMutation(Technique):
    """Copy the best point; each knob independently (at least one) moves by
    a normal step of sigma x its range, rounded and clipped."""
    name = "normal_mutation"

    def __init__(self, rate: float = 0.3, sigma: float = 0.1):
        self.rate, self.sigma = rate, sigma

    def propose(self, space, search, rng):
        p = list(search.best_point)
        live = [k for k, n in enumerate(space.sizes) if n > 1]
        hit = [k for k in live if rng.random() < self.rate] or [live[int(rng.integers(len(live)))]]
        for k in hit:
            n = space.sizes[k]
            step = int(round(rng.normal(0.0, max(self.sigma * n, 0.6))))
            p[k] = min(max(p[k] + (step or (1 if rng.random() < 0.5 else -1)), 0), n - 1)
        return space.repair(tuple(p))


class DifferentialEvolution(Technique):
    """x = a + F (b - c) over index vectors of three ranked points, crossed
    over with a fourth at rate CR (the population is the best ``pop``
    points seen)."""
    name = "differential_evolution"

    def __init__(self, pop: int = 30, F: float = 0.7, CR: float = 0.5):
        self.pop, self.F, self.CR = pop, F, CR

    def propose(self, space, search, rng):
        ranked = search.ranked_points(self.pop)
        if len(ranked) < 4:
            return space.random(rng)
        i = rng.choice(len(ranked), 4, replace=False)
        x, a, b, c = (ranked[j] for j in i)
        out = []
        kf = int(rng.integers(len(space.sizes)))
        for k, n in enumerate(space.sizes):
            if k == kf or rng.random() < self.CR:
                v = int(round(a[k] + self.F * (b[k] - c[k])))
                out.append(min(max(v, 0), n - 1))
            else:
                out.append(x[k])
        return space.repair(tuple(out))


class AUCBandit:
    """Technique choice by area under the curve of recent successes (a use
    scores 1 when its proposal became the new best) plus an exploration
    bonus C sqrt(2 ln T / n), over a sliding window of uses."""

    def __init__(self, techniques, C: float = 0.05, window: int = 500):
        self.techniques = list(techniques)
        self.C, self.window = C, window
        self.history = []   # (technique index, success)

    def _auc(self, k):
        uses = [s for t, s in self.history if t == k]
        if not uses:
            return 0.0
        # later successes weigh more: sum_i i * s_i normalised
        n = len(uses)
        return sum((i + 1) * s for i, s in enumerate(uses)) * 2.0 / (n * (n + 1))

    def choose(self, rng) -> int:
        T = len(self.history)
        best, bv = 0, -1.0
        for k in range(len(self.techniques)):
            n = sum(1 for t, _ in self.history if t == k)
            if n == 0:
                return k
            v = self._auc(k) + self.C * math.sqrt(2.0 * math.log(T) / n)
            if v > bv:
                best, bv = k, v
        return best

    def credit(self, k: int, success: bool) -> None:
        self.history.append((k, 1 if success else 0))
        if len(self.history) > self.window:
            self.history.pop(0)


# ---------------------------------------------------------------- search
@dataclasses.dataclass
class Result:
    accuracy: float
    ms: float


class Search:
    """Constrained minimisation of ms subject to accuracy >= target."""

    def __init__(self, space: Space, evaluate, baseline: Config, qos_drop: float = 0.05, seed: int = 0,
                 batch: int = 36, techniques=None):
        self.space, self.evaluate = space, evaluate
        self.rng = np.random.default_rng(seed)
        self.batch = batch
        self.bandit = AUCBandit(techniques or [UniformRandom(), GreedyMutation(), NormalMutation(),
                                               DifferentialEvolution()])
        self.results = {}   # Config -> Result
        got = evaluate([baseline])
        self.results.update(got)
        base = got[baseline]
        self.baseline, self.base_result = baseline, base
        self.target = base.accuracy - qos_drop
        self.best = baseline
        self.best_point = space.point(baseline) if space.contains(baseline) else space.random(self.rng)
        self.trace = [(1, 0.0, 1.0)]   # (evaluations, seconds, running-best speedup)
        self.t0 = time.perf_counter()

    def feasible(self, c: Config) -> bool:
        return self.results[c].accuracy >= self.target

    def fitness(self, c: Config):
        r = self.results[c]
        return (0, r.ms) if r.accuracy >= self.target else (1, self.target - r.accuracy)

    def ranked_points(self, n: int):
        cs = [c for c in self.results if self.space.contains(c)]
        cs.sort(key=self.fitness)
        return [self.space.point(c) for c in cs[:n]]

    def speedup(self, c: Config) -> float:
        return self.base_result.ms / self.results[c].ms

    def step(self) -> int:
        """One batch of proposals; returns the number of new evaluations."""
        props, used = [], []
        seen = set()
        for _ in range(self.batch * 4):
            if len(props) == self.batch:
                break
            k = self.bandit.choose(self.rng)
            c = self.space.config(self.bandit.techniques[k].propose(self.space, self, self.rng))
            if c in self.results or c in seen:
                self.bandit.credit(k, False)
                continue
            seen.add(c)
            props.append(c)
            used.append(k)
        if len(props) < self.batch and math.prod(self.space.sizes) <= 20000:
            # a small space whose proposals keep repeating: fill the batch
            # with points not yet evaluated
            rest = [c for c in map(self.space.config, self.space.all_points())
                    if c not in self.results and c not in seen]
            for i in self.rng.permutation(len(rest))[:self.batch - len(props)]:
                seen.add(rest[i])
                props.append(rest[i])
                used.append(0)   # credited to uniform random
        if not props:
            return 0
        got = self.evaluate(props)
        for c, r in got.items():
            self.results[c] = r
        for c, k in zip(props, used):
            better = self.feasible(c) and self.results[c].ms < self.results[self.best].ms
            if better:
                self.best = c
                self.best_point = self.space.point(c)
            self.bandit.credit(k, better)
        for c in got:   # extra configurations the batched evaluator scored
            if c not in seen and self.space.contains(c) and self.feasible(c) and \
                    self.results[c].ms < self.results[self.best].ms:
                self.best, self.best_point = c, self.space.point(c)
        self.trace.append((len(self.results), time.perf_counter() - self.t0, self.speedup(self.best)))
        return len(got)

    def run(self, evaluations: int | None = None, seconds: float | None = None):
        idle = 0
        while idle < 8:   # eight batches without a new point: the space is exhausted
            if evaluations is not None and len(self.results) >= evaluations:
                break
            if seconds is not None and time.perf_counter() - self.t0 >= seconds:
                break
            idle = idle + 1 if self.step() == 0 else 0
        return self

    def report(self) -> dict:
        b = self.best
        return {"mode": self.space.mode, "log10_space": round(self.space.log10_size(), 2),
                "evaluations": len(self.results), "seconds": round(time.perf_counter() - self.t0, 3),
                "baseline": dataclasses.asdict(self.baseline), "baseline_accuracy": self.base_result.accuracy,
                "baseline_ms": self.base_result.ms, "qos_target": self.target,
                "best": dataclasses.asdict(b), "best_accuracy": self.results[b].accuracy,
                "best_ms": self.results[b].ms, "speedup": self.speedup(b),
                "techniques": {t.name: sum(1 for k, _ in self.bandit.history if k == i)
                               for i, t in enumerate(self.bandit.techniques)},
                "running_best": [list(map(lambda v: round(v, 4), t)) for t in _thin(self.trace, 24)]}


def _thin(trace, n):
    if len(trace) <= n:
        return trace
    idx = sorted(set(np.linspace(0, len(trace) - 1, n).round().astype(int).tolist()))
    return [trace[i] for i in idx]


# ---------------------------------------------------------- GPU evaluator
class GpuEvaluator:
    """Trained snapshots per (enc, dim, epochs), validation hypervectors per
    (enc, dim), and measured cost tables; scores configurations through
    hdc_sweep_eval and prices them from the tables."""

    def __init__(self, workload: str, max_epochs: int, dims, n_train=None, n_val=None, device="cuda",
                 reps: int = 5, encs=ENCS):
        import torch
        from . import hdc, synth
        self.torch, self.hdc, self.encs = torch, hdc, tuple(encs)
        self.w = w = synth.WORKLOADS[workload] if isinstance(workload, str) else workload
        d = synth.make(w, n_train=n_train, n_query=n_val)
        dev = torch.device(device)
        self.dev, self.reps = dev, reps
        self.Bt = torch.from_numpy(d["Bt"]).to(dev)
        self.Xtr = torch.from_numpy(d["Xtr"]).to(dev)
        self.ytr = torch.from_numpy(d["ytr"]).to(dev)
        self.Xv = torch.from_numpy(d["Xq"]).to(dev)
        self.yv = torch.from_numpy(d["yq"]).to(dev)
        # Level-ID: the caller's draws (ID rows, level end points, flip levels
        # per N_LEVELS) and the feature range of the training set
        self.lid = {}
        self.x_lo, self.x_hi = float(d["Xtr"].min()), float(d["Xtr"].max())
        for enc in self.encs:
            if lid_levels(enc):
                self.lid[enc] = tuple(torch.from_numpy(a).to(dev)
                                      for a in synth.levelid_hvs(w.F, w.D, lid_levels(enc), w.seed))
        self.max_epochs, self.dims = max_epochs, tuple(dims)
        # per family (enc, dim, feature perforation): the accumulators after
        # each epoch, the validation hypervectors and the measured training
        # times; families with a perforated encoding are built on first use
        # and the least recently used of them dropped past `max_families`
        self.fam = collections.OrderedDict()
        self.max_families = 96
        self.t_classify = {}
        self.sweep_launches = 0
        self.families_built = 0
        for enc in self.encs:
            for dim in self.dims:
                self._family((enc, dim, NO_FPERF), pin=True)
        torch = self.torch
        torch.cuda.synchronize()

    def _ms(self, fn) -> float:
        torch = self.torch
        fn()
        ts = []
        for _ in range(self.reps):
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        return float(np.median(ts))

    def _lid_model(self, enc: str, dim: int, cfg=None):
        ids, lo, hi, flip = self.lid[enc]
        return self.hdc.LevelIdModel(ids[:, :dim].contiguous(), lo[:dim].contiguous(), hi[:dim].contiguous(),
                                     flip[:dim].contiguous(), lid_levels(enc), self.x_lo, self.x_hi, cfg)

    def _rp_cfg(self, enc: str, fperf, **kw):
        return self.hdc.ApproxConfig(enc=enc, enc_perf_start=fperf[0], enc_perf_end=fperf[1],
                                     enc_perf_stride=fperf[2], **kw)

    def _encoder(self, enc: str, dim: int, N: int, fperf=NO_FPERF):
        """(encode(X, out) for N rows at D' = dim, words per row)."""
        hdc = self.hdc
        if lid_levels(enc):
            m = self._lid_model(enc, dim)
            return (lambda X, out: hdc.levelid_encode(X, m, out=out)), m.W
        base = hdc.Model(self.Bt[:dim], self._rp_cfg(enc, fperf))
        ws = base.workspace(N)
        return (lambda X, out: hdc.encode(X, base, ws=ws, out=out)), base.W

    def _family(self, key, pin: bool = False) -> dict:
        """Train the family (enc, dim, fperf) as the application runs it --
        bundling, then every epoch, each pass timed and the accumulators kept
        after each -- and encode the validation set."""
        if key in self.fam:
            self.fam.move_to_end(key)
            return self.fam[key]
        torch, hdc, w = self.torch, self.hdc, self.w
        enc, dim, fperf = key
        N = self.Xtr.shape[0]
        encf, W = self._encoder(enc, dim, N, fperf)
        Htr = torch.empty((N, W), dtype=torch.int32, device=self.dev)
        f = {"pin": pin, "t_encode": self._ms(lambda: encf(self.Xtr, Htr)), "snap": [], "t_train": []}
        n = ctypes.c_size_t()
        hdc._call("hdc_train_workspace_bytes", N, dim, w.C, ctypes.byref(n))
        tws = hdc._empty_bytes(n.value, self.dev)
        acc = torch.empty((w.C, dim), dtype=torch.int32, device=self.dev)
        cls = torch.empty((w.C, hdc.words(dim)), dtype=torch.int32, device=self.dev)
        for rep in range(2):   # the first run warms up
            times = []
            for ep in range(self.max_epochs + 1):
                a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                a.record()
                hdc.train_epoch(Htr, self.ytr, dim, w.C, 0 if ep == 0 else 1, acc, cls, ws=tws)
                b.record()
                if rep:
                    f["snap"].append(acc.clone())
                times.append((a, b))
            torch.cuda.synchronize()
        f["t_train"] = [float(v) for v in np.cumsum([a.elapsed_time(b) for a, b in times])]
        encv, _ = self._encoder(enc, dim, self.Xv.shape[0], fperf)
        f["Hv"] = torch.empty((self.Xv.shape[0], W), dtype=torch.int32, device=self.dev)
        encv(self.Xv, f["Hv"])
        self.fam[key] = f
        self.families_built += 1
        while len(self.fam) > self.max_families:   # drop the least recently used unpinned family
            victim = next((k for k, v in self.fam.items() if not v["pin"]), None)
            if victim is None:
                break
            del self.fam[victim]
        return f

    @staticmethod
    def _key(c: Config):
        return (c.enc, c.dim, c.fperf())

    def classify_ms(self, c: Config) -> float:
        hdc, torch = self.hdc, self.torch
        if lid_levels(c.enc):
            # Level-ID encode of the kept dims + Hamming arg-min over them
            cfg = hdc.ApproxConfig(perf_start=c.start, perf_end=c.end, perf_stride=c.stride)
            Dk = hdc.kept_dims(c.dim, cfg)
            key = (c.enc, Dk, 1, "binary", self.w.F)
            if key not in self.t_classify:
                m = self._lid_model(c.enc, c.dim, cfg)
                H = torch.empty((self.Xv.shape[0], m.W), dtype=torch.int32, device=self.dev)
                cls = torch.zeros((self.w.C, m.W), dtype=torch.int32, device=self.dev)
                self.t_classify[key] = self._ms(lambda: (hdc.levelid_encode(self.Xv, m, out=H),
                                                         hdc.hamming_argmin(H, cls, Dk)))
            return self.t_classify[key]
        cfg = self._rp_cfg(c.enc, c.fperf(), class_bits=c.bits, perf_start=c.start, perf_end=c.end,
                           perf_stride=c.stride, float_query=c.query == "float")
        fam = self._family(self._key(c))
        model = None
        Dk = hdc.kept_dims(c.dim, cfg)
        Fk = len(range(int(np.floor(np.float64(np.float32(c.e_start)) * self.w.F)),
                       int(np.floor(np.float64(np.float32(c.e_end)) * self.w.F)), c.e_stride))
        key = (c.enc, Dk, c.bits, c.query, Fk)
        if key not in self.t_classify:
            model = hdc.Model(self.Bt[:c.dim], cfg, acc=fam["snap"][0])
            ws = model.workspace(self.Xv.shape[0])
            lab = torch.empty(self.Xv.shape[0], dtype=torch.int32, device=self.dev)
            self.t_classify[key] = self._ms(lambda: hdc.classify(self.Xv, model, ws=ws, labels=lab))
        return self.t_classify[key]

    def ms(self, c: Config) -> float:
        fam = self._family(self._key(c))
        return fam["t_encode"] + fam["t_train"][c.epochs] + self.classify_ms(c)

    def float_accuracy(self, c: Config) -> float:
        """A float-query candidate: classify the validation set with a model
        prepared for it (the sweep scores binary queries only)."""
        hdc = self.hdc
        cfg = self._rp_cfg(c.enc, c.fperf(), class_bits=c.bits, perf_start=c.start, perf_end=c.end,
                           perf_stride=c.stride, float_query=True)
        model = hdc.Model(self.Bt[:c.dim], cfg, acc=self._family(self._key(c))["snap"][c.epochs])
        lab = hdc.classify(self.Xv, model)
        return float((lab == self.yv).sum().item()) / self.Xv.shape[0]

    def accuracy(self, configs) -> dict:
        """Accuracy of every (entry, width) the batch's sweeps score: the
        proposals and, for free, their entries under the other widths;
        float-query proposals one by one."""
        hdc = self.hdc
        N = self.Xv.shape[0]
        out = {c: self.float_accuracy(c) for c in configs if c.query == "float"}
        groups = {}
        for c in configs:
            if c.query == "float":
                continue
            groups.setdefault((self._key(c), c.epochs), set()).add((c.start, c.end, c.stride))
        pending = []
        for (key, ep), entries in groups.items():
            fam = self._family(key)
            entries = sorted(entries)
            for i in range(0, len(entries), 6):
                chunk = entries[i:i + 6]
                sw = hdc.Sweep(key[1], self.w.C, [e[2] for e in chunk], BITS, N, self.dev,
                               starts=[e[0] for e in chunk], ends=[e[1] for e in chunk])
                sw(fam["Hv"], self.yv, fam["snap"][ep])
                self.sweep_launches += 1
                pending.append((key, ep, chunk, sw.correct))
        for (enc, dim, fperf), ep, chunk, corr in pending:
            corr = corr.cpu().numpy()
            for jb, b in enumerate(BITS):
                if lid_levels(enc) and b != 1:
                    continue   # Level-ID candidates are Hamming only
                for j, (s, e, st) in enumerate(chunk):
                    out[Config(enc, dim, ep, s, e, st, b, "binary", *fperf)] = float(corr[jb, j]) / N
        return out

    def __call__(self, configs) -> dict:
        acc = self.accuracy(configs)
        return {c: Result(a, self.ms(c)) for c, a in acc.items()}


class ClusterEvaluator:
    """HD-Clustering candidates: each is encoded and clustered through
    hdc_cluster (K-means iterations cannot share one launch the way the
    classification sweep does); QoS = NMI; time = one CUDA-graph replay of
    encode + clustering, measured once per (enc, D', iterations, kept dims
    of both similarity ops)."""

    def __init__(self, workload: str = "cluster_F617_D1024_K26", device="cuda"):
        from . import cluster
        self.cl = cluster
        self.run = cluster.ClusterRun(workload, device)
        self.t = {}
        self.runs = 0

    def _cc(self, c: ClusterCfg):
        return self.cl.ClusterConfig(c.enc, c.dim, c.iters, (c.t_start, c.t_end, c.t_stride),
                                     (c.i_start, c.i_end, c.i_stride))

    def ms(self, c: ClusterCfg) -> float:
        from . import hdc
        kt = hdc.kept_dims(c.dim, hdc.ApproxConfig(perf_start=c.t_start, perf_end=c.t_end, perf_stride=c.t_stride))
        ki = hdc.kept_dims(c.dim, hdc.ApproxConfig(perf_start=c.i_start, perf_end=c.i_end, perf_stride=c.i_stride))
        key = (c.enc, c.dim, c.iters, kt, ki)
        if key not in self.t:
            self.t[key] = self.run.graph_ms(self._cc(c), reps=3)[0]
        return self.t[key]

    def __call__(self, configs) -> dict:
        out = {}
        for c in configs:
            out[c] = Result(self.run.run(self._cc(c))["nmi"], self.ms(c))
            self.runs += 1
        return out


def cluster_baseline(D: int, max_iters: int) -> ClusterCfg:
    """The unapproximated clustering: FP32 encoding at the full D, every
    iteration, no perforation of either similarity op."""
    return ClusterCfg("fp32", D, max_iters, 0.0, 1.0, 1, 0.0, 1.0, 1)


def baseline_config(D: int, max_epochs: int) -> Config:
    """The unapproximated application, the paper's float + cosine form: fp32
    encoding at the full D, every retraining epoch, no perforation, float
    query hypervectors, cosine against the widest class width (8 bits)."""
    return Config("fp32", D, max_epochs, 0.0, 1.0, 1, 8, "float")


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="approximation tuner over the batched evaluator")
    ap.add_argument("--app", default="classify", choices=["classify", "cluster"])
    ap.add_argument("--workload", default=None, help="default: classify_F617_D2048_C26 / cluster_F617_D1024_K26")
    ap.add_argument("--epochs", type=int, default=None,
                    help="TRAIN_ITERATIONS of the baseline (the knob's max; default: the workload's)")
    ap.add_argument("--qos-drop", type=float, default=0.05)
    ap.add_argument("--evaluations", type=int, default=3000, help="budget per pruning mode")
    ap.add_argument("--seconds", type=float, default=None, help="time budget per pruning mode")
    ap.add_argument("--modes", default=",".join(MODES))
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--levelid", action="store_true", help="add the Level-ID encoder (N_LEVELS knob)")
    a = ap.parse_args(argv)
    from . import hdc, synth
    hdc.load()
    wl = a.workload or ("classify_F617_D2048_C26" if a.app == "classify" else "cluster_F617_D1024_K26")
    w = synth.WORKLOADS[wl]
    epochs = a.epochs if a.epochs is not None else w.epochs
    t = time.perf_counter()
    if a.app == "classify":
        dims = Space("none", w.D, epochs).values["dim"]
        ev = GpuEvaluator(wl, epochs, dims, encs=ENCS + (LID_ENCS if a.levelid else ()))
        space_cls, base = (lambda m, D, e: Space(m, D, e, levelid=a.levelid)), baseline_config(w.D, epochs)
    else:
        ev = ClusterEvaluator(wl)
        space_cls, base = ClusterSpace, cluster_baseline(w.D, epochs)
    prep = time.perf_counter() - t
    reports = []
    for mode in a.modes.split(","):
        s = Search(space_cls(mode, w.D, epochs), ev, base, a.qos_drop, a.seed)
        reports.append(s.run(a.evaluations, a.seconds).report())
    extra = ({"sweep_launches": ev.sweep_launches, "classify_cost_entries": len(ev.t_classify),
              "trained_families": ev.families_built}
             if a.app == "classify" else {"cluster_runs": ev.runs, "graph_cost_entries": len(ev.t)})
    print(json.dumps({"app": a.app, "workload": wl, "prepare_s": round(prep, 3), **extra, "modes": reports}))


if __name__ == "__main__":
    main()
