"""Batched approximation sweep: many candidate configurations in one launch.

The paper's tuner (Sec. 3) proposes approximation configurations, compiles
and runs the application for each, and reads back its QoS (accuracy). Here
the candidate evaluations of one tuning round run as ONE replay of a CUDA
graph on the GPU:

* one model per (seed, encoding element type): base hypermatrix drawn with
  the seed, training set encoded with that element type, bundling + the
  retraining epochs (TRAIN_ITERATIONS);
* the validation queries are encoded once per model at the full D
  (hdc_encode), then hdc_sweep_eval scores every (class width x perforation
  stride) configuration of that model from those hypervectors;
* all encodes and sweep evaluations are captured in one CUDA graph.

The sweep kernel's launch shape (threads per block, words per shared-memory
chunk) is picked by ``autotune.tune_sweep``; results do not depend on it.
Single-configuration graphs (hdc_classify with a model prepared for one
configuration) are timed for comparison.
"""
from __future__ import annotations

import dataclasses
import json
import time

import numpy as np
import torch

from . import autotune, hdc, synth

ENCS = ("fp32", "bf16", "fp8")
STRIDES = (1, 2, 4, 8)
BITS = (1, 4, 8)


@dataclasses.dataclass
class SweepModel:
    seed: int
    enc: str
    Bt: torch.Tensor
    acc: torch.Tensor
    base: hdc.Model          # base-only model for the full-D validation encode
    H: torch.Tensor          # N_val x W(D) validation hypervectors (graph output)
    ws: torch.Tensor         # encode workspace


def base_for_seed(w: synth.Workload, seed: int) -> np.ndarray:
    """Base hypermatrix of one tuning seed (seed stream 100*seed past the
    workload's own streams)."""
    return synth.base_gauss(w.D, w.F, w.seed + 3 + 100 * seed)


def train_models(workload: str, seeds, encs, n_train: int, n_val: int, epochs: int, device) -> tuple:
    w = synth.WORKLOADS[workload]
    d = synth.make(w, n_train=n_train, n_query=n_val)
    Xtr = torch.from_numpy(d["Xtr"]).to(device)
    ytr = torch.from_numpy(d["ytr"]).to(device)
    Xv = torch.from_numpy(d["Xq"]).to(device)
    yv = torch.from_numpy(d["yq"]).to(device)
    models = []
    for seed in seeds:
        Bt = torch.from_numpy(base_for_seed(w, seed)).to(device)
        for enc in encs:
            base = hdc.Model(Bt, hdc.ApproxConfig(enc=enc))
            Htr = hdc.encode(Xtr, base)
            acc, _, _ = hdc.train(Htr, ytr, w.D, w.C, epochs)
            H = torch.empty((n_val, base.W), dtype=torch.int32, device=device)
            models.append(SweepModel(seed, enc, Bt, acc, base, H, base.workspace(n_val)))
    return models, Xv, yv, w


class BatchedSweep:
    """All models' validation encodes + configuration sweeps; capturable."""

    def __init__(self, models, Xv, yv, w, strides=STRIDES, bits=BITS, controls=True, tuned=(0, 0)):
        self.models, self.Xv, self.yv, self.w = models, Xv, yv, w
        self.strides, self.bits = tuple(strides), tuple(bits)
        N = Xv.shape[0]
        self.sweeps = [hdc.Sweep(w.D, w.C, strides, bits, N, Xv.device, *tuned) for _ in models]
        # controls: the first FP32 model against its unquantised accumulators
        self.control = None
        if controls:
            i = next(i for i, m in enumerate(models) if m.enc == "fp32")
            self.control = (i, hdc.Sweep(w.D, w.C, strides, (0,), N, Xv.device, *tuned))
        self.graph = None

    def run(self):
        for m, sw in zip(self.models, self.sweeps):
            hdc.encode(self.Xv, m.base, ws=m.ws, out=m.H)
            sw(m.H, self.yv, m.acc)
        if self.control:
            i, sw = self.control
            sw(self.models[i].H, self.yv, self.models[i].acc)

    def capture(self):
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            self.run()                       # warm-up outside the graph
        torch.cuda.current_stream().wait_stream(s)
        torch.cuda.synchronize()
        self.graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(self.graph):
            self.run()
        return self

    def replay(self):
        self.graph.replay()

    def results(self):
        N = self.Xv.shape[0]
        out = []
        for m, sw in zip(self.models, self.sweeps):
            c = sw.correct.cpu().numpy()
            for jb, b in enumerate(self.bits):
                for i, s in enumerate(self.strides):
                    out.append(dict(seed=m.seed, enc=m.enc, class_bits=b, stride=s, accuracy=float(c[jb, i]) / N))
        if self.control:
            i, sw = self.control
            c = sw.correct.cpu().numpy()
            for j, s in enumerate(self.strides):
                out.append(dict(seed=self.models[i].seed, enc=self.models[i].enc, class_bits=32, stride=s,
                                accuracy=float(c[0, j]) / N, control="unquantised int32 accumulators"))
        return out


def time_graph(replay, reps=10) -> float:
    """Median device time (ms) of a graph replay, CUDA events."""
    ts = []
    for _ in range(reps):
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        replay()
        b.record()
        b.synchronize()
        ts.append(a.elapsed_time(b))
    return float(np.median(ts))


def single_config_ms(m: SweepModel, Xv, enc: str, b: int, s: int, reps=5) -> float:
    """hdc_classify of one configuration, captured alone and replayed."""
    model = hdc.Model(m.Bt, hdc.ApproxConfig(enc=enc, class_bits=b, perf_stride=s), acc=m.acc)
    ws = model.workspace(Xv.shape[0])
    labels = torch.empty(Xv.shape[0], dtype=torch.int32, device=Xv.device)
    hdc.classify(Xv, model, ws=ws, labels=labels)
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g):
        hdc.classify(Xv, model, ws=ws, labels=labels)
    return time_graph(g.replay, reps)


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description=__doc__.split("\n")[0])
    ap.add_argument("--workload", default="sweep_F561_D10000_C6")
    ap.add_argument("--seeds", type=int, default=7)
    ap.add_argument("--n-train", type=int, default=10000)
    ap.add_argument("--epochs", type=int, default=10)
    ap.add_argument("--single", type=int, default=12, help="configurations timed alone (0 = all)")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    hdc.load()
    w = synth.WORKLOADS[a.workload]
    t = time.perf_counter()
    models, Xv, yv, w = train_models(a.workload, range(a.seeds), ENCS, a.n_train, w.n_query, a.epochs, dev)
    torch.cuda.synchronize()
    train_s = time.perf_counter() - t
    m0 = models[0]
    hdc.encode(Xv, m0.base, ws=m0.ws, out=m0.H)
    tuned = autotune.tune_sweep(m0.H, yv, m0.acc, w.D, w.C, STRIDES, BITS)
    bs = BatchedSweep(models, Xv, yv, w, tuned=tuned).capture()
    bs.replay()
    torch.cuda.synchronize()
    res = bs.results()
    graph_ms = time_graph(bs.replay)
    singles = []
    cfgs = [(m, b, s) for m in models for b in BITS for s in STRIDES]
    for m, b, s in (cfgs if a.single == 0 else cfgs[:a.single]):
        singles.append(dict(seed=m.seed, enc=m.enc, class_bits=b, stride=s,
                            ms=single_config_ms(m, Xv, m.enc, b, s)))
    n_cfg = len(res)
    mean_single = float(np.mean([x["ms"] for x in singles]))
    print(json.dumps({"workload": a.workload, "configs": n_cfg, "queries": int(Xv.shape[0]),
                      "graph_ms": graph_ms, "ms_per_config_batched": graph_ms / n_cfg,
                      "ms_per_config_alone": mean_single, "batched_speedup": mean_single * n_cfg / graph_ms,
                      "tuned_launch": {"block_threads": tuned[0], "words_per_chunk": tuned[1]},
                      "train_s": train_s, "results": res, "single_config": singles}))


if __name__ == "__main__":
    main()
