"""HD-Clustering driver (Sec. 5.1 / 5.2): encode every point, run K-means
over the binary hypervectors (hdc_cluster), score the clusters by NMI.

Knobs: element type of the encoding, dimensionality D' (first D' rows of
the base hypermatrix), TRAIN_ITERATIONS (K-means iterations), and the two
independently perforated similarity ops (assignment during training,
final assignment at inference).  graph_ms times a configuration as one CUDA
graph (the tuner's application time); bench_kernels.py's `cluster`
subcommand reports a set of configurations."""
from __future__ import annotations

import dataclasses
import json

import numpy as np
import torch

from . import hdc, metrics, synth


@dataclasses.dataclass(frozen=True)
class ClusterConfig:
    enc: str = "fp32"
    dim: int = 1024
    iters: int = 20
    train_perf: tuple = (0.0, 1.0, 1)
    infer_perf: tuple = (0.0, 1.0, 1)


def sim_config(p):
    """The perforation (start, end, stride) of a similarity op as a config."""
    return hdc.ApproxConfig(perf_start=p[0], perf_end=p[1], perf_stride=p[2])


class ClusterRun:
    """Device-resident points of one workload; run(cfg) encodes and clusters."""

    def __init__(self, workload: str = "cluster_F617_D1024_K26", device="cuda"):
        self.w = w = synth.WORKLOADS[workload] if isinstance(workload, str) else workload
        d = synth.make(w)
        self.dev = torch.device(device)
        self.Bt = torch.from_numpy(d["Bt"]).to(self.dev)
        self.X = torch.from_numpy(d["Xq"]).to(self.dev)
        self.y = d["yq"]
        self.init_idx = torch.from_numpy(synth.cluster_init(self.X.shape[0], w.C, w.seed)).to(self.dev)
        self._models = {}

    def model(self, enc: str, dim: int):
        key = (enc, dim)
        if key not in self._models:
            m = hdc.Model(self.Bt[:dim], hdc.ApproxConfig(enc=enc))
            self._models[key] = (m, m.workspace(self.X.shape[0]))
        return self._models[key]

    def run(self, c: ClusterConfig, timed: bool = False):
        m, ws = self.model(c.enc, c.dim)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(3)] if timed else None
        if timed:
            ev[0].record()
        H = hdc.encode(self.X, m, ws=ws)
        if timed:
            ev[1].record()
        init = H[self.init_idx].contiguous()
        lab, cls, acc, changes = hdc.cluster(H, c.dim, init, c.iters, sim_config(c.train_perf), sim_config(c.infer_perf))
        if timed:
            ev[2].record()
        lab = lab.cpu().numpy()
        out = {"nmi": metrics.nmi(self.y, lab), "changes": changes.cpu().numpy().tolist()}
        if timed:
            out["encode_ms"] = ev[0].elapsed_time(ev[1])
            out["cluster_ms"] = ev[1].elapsed_time(ev[2])
        return out

    def graph_ms(self, c: ClusterConfig, reps: int = 20):
        """Encode + cluster captured in one CUDA graph (the per-iteration
        launches then cost no host time): the tuner's application time for
        a clustering configuration.  Returns (ms per replay, NMI)."""
        m, ws = self.model(c.enc, c.dim)
        self.run(c)   # warm-up: lazy module loads and kernel attributes
        torch.cuda.synchronize()
        g = torch.cuda.CUDAGraph()
        s = torch.cuda.Stream()
        s.wait_stream(torch.cuda.current_stream())
        with torch.cuda.stream(s):
            with torch.cuda.graph(g, stream=s):
                H = hdc.encode(self.X, m, ws=ws)
                init = H[self.init_idx].contiguous()
                lab, _, _, _ = hdc.cluster(H, c.dim, init, c.iters, sim_config(c.train_perf),
                                           sim_config(c.infer_perf))
        torch.cuda.current_stream().wait_stream(s)
        g.replay()
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            g.replay()
        b.record()
        b.synchronize()
        return a.elapsed_time(b) / reps, metrics.nmi(self.y, lab.cpu().numpy())
