#!/usr/bin/env python3
"""Per-kernel throughput of the library's passes outside the headline step,
each beside the roofline that bounds it (the numbers under profiles/).

Subcommands (one JSON line each):

  hamming   hdc_hamming_argmin on packed binary hypervectors at the shapes of
            the retraining and clustering passes.  Up to 32 classes (and above
            256) the distances are popcounts, bound by the popcount unit (16
            results per clock per SM); 33..256 classes run as a tensor-core
            product of the rows expanded to +-1.
  training  hdc_train_epoch: one bundling pass and one retraining epoch
            (started from the bundle) over packed samples made of C random
            prototypes with each bit flipped with probability p, timed as
            CUDA-graph replays, against HBM (bundling reads the N x W words
            once; an epoch reads them for the prediction and the updated rows
            twice more).
  levelid   hdc_levelid_encode at the Micro-HD-Classification shapes (Sec.
            5.3: F = 617, D = 1024, L = 128) and around them, bound by 32-bit
            integer logic: per query, feature and 32-dim word at least one
            XOR (binding) and one full adder of the count (two 3-input logic
            operations), 3 LOP3 against 64 LOP3 per clock per SM.
  classify  hdc_classify of one configuration on a batch of a workload's
            queries: step time and the encoding kernel's time and FLOP rate
            against the measured tensor peak (the small cases profiles/ captures).
  cluster   HD-Clustering (encode + hdc_cluster) eagerly and as one CUDA
            graph, with the NMI of each configuration.

Clock-based peaks use the SM clock sampled (through NVML, read-only) while
the measured launches ran, and the device's own SM count.
"""
from __future__ import annotations

import argparse
import dataclasses
import json
import os
import statistics
import sys

import numpy as np
import torch

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from bench import ClockSampler  # noqa: E402
from paper_2606_26547_gb300 import hdc, synth  # noqa: E402

POPC_PER_CLK_SM = 16
LOP3_PER_CLK_SM = 64


def sms() -> int:
    return torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count


def timed_ms(fn, reps: int) -> tuple:
    """Mean device time of fn() over reps launches (CUDA events on the
    current stream) and the median SM clock sampled meanwhile."""
    fn()
    torch.cuda.synchronize()
    clk = ClockSampler(torch.cuda.current_device(), period=0.002)
    clk.start()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    clk.mark("t0")
    a.record()
    for _ in range(reps):
        fn()
    b.record()
    b.synchronize()
    clk.mark("t1")
    c = clk.stop()
    return a.elapsed_time(b) / reps, c


def popcount_roofline(word_compares_per_s: float, n_sms: int, mhz: float) -> dict:
    """Word comparisons per second against the popcount unit's peak."""
    peak = POPC_PER_CLK_SM * n_sms * mhz * 1e6
    return {"bound": "alu (popcount)", "achieved_per_s": word_compares_per_s, "peak_per_s": peak,
            "frac": word_compares_per_s / peak, "sms": n_sms, "sm_mhz": mhz}


def lop3_roofline(lops_per_s: float, n_sms: int, mhz: float) -> dict:
    peak = LOP3_PER_CLK_SM * n_sms * mhz * 1e6
    return {"bound": "alu (LOP3)", "achieved_tlops": lops_per_s / 1e12, "peak_tlops": peak / 1e12,
            "frac": lops_per_s / peak, "sms": n_sms, "sm_mhz": mhz}


def clock_of(c: dict) -> float:
    return c.get("sm_mhz") or c.get("sm_max_mhz") or 2070.0


# ------------------------------------------------------------------ hamming

def random_rows(n: int, D: int, W: int, g: torch.Generator, dev) -> torch.Tensor:
    """n x W packed words with the first D bits uniform and pad bits zero."""
    r = torch.randint(-2 ** 31, 2 ** 31 - 1, (n, W), generator=g, device=dev, dtype=torch.int64).to(torch.int32)
    if D % 32:
        r[:, D // 32] &= (1 << (D % 32)) - 1
    r[:, (D + 31) // 32:] = 0
    return r


def hamming(N: int, D: int, C: int, reps: int = 10, seed: int = 0) -> dict:
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    W = hdc.words(D)
    Q, Cl = random_rows(N, D, W, g, dev), random_rows(C, D, W, g, dev)
    ms, clk = timed_ms(lambda: hdc.hamming_argmin(Q, Cl, D), reps)
    assert hdc.stream_status() == 0
    tc = 32 < C <= 256
    out = {"N": N, "D": D, "C": C, "W": W, "ms": round(ms, 4), "queries_per_s": N / (ms / 1e3),
           "word_compares_per_s": N * C * W / (ms / 1e3),
           "route": "tensor cores (rows expanded to +-1)" if tc else "popcount", "clocks": clk}
    if not tc:
        out["roofline"] = popcount_roofline(out["word_compares_per_s"], sms(), clock_of(clk))
    return out


# ----------------------------------------------------------------- training

def packed_bernoulli(n: int, D: int, W: int, p: float, g: torch.Generator, dev) -> torch.Tensor:
    """n x W packed words whose first D bits are 1 with probability p (pad bits 0)."""
    shifts = torch.arange(32, device=dev, dtype=torch.int32)
    out = torch.empty((n, W), dtype=torch.int32, device=dev)
    for r0 in range(0, n, 8192):
        r1 = min(n, r0 + 8192)
        bits = torch.rand((r1 - r0, W * 32), generator=g, device=dev) < p
        bits[:, D:] = False
        words = (bits.view(r1 - r0, W, 32).to(torch.int32) << shifts).sum(-1, dtype=torch.int64)
        out[r0:r1] = words.to(torch.int32)
    return out


def graph_of(fn):
    """fn() captured in one CUDA graph (after one eager warm-up call)."""
    fn()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    st = torch.cuda.Stream()
    st.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(st):
        with torch.cuda.graph(g, stream=st):
            fn()
    torch.cuda.current_stream().wait_stream(st)
    torch.cuda.synchronize()
    return g


def replay_ms(g, reps: int) -> float:
    """Mean device time of one replay of graph g (back to back, CUDA events)."""
    g.replay()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        g.replay()
    b.record()
    b.synchronize()
    return a.elapsed_time(b) / reps


def training(N: int, D: int, C: int, p: float = 0.48, reps: int = 20, seed: int = 0) -> dict:
    """Device time of one bundling pass and of one retraining epoch started
    from the bundle, each as CUDA-graph replays (a graph of the bundle, a
    graph of bundle + epoch; the epoch is their difference), so the host's
    launch of the pass's kernels is not in the figure; the eager time of one
    hdc_train_epoch call from Python is reported beside it."""
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    W = hdc.words(D)
    protos = packed_bernoulli(C, D, W, 0.5, g, dev)
    y = torch.randint(0, C, (N,), generator=g, device=dev, dtype=torch.int32)
    H = protos[y.long()] ^ packed_bernoulli(N, D, W, p, g, dev)
    acc = torch.empty((C, D), dtype=torch.int32, device=dev)
    cls = torch.empty((C, W), dtype=torch.int32, device=dev)
    nu = torch.zeros(1, dtype=torch.int32, device=dev)
    ws = hdc.train_workspace(N, D, C, dev)
    out = {"N": N, "D": D, "C": C, "W": W, "flip_p": p}
    bundle = lambda: hdc.train_epoch(H, y, D, C, 0, acc, cls, ws=ws)
    epoch = lambda: hdc.train_epoch(H, y, D, C, 1, acc, cls, n_updates=nu, ws=ws)

    def both():
        bundle()
        epoch()
    clk = ClockSampler(torch.cuda.current_device(), period=0.002)
    clk.start()
    clk.mark("t0")
    ga, gb = graph_of(bundle), graph_of(both)
    t_bundle = replay_ms(ga, reps)
    t_both = replay_ms(gb, reps)
    upd = int(nu.item())
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    eager = {}
    for name, fn in (("bundle", bundle), ("retrain_epoch", epoch)):
        ts = []
        for _ in range(9):
            bundle()
            a.record()
            fn()
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        eager[name] = sorted(ts)[len(ts) // 2]
    clk.mark("t1")
    for name, ms, u in (("bundle", t_bundle, 0), ("retrain_epoch", t_both - t_bundle, upd)):
        nbytes = N * W * 4 + 2 * u * W * 4
        out[name] = {"ms": round(ms, 4), "updates": u, "algorithmic_bytes": nbytes,
                     "gbs": round(nbytes / (ms / 1e3) / 1e9, 1), "eager_call_ms": round(eager[name], 4)}
    out["clocks"] = clk.stop()
    assert hdc.stream_status() == 0
    return out


# ------------------------------------------------------------------ levelid

def levelid(F: int, D: int, L: int, N: int, stride: int = 1, reps: int = 10, seed: int = 1) -> dict:
    dev = torch.device("cuda")
    ids, lo, hi, flip = synth.levelid_hvs(F, D, L, seed)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    m = hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), L, -3.0, 3.0, hdc.ApproxConfig(perf_stride=stride))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    X = torch.randn((N, F), generator=g, device=dev)
    H = torch.empty((N, m.W), dtype=torch.int32, device=dev)
    ms, clk = timed_ms(lambda: hdc.levelid_encode(X, m, out=H), reps)
    words = (m.Dk + 31) // 32
    lops = 3.0 * N * F * words
    assert hdc.stream_status() == 0
    return {"F": F, "D": D, "Dk": m.Dk, "L": L, "queries": N, "ms": round(ms, 4),
            "queries_per_s": N / (ms / 1e3), "clocks": clk,
            "roofline": lop3_roofline(lops / (ms / 1e3), sms(), clock_of(clk))}


# ----------------------------------------------------------------- classify

def classify(workload: str, enc: str, stride: int, class_bits: int, float_query: bool, batch: int,
             reps: int = 10) -> dict:
    """hdc_classify on `batch` queries of a workload's mixture with a model
    trained on its training set (FP32 encode, bundling + one epoch): device
    time per call and of the library's encoding kernel (hdc_profile_events),
    with the kernel's FLOP rate against the measured tensor peak."""
    w = synth.WORKLOADS[workload]
    d = synth.make(w, n_train=min(w.n_train, 20000), n_query=1)
    dev = torch.device("cuda")
    Bt = torch.from_numpy(d["Bt"]).to(dev)
    H = hdc.encode(torch.from_numpy(d["Xtr"]).to(dev), hdc.Model(Bt, hdc.ApproxConfig(enc="fp32")))
    acc, _, _ = hdc.train(H, torch.from_numpy(d["ytr"]).to(dev), w.D, w.C, 1)
    del H
    m = hdc.Model(Bt, hdc.ApproxConfig(enc=enc, perf_stride=stride, class_bits=class_bits,
                                       float_query=float_query), acc=acc)
    X, _ = synth.device_gauss_queries(batch, w, seed=99, device=dev)
    labels = torch.empty(batch, dtype=torch.int32, device=dev)
    ws = m.workspace(batch)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in evs:   # torch creates an event's handle on its first record
        a.record()
        b.record()
    it = iter(range(reps))

    def step():
        i = next(it, None)
        if i is not None:
            hdc.profile_events(*evs[i])
        hdc.classify(X, m, ws=ws, labels=labels)
        hdc.profile_events(None, None)
    hdc.classify(X, m, ws=ws, labels=labels)
    torch.cuda.synchronize()
    ms, clk = timed_ms(step, reps)
    kern = statistics.median(a.elapsed_time(b) for a, b in evs)
    assert hdc.stream_status() == 0
    flops = 2.0 * batch * w.F * m.Dk
    pk = {}
    try:
        pk = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    peak = pk.get("bf16_tflops", 1900.0) * (2.0 if enc == "fp8" else 1.0)
    return {"workload": workload, "enc": enc, "stride": stride, "class_bits": class_bits,
            "float_query": float_query, "queries": batch, "Dk": m.Dk, "step_ms": round(ms, 4),
            "queries_per_s": batch / (ms / 1e3), "kernel_ms": round(kern, 4),
            "kernel_tflops": flops / (kern / 1e3) / 1e12, "frac_of_tensor_peak": flops / (kern / 1e3) / 1e12 / peak,
            "clocks": clk}


# ------------------------------------------------------------------ cluster

def cluster(workload: str) -> dict:
    from paper_2606_26547_gb300.cluster import ClusterConfig, ClusterRun
    cr = ClusterRun(workload)
    w = cr.w
    rows = []
    for c in (ClusterConfig("fp32", w.D, w.epochs), ClusterConfig("fp8", w.D, w.epochs),
              ClusterConfig("fp8", w.D, 3), ClusterConfig("fp8", w.D, 3, infer_perf=(0.0, 0.9, 1)),
              ClusterConfig("fp8", w.D, 3, train_perf=(0.0, 0.5, 1), infer_perf=(0.0, 0.9, 1)),
              ClusterConfig("fp8", w.D // 2, 3)):
        r = cr.run(c)
        cr.run(c)
        eager = []
        for _ in range(5):
            t = cr.run(c, timed=True)
            eager.append(t["encode_ms"] + t["cluster_ms"])
        gms, gnmi = cr.graph_ms(c)
        assert gnmi == r["nmi"]
        rows.append({**dataclasses.asdict(c), "nmi": round(r["nmi"], 4), "ms": round(statistics.median(eager), 4),
                     "graph_ms": round(gms, 4), "changes_last": r["changes"][-1:]})
    return {"workload": w.name, "points": int(cr.X.shape[0]), "K": w.C, "configs": rows}


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    sub = ap.add_subparsers(dest="cmd", required=True)
    h = sub.add_parser("hamming")
    h.add_argument("--shapes", default="100000x16384x100,100000x16384x40,100000x16384x256,1000000x1024x26,"
                                       "60000x10000x10")
    t = sub.add_parser("training")
    t.add_argument("--shapes", default="60000x10000x10,100000x16384x100,200000x1024x26")
    t.add_argument("--flip", type=float, default=0.48, help="bit-flip probability of a sample")
    lv = sub.add_parser("levelid")
    lv.add_argument("--queries", type=int, default=262144)
    cf = sub.add_parser("classify")
    cf.add_argument("--workload", default="precision_F784_D10000_C10")
    cf.add_argument("--enc", default="fp8")
    cf.add_argument("--stride", type=int, default=2)
    cf.add_argument("--class-bits", type=int, default=1)
    cf.add_argument("--float-query", action="store_true")
    cf.add_argument("--batch", type=int, default=1 << 20)
    cl = sub.add_parser("cluster")
    cl.add_argument("--workload", default="cluster_F617_D1024_K26")
    a = ap.parse_args(argv)
    from paper_2606_26547_gb300 import build
    build.build()
    hdc.load()
    if a.cmd == "hamming":
        out = {"op": "hamming_argmin", "runs": [hamming(*(int(v) for v in s.split("x"))) for s in a.shapes.split(",")]}
    elif a.cmd == "training":
        out = {"op": "train_epoch", "runs": [training(*(int(v) for v in s.split("x")), p=a.flip)
                                             for s in a.shapes.split(",")]}
    elif a.cmd == "levelid":
        q = a.queries
        out = {"encoder": "level-id", "runs": [levelid(617, 1024, 128, q), levelid(617, 512, 128, q),
                                               levelid(617, 1024, 32, q), levelid(617, 2048, 128, q),
                                               levelid(617, 10000, 128, q // 4), levelid(617, 1024, 814, q)]}
    elif a.cmd == "classify":
        out = classify(a.workload, a.enc, a.stride, a.class_bits, a.float_query, a.batch)
    else:
        out = cluster(a.workload)
    print(json.dumps(out))


if __name__ == "__main__":
    main()
