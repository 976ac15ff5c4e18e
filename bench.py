#!/usr/bin/env python3
"""Throughput of the HDC classification hot path on GB300.

Workload: precision_F784_D10000_C10 (F = 784 FP32 features, 10-class
Gaussian mixture, base hypermatrix 784 x 10,000 N(0,1), 60,000 training
samples, bundling + 20 retraining epochs).  One step classifies one batch of
queries drawn from the same mixture (default 1,048,576 queries = 3.3 GB of
FP32 features, larger than L2) with the approximate configuration: FP8 E4M3
encoding with per-row power-of-two scales on the tensor cores, dimension
perforation of stride 2 (D' = 5,000), binary class hypervectors, Hamming
arg-min -- quantise kernel + fused tcgen05 kernel per step.

Also measured on the same GPU: the plain exact form (FP32 FFMA encode at the
full D, packed Hamming), the accuracy of both on the 10,000-query set, an
end-to-end figure through the same C-ABI call with pinned host buffers (with
the rate of one plain pinned copy of the same rows in the same run, the bound
that figure meets), the bundling and retraining-epoch passes, and the CPU
oracle on a bounded sample.  `--impl reference` times the CPU oracle
alone on the host cores.

Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

WORKLOAD = "precision_F784_D10000_C10"
METRIC = "queries/sec at D=10,000 (approx vs exact, same GB300, <=1pt acc loss)"
UNIT = "queries/s"


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=300)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default=WORKLOAD, help="synth.WORKLOADS key")
    ap.add_argument("--batch", type=int, default=1 << 20, help="queries per step (per GPU)")
    ap.add_argument("--enc", default="fp8", choices=["bf16", "fp8"])
    ap.add_argument("--stride", type=int, default=2)
    ap.add_argument("--class-bits", type=int, default=None, help="1 (default), 4 or 8 (8 with --float-query)")
    ap.add_argument("--float-query", action="store_true",
                    help="cosine on non-binarised (BF16) query hypervectors against b-bit classes")
    ap.add_argument("--exact-steps", type=int, default=5)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=15.0, help="target CPU work of the oracle sample")
    return ap.parse_args()


# ------------------------------------------------------------------ clocks

class ClockSampler:
    """nvidia-smi samples every 200 ms while running (read-only query)."""
    FIELDS = ("timestamp,index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.path = tempfile.mktemp(suffix=".csv")
        self.proc = None
        self.gpu = gpu_index
        self.t0 = self.t1 = None

    def start(self):
        try:
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.FIELDS,
                                          "--format=csv,noheader,nounits", "-lms", "200"], stdout=self.f,
                                         stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def mark(self, which):
        setattr(self, which, time.time())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(5)
        except Exception:
            self.proc.kill()
        self.f.close()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 10:
                continue
            try:
                ts = time.mktime(time.strptime(parts[0].split(".")[0], "%Y/%m/%d %H:%M:%S"))
                rows.append((ts, float(parts[2]), float(parts[3]), parts[6:10]))
            except Exception:
                continue
        os.unlink(self.path)
        inside = [r for r in rows if self.t0 and self.t1 and self.t0 - 1 <= r[0] <= self.t1 + 1] or rows
        if not inside:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({n for r in inside for n, v in zip(names, r[3]) if v.lower() == "active"})
        return {"sm_mhz": statistics.median(r[1] for r in inside), "sm_max_mhz": max(r[2] for r in inside),
                "reasons": reasons, "samples": len(inside)}


# --------------------------------------------------------------- helpers

# DRAM traffic of the fused kernel from one ncu capture (profiles/
# tc_encode_kernel_fp8_F784_D10000_stride2.md): bytes per query, valid only
# while the kernel sources hash to the value they had when it was taken.
PROFILED_TRAFFIC = {"sources_sha1_16": "4306b1b282f7211f", "enc": "fp8", "stride": 2,
                    "dram_bytes_per_query": (239427072 + 3662080) / 262144}


def tc_sources_sha():
    import hashlib
    d = os.path.join(ROOT, "paper_2606_26547_gb300", "csrc")
    h = hashlib.sha1()
    for f in ("tc_kernel.cuh", "k_tc.cu", "k_tc_fp8.cu"):
        h.update(open(os.path.join(d, f), "rb").read())
    return h.hexdigest()[:16]


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def oracle_sample_qps(data, w, acc, enc_code, stride, target_s, threads):
    """Time the CPU oracle (as it stands) on a bounded sample of queries: the
    workload's query rows, then further rows of the same mixture, growing the
    sample until one timed run takes about two thirds of target_s."""
    import numpy as np
    import oracle
    from paper_2606_26547_gb300 import synth
    pool, Bt = data["Xq"], data["Bt"]
    n = threads
    while True:
        if n > pool.shape[0]:
            extra, _ = synth.more_queries(w, n - pool.shape[0])
            pool = np.concatenate([pool, extra])
        t = time.perf_counter()
        labels, _ = oracle.classify(pool[:n], Bt, acc, enc_code, 0.0, 1.0, stride, 1, threads=threads)
        dt = time.perf_counter() - t
        if dt >= target_s * 2 / 3:
            return n / dt, n, dt, labels
        n = max(2 * n, int(n * target_s * 0.8 / max(dt, 1e-3))) // threads * threads


def train_model(hdc, torch, data, dev, epochs):
    Bt = torch.from_numpy(data["Bt"]).to(dev)
    base = hdc.Model(Bt, hdc.ApproxConfig(enc="fp32"))
    Xtr = torch.from_numpy(data["Xtr"]).to(dev)
    ytr = torch.from_numpy(data["ytr"]).to(dev)
    torch.cuda.synchronize()
    t = time.perf_counter()
    H = hdc.encode(Xtr, base)
    acc, cls, ups = hdc.train(H, ytr, Bt.shape[0], int(data["ytr"].max()) + 1, epochs)
    torch.cuda.synchronize()
    return Bt, acc, ups, time.perf_counter() - t, H, ytr


def time_training(hdc, torch, H, y, D, C, reps=5):
    """Device time of one bundling pass and one retraining epoch over the
    packed training hypervectors H, with HBM throughput against algorithmic
    bytes (bundling reads N*W*4; an epoch reads them for the prediction and
    the misclassified rows twice more for the update)."""
    N, W = H.shape
    acc = torch.empty((C, D), dtype=torch.int32, device=H.device)
    cls = torch.empty((C, W), dtype=torch.int32, device=H.device)
    nu = torch.zeros(1, dtype=torch.int32, device=H.device)
    n = __import__("ctypes").c_size_t()
    hdc._call("hdc_train_workspace_bytes", N, D, C, __import__("ctypes").byref(n))
    ws = hdc._empty_bytes(n.value, H.device)
    out = {}
    for name, mode in (("bundle", 0), ("retrain_epoch", 1)):
        hdc.train_epoch(H, y, D, C, 0, acc, cls, ws=ws)      # start from the bundle
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        ts = []
        for _ in range(reps):
            if mode == 1:
                hdc.train_epoch(H, y, D, C, 0, acc, cls, ws=ws)
            a.record()
            hdc.train_epoch(H, y, D, C, mode, acc, cls, n_updates=nu, ws=ws)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b) / 1e3)
        t = sorted(ts)[len(ts) // 2]
        upd = int(nu.item()) if mode == 1 else 0
        nbytes = N * W * 4 + 2 * upd * W * 4
        out[name] = {"ms": t * 1e3, "algorithmic_bytes": nbytes, "gbs": nbytes / t / 1e9,
                     "updates": upd}
    return out


def timed_steps(torch, fn, steps, stream):
    """Device time of `steps` calls of fn(i) between CUDA events."""
    start, stop = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    start.record(stream)
    for i in range(steps):
        fn(i)
    stop.record(stream)
    stop.synchronize()
    return start.elapsed_time(stop) / 1e3


# ---------------------------------------------------------------- our arm

def run_ours(a):
    import numpy as np
    import torch
    import torch.distributed as dist

    from paper_2606_26547_gb300 import build, hdc, synth
    from paper_2606_26547_gb300 import dist as hdist

    rank = int(os.environ.get("RANK", 0))
    world = int(os.environ.get("WORLD_SIZE", 1))
    local = int(os.environ.get("LOCAL_RANK", 0))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    build.build()
    hdc.load()
    w = synth.WORKLOADS[a.workload]
    data = synth.make(w, n_query=min(w.n_query, 20000))
    Bt, acc, ups, train_s, Htr, ytr = train_model(hdc, torch, data, dev, w.epochs)
    train_passes = time_training(hdc, torch, Htr, ytr, w.D, w.C)
    del Htr

    cbits = a.class_bits or (8 if a.float_query else 1)
    approx_cfg = hdc.ApproxConfig(enc=a.enc, perf_stride=a.stride, class_bits=cbits, float_query=a.float_query)
    exact_cfg = hdc.ApproxConfig(enc="fp32")
    m_apx = hdc.Model(Bt, approx_cfg, acc=acc)
    m_ex = hdc.Model(Bt, exact_cfg, acc=acc)

    # accuracy on the 10,000-query set
    Xq = torch.from_numpy(data["Xq"]).to(dev)
    yq = data["yq"]
    lab_ex = hdc.classify(Xq, m_ex).cpu().numpy()
    lab_apx = hdc.classify(Xq, m_apx).cpu().numpy()
    acc_ex = float((lab_ex == yq).mean())
    acc_apx = float((lab_apx == yq).mean())

    # throughput batch (this rank's shard of the job: weak scaling)
    B = a.batch
    X, _ = synth.device_gauss_queries(B, w, seed=777 + rank, device=dev)
    labels = torch.empty(B, dtype=torch.int32, device=dev)
    ws = m_apx.workspace(B)
    stream = torch.cuda.current_stream()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(a.steps)]
    for s, e in evs:  # torch creates the event handles on first record
        s.record(stream)
        e.record(stream)
    torch.cuda.synchronize()

    def step_apx(i):
        hdc.classify(X, m_apx, ws=ws, labels=labels)

    def step_apx_prof(i):
        hdc.profile_events(*evs[i])
        hdc.classify(X, m_apx, ws=ws, labels=labels)

    for i in range(a.warmup):
        step_apx(i)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    time.sleep(0.6)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clk.mark("t0")
    el = timed_steps(torch, step_apx_prof, a.steps, stream)
    clk.mark("t1")
    hdc.profile_events(None, None)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clocks = clk.stop()
    assert hdc.stream_status() == 0
    kern_s = [s.elapsed_time(e) / 1e3 for s, e in evs]
    el = hdist.max_over_ranks(el, device=dev)
    value = hdist.job_throughput(B, a.steps, world, el)

    # exact form on the same GPU
    ws_ex = m_ex.workspace(B)
    hdc.classify(X, m_ex, ws=ws_ex, labels=labels)
    torch.cuda.synchronize()
    el_ex = timed_steps(torch, lambda i: hdc.classify(X, m_ex, ws=ws_ex, labels=labels), a.exact_steps, stream)
    exact_qps = B * a.exact_steps / el_ex
    del ws_ex

    # end to end through the C ABI with HOST buffers (hdc_classify_host: rows
    # copied in, classified, labels copied out); chunks alternate between two
    # streams so one chunk's copy overlaps another's kernels
    Xh = X.cpu().pin_memory()
    Lh = torch.empty(B, dtype=torch.int32).pin_memory()
    Xd = torch.empty_like(X)
    e2e_steps = max(3, min(a.steps, 20))
    nch = 8
    bounds = [B * c // nch for c in range(nch + 1)]
    e2e_streams = [torch.cuda.Stream(device=dev) for _ in range(2)]
    ws_e2e = [m_apx.workspace(bounds[1] - bounds[0] + 1) for _ in e2e_streams]

    def step_e2e(i):
        for s in e2e_streams:
            s.wait_stream(stream)
        for c in range(nch):
            lo, hi = bounds[c], bounds[c + 1]
            hdc.classify_host([Xh[lo:hi]], m_apx, Xd[lo:hi], labels[lo:hi], Lh[lo:hi], ws_e2e[c % 2],
                              stream=e2e_streams[c % 2])
        for s in e2e_streams:
            stream.wait_stream(s)

    step_e2e(0)
    torch.cuda.synchronize()
    el_e2e = timed_steps(torch, step_e2e, e2e_steps, stream)
    e2e_qps = world * B * e2e_steps / el_e2e
    # the host link on this machine: one plain pinned copy of the same rows, so
    # the e2e figure can be read against the copy bound it meets
    el_copy = timed_steps(torch, lambda i: Xd.copy_(Xh, non_blocking=True), 3, stream)
    h2d_gbs = 3 * B * w.F * 4 / el_copy / 1e9

    # roofline of the dominant kernel (fused tcgen05 encode + Hamming + arg-min)
    F, Dk = w.F, m_apx.Dk
    avg_k = sum(kern_s) / len(kern_s)
    flops = 2.0 * B * F * Dk
    pk = peaks()
    ratio = 2.0 if a.enc == "fp8" else 1.0
    if "bf16_tflops_sustained" in pk:
        peak = pk["bf16_tflops_sustained"] * ratio
        peak_src = "measured bf16 sustained x %.0f (nominal fp8/bf16 ratio)" % ratio if ratio != 1 else \
            "measured bf16 sustained"
    else:
        peak = 1700.0 * ratio
        peak_src = "fallback"
    achieved = flops / avg_k / 1e12
    pt = PROFILED_TRAFFIC
    traffic = (pt["dram_bytes_per_query"] * B if tc_sources_sha() == pt["sources_sha1_16"] and a.enc == pt["enc"]
               and a.stride == pt["stride"] and a.workload == WORKLOAD and cbits == 1 and not a.float_query
               else None)
    fused = cbits == 1 and not a.float_query

    out = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": a.steps, "warmup": a.warmup,
        "ms_per_step": el / a.steps * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "%s operands, fp32 accumulate, %s" % ("e4m3" if a.enc == "fp8" else "bf16",
                                                         "bf16 query hypervectors" if a.float_query
                                                         else "binary hypervectors"),
        "data": "synthetic (seeded Gaussian mixture shaped like the workload; no dataset)",
        "config": {"workload": a.workload, "F": F, "D": w.D, "C": w.C, "enc": a.enc,
                   "perforation": [0.0, 1.0, a.stride], "Dk": Dk, "class_bits": cbits,
                   "query": "float (BF16 projections, cosine)" if a.float_query else "binary", "queries_per_step": B,
                   "train": "bundling + %d retraining epochs on %d samples (FP32 encode)" % (w.epochs, w.n_train),
                   "l2": "inputs larger than L2 (%.1f GB of FP32 queries per step)" % (B * F * 4 / 1e9),
                   "parallelism": "dp%d (queries sharded, no collective)" % world},
        "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                     "frac": achieved / peak, "traffic": traffic,
                     "kernel": "tc_encode_kernel (%s)" % ("classify" if fused else "encode"),
                     "peak_source": peak_src + " of measured", "kernel_ms": avg_k * 1e3,
                     "algorithmic_flops_per_launch": flops},
        "e2e": {"value": e2e_qps, "unit": UNIT, "h2d_bytes_per_step": B * F * 4, "d2h_bytes_per_step": B * 4,
                "h2d_copy_gbs": h2d_gbs, "frac_of_copy_bound": e2e_qps / world / (h2d_gbs * 1e9 / (F * 4))},
        "gpu_launches": (2 if fused else 3) * a.steps,   # quantise + fused, or + similarity / cosine
        "clocks": clocks,
        "exact": {"value": exact_qps, "unit": UNIT, "enc": "fp32 (FFMA)", "Dk": w.D,
                  "ms_per_step": el_ex / a.exact_steps * 1e3},
        "speedup_vs_exact": value / exact_qps / world,
        "accuracy": {"exact": acc_ex, "approx": acc_apx, "loss_pts": 100.0 * (acc_ex - acc_apx),
                     "label_agreement": float((lab_ex == lab_apx).mean()), "queries": int(yq.size)},
        "train_s": train_s, "train_updates": ups,
        "train_passes": dict(train_passes, hbm_peak_gbs=pk.get("hbm_gbs")),
    }
    if rank == 0 and world == 1 and not a.no_cpu_baseline and fused:   # the oracle sample times the binary path
        import oracle
        threads = os.cpu_count() or 1
        acc_np = acc.cpu().numpy().astype(np.int64)
        qps, n, dt, olab = oracle_sample_qps(data, w, acc_np, {"bf16": 1, "fp8": 2}[a.enc], a.stride,
                                             a.cpu_seconds, threads)
        m = min(n, lab_apx.shape[0])
        out["cpu_baseline"] = {"value": qps, "unit": UNIT, "cores": threads, "kind": "oracle",
                               "sample": "%d queries of the same mixture (the first %d are the accuracy set), "
                                         "same config, %.1f s" % (n, m, dt),
                               "label_agreement_with_gpu": float((olab[:m] == lab_apx[:m]).mean())}
    if rank == 0:
        print(json.dumps(out), flush=True)
    if world > 1:
        dist.destroy_process_group()


# ---------------------------------------------------------- reference arm

def run_reference(a):
    """The CPU oracle, as it stands, on the host cores (rank 0 only)."""
    rank = int(os.environ.get("RANK", 0))
    if rank != 0:
        return
    import numpy as np
    import oracle
    from paper_2606_26547_gb300 import synth
    oracle.build()
    w = synth.WORKLOADS[a.workload]
    threads = os.cpu_count() or 1
    n_train = 32 * threads
    data = synth.make(w, n_train=n_train, n_query=min(w.n_query, 20000))
    dims = oracle.kept_dims(w.D)
    bits, _, _, _ = oracle.encode_bits(data["Xtr"], data["Bt"], oracle.ENC_FP32, dims, threads=threads)
    acc, _ = oracle.train(bits, data["ytr"], w.C, 2)
    enc = {"bf16": 1, "fp8": 2}[a.enc]
    Xq = data["Xq"]
    # size each step so warm-up + timed steps take about two minutes
    t = time.perf_counter()
    oracle.classify(Xq[:threads], data["Bt"], acc, enc, 0.0, 1.0, a.stride, 1, threads=threads)
    probe = time.perf_counter() - t
    per_step = threads * max(1, int(120.0 / max(1, a.steps + a.warmup) / max(probe, 1e-3)))
    per_step = min(per_step, Xq.shape[0] // 2)
    for i in range(a.warmup):
        oracle.classify(Xq[:per_step], data["Bt"], acc, enc, 0.0, 1.0, a.stride, 1, threads=threads)
    t = time.perf_counter()
    for i in range(a.steps):
        lo = (i * per_step) % (Xq.shape[0] - per_step)
        oracle.classify(Xq[lo:lo + per_step], data["Bt"], acc, enc, 0.0, 1.0, a.stride, 1, threads=threads)
    dt = time.perf_counter() - t
    qps = per_step * a.steps / dt
    out = {"impl": "reference", "metric": METRIC, "value": qps, "unit": UNIT, "n_gpus": a.gpus, "steps": a.steps,
           "warmup": a.warmup, "ms_per_step": dt / a.steps * 1e3, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": "f64 oracle of the %s path" % a.enc, "data": "synthetic",
           "config": {"workload": a.workload, "enc": a.enc, "perforation": [0.0, 1.0, a.stride],
                      "queries_per_step": per_step,
                      "train": "bundling + 2 retraining epochs on %d samples (oracle)" % n_train},
           "cpu_baseline": {"value": qps, "unit": UNIT, "cores": threads, "kind": "oracle",
                            "sample": "%d queries per step x %d steps" % (per_step, a.steps)},
           "e2e": {"value": qps, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out), flush=True)


if __name__ == "__main__":
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)
