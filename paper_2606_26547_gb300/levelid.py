"""Level-ID encoder throughput (hdc_levelid_encode) at the shapes of the
paper's Micro-HD-Classification comparison (Sec. 5.3: F = 617 features,
D = 1024, L = 128 levels) and around them.

Roofline: the encoder is bound by 32-bit integer logic.  Per query, feature
and 32-dim word the algorithm needs at least one XOR (binding) and one full
adder of the per-dim count (two 3-input logic operations): 3 LOP3.  The peak
is the integer pipe's 64 LOP3 per clock per SM x 152 SMs x the maximum SM
clock (2.07 GHz), so the fraction reported is a lower bound when the clock
runs below its maximum."""
from __future__ import annotations

import json
import subprocess

import numpy as np
import torch

from . import hdc, synth

LOP3_PER_CLK_SM = 64
SMS = 152


def sm_clock_mhz() -> float:
    """The maximum SM clock (nvidia-smi), 2070 MHz if it cannot be read."""
    try:
        out = subprocess.run(["nvidia-smi", "--query-gpu=clocks.max.sm", "--format=csv,noheader,nounits", "-i", "0"],
                             capture_output=True, text=True, timeout=10).stdout.strip().splitlines()
        return float(out[0])
    except (OSError, ValueError, IndexError, subprocess.SubprocessError):
        return 2070.0


def measure(F: int, D: int, L: int, N: int, stride: int = 1, reps: int = 10, seed: int = 1) -> dict:
    dev = torch.device("cuda")
    ids, lo, hi, flip = synth.levelid_hvs(F, D, L, seed)
    T = lambda a: torch.from_numpy(np.ascontiguousarray(a)).to(dev)
    m = hdc.LevelIdModel(T(ids), T(lo), T(hi), T(flip), L, -3.0, 3.0, hdc.ApproxConfig(perf_stride=stride))
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    X = torch.randn((N, F), generator=g, device=dev)
    H = torch.empty((N, m.W), dtype=torch.int32, device=dev)
    hdc.levelid_encode(X, m, out=H)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        hdc.levelid_encode(X, m, out=H)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    mhz = sm_clock_mhz()
    words = (m.Dk + 31) // 32
    lops = 3.0 * N * F * words
    peak = LOP3_PER_CLK_SM * SMS * mhz * 1e6
    assert hdc.stream_status() == 0
    return {"F": F, "D": D, "Dk": m.Dk, "L": L, "queries": N, "ms": round(ms, 4),
            "queries_per_s": N / (ms / 1e3), "roofline": {"bound": "alu", "achieved_tlops": lops / (ms / 1e3) / 1e12,
                                                           "peak_tlops": peak / 1e12,
                                                           "frac": lops / (ms / 1e3) / peak,
                                                           "sm_max_mhz": mhz}}


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Level-ID encoder throughput")
    ap.add_argument("--queries", type=int, default=262144)
    a = ap.parse_args(argv)
    hdc.load()
    rows = [measure(617, 1024, 128, a.queries), measure(617, 512, 128, a.queries),
            measure(617, 1024, 32, a.queries), measure(617, 2048, 128, a.queries),
            measure(617, 10000, 128, a.queries // 4), measure(617, 1024, 814, a.queries)]
    print(json.dumps({"encoder": "level-id", "runs": rows}))


if __name__ == "__main__":
    main()
