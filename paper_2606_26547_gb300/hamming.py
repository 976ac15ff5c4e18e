"""Hamming arg-min throughput (hdc_hamming_argmin) on packed binary
hypervectors at the shapes of the retraining and clustering passes.

Up to 32 classes (and above 256) the distances are popcounts, bound by the
popcount unit (about 16 results per clock per SM); 33..256 classes run as a
tensor-core product of the rows expanded to +-1.  Reported per shape: time,
queries/s, 32-dim word comparisons per second (N * C * W) and, on the
popcount route, their fraction of 16 popcounts per clock per SM x the SMs x
the maximum SM clock (a lower bound when the clock ran lower)."""
from __future__ import annotations

import json

import torch

from . import hdc
from .levelid import sm_clock_mhz

POPC_PER_CLK_SM = 16


def popcount_roofline(word_compares_per_s: float, sms: int, mhz: float) -> dict:
    """Word comparisons per second against the popcount unit's peak."""
    peak = POPC_PER_CLK_SM * sms * mhz * 1e6
    return {"bound": "alu (popcount)", "achieved_per_s": word_compares_per_s, "peak_per_s": peak,
            "frac": word_compares_per_s / peak, "sms": sms, "sm_max_mhz": mhz}


def measure(N: int, D: int, C: int, reps: int = 10, seed: int = 0) -> dict:
    dev = torch.device("cuda")
    g = torch.Generator(device=dev)
    g.manual_seed(seed)
    W = ((D + 31) // 32 + 3) // 4 * 4

    def rows(n):
        r = torch.randint(-2 ** 31, 2 ** 31 - 1, (n, W), generator=g, device=dev, dtype=torch.int64).to(torch.int32)
        if D % 32:
            r[:, D // 32] &= (1 << (D % 32)) - 1
        r[:, (D + 31) // 32:] = 0
        return r

    Q, Cl = rows(N), rows(C)
    labels = torch.empty(N, dtype=torch.int32, device=dev)
    hdc.hamming_argmin(Q, Cl, D)
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record()
    for _ in range(reps):
        labels = hdc.hamming_argmin(Q, Cl, D)
    b.record()
    b.synchronize()
    ms = a.elapsed_time(b) / reps
    assert hdc.stream_status() == 0
    tc = 32 < C <= 256
    out = {"N": N, "D": D, "C": C, "W": W, "ms": round(ms, 4), "queries_per_s": N / (ms / 1e3),
           "word_compares_per_s": N * C * W / (ms / 1e3),
           "route": "tensor cores (rows expanded to +-1)" if tc else "popcount"}
    if not tc:
        sms = torch.cuda.get_device_properties(dev).multi_processor_count
        out["roofline"] = popcount_roofline(out["word_compares_per_s"], sms, sm_clock_mhz())
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="Hamming arg-min throughput")
    ap.add_argument("--shapes", default="100000x16384x100,100000x16384x40,100000x16384x256,1000000x1024x26,"
                                        "60000x10000x10")
    a = ap.parse_args(argv)
    hdc.load()
    runs = [measure(*(int(v) for v in s.split("x"))) for s in a.shapes.split(",")]
    print(json.dumps({"op": "hamming_argmin", "runs": runs}))


if __name__ == "__main__":
    main()
