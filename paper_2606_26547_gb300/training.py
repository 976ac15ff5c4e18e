"""Bundling and retraining-epoch throughput (hdc_train_epoch) on packed
binary hypervectors.

The samples of each shape are C random prototypes with each bit flipped
with probability p (0.48 by default, close enough to 1/2 that a retraining
epoch has misclassified samples to update).  Reported per shape: the device
time of one bundling pass (mode 0) and of one retraining epoch (mode 1,
started from the bundle), the update count, and HBM throughput against the
algorithmic bytes (bundling reads the N x W words once; an epoch reads them
for the prediction and the updated rows twice more)."""
from __future__ import annotations

import json

import torch

from . import hdc


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


def measure(N: int, D: int, C: int, p: float = 0.48, reps: int = 9, seed: int = 0) -> dict:
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
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    for name, mode in (("bundle", 0), ("retrain_epoch", 1)):
        ts = []
        for _ in range(reps):
            hdc.train_epoch(H, y, D, C, 0, acc, cls, ws=ws)   # an epoch starts from the bundle
            a.record()
            hdc.train_epoch(H, y, D, C, mode, acc, cls, n_updates=nu, ws=ws)
            b.record()
            b.synchronize()
            ts.append(a.elapsed_time(b))
        ms = sorted(ts)[len(ts) // 2]
        upd = int(nu.item()) if mode == 1 else 0
        nbytes = N * W * 4 + 2 * upd * W * 4
        out[name] = {"ms": round(ms, 4), "updates": upd, "algorithmic_bytes": nbytes,
                     "gbs": round(nbytes / (ms / 1e3) / 1e9, 1)}
    assert hdc.stream_status() == 0
    return out


def main(argv=None):
    import argparse
    ap = argparse.ArgumentParser(description="bundling and retraining-epoch throughput")
    ap.add_argument("--shapes", default="60000x10000x10,100000x16384x100,200000x1024x26")
    ap.add_argument("--flip", type=float, default=0.48, help="bit-flip probability of a sample")
    a = ap.parse_args(argv)
    hdc.load()
    runs = [measure(*(int(v) for v in s.split("x")), p=a.flip) for s in a.shapes.split(",")]
    print(json.dumps({"op": "train_epoch", "runs": runs}))


if __name__ == "__main__":
    main()
