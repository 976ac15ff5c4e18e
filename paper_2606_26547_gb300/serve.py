"""Continuous-batching classification server over resident HDC models.

Requests (a block of query rows for one model) arrive at any time.  The
scheduler keeps a pending queue per model; whenever a model has a free
in-flight slot and the device-memory arena can hold the batch's buffers, it
forms a batch from the oldest pending requests (slicing a request larger
than ``chunk`` rows into pieces), copies the rows to the device, runs the
classify kernels on that slot's stream, copies the labels back and records
an event.  Completed batches are polled without blocking, their memory is
returned to the arena and finished requests are handed back with their
latency.  Batches of different models and of the same model (several slots)
overlap on the GPU; base and class hypervectors stay resident.

Each query row is classified independently by the kernels, so a request's
labels are identical whether it runs alone or inside any batch.

The executor is pluggable: ``GpuExecutor`` drives libhdc; tests drive the
host logic with a fake executor on the CPU.
"""
from __future__ import annotations

import collections
import dataclasses
import time

import numpy as np

ALIGN = 256


class Arena:
    """First-fit allocator of byte ranges of a fixed device budget."""

    def __init__(self, capacity: int):
        self.capacity = int(capacity)
        self.free_list = [(0, self.capacity)]   # sorted (offset, size)
        self.used = 0

    def alloc(self, n: int):
        n = (int(n) + ALIGN - 1) // ALIGN * ALIGN
        for i, (off, size) in enumerate(self.free_list):
            if size >= n:
                if size == n:
                    self.free_list.pop(i)
                else:
                    self.free_list[i] = (off + n, size - n)
                self.used += n
                return off, n
        return None

    def free(self, block) -> None:
        off, n = block
        self.used -= n
        fl = self.free_list
        i = 0
        while i < len(fl) and fl[i][0] < off:
            i += 1
        fl.insert(i, (off, n))
        # merge with neighbours
        if i + 1 < len(fl) and fl[i][0] + fl[i][1] == fl[i + 1][0]:
            fl[i] = (fl[i][0], fl[i][1] + fl[i + 1][1])
            fl.pop(i + 1)
        if i > 0 and fl[i - 1][0] + fl[i - 1][1] == fl[i][0]:
            fl[i - 1] = (fl[i - 1][0], fl[i - 1][1] + fl[i][1])
            fl.pop(i)

    @property
    def free_bytes(self) -> int:
        return self.capacity - self.used


@dataclasses.dataclass
class Request:
    rid: int
    model: int
    X: object                     # n x F float32 host rows (numpy, or pinned torch)
    t_arrive: float
    labels: np.ndarray | None = None
    done_rows: int = 0
    t_done: float | None = None

    @property
    def n(self) -> int:
        return self.X.shape[0]


@dataclasses.dataclass
class Batch:
    model: int
    parts: list                   # (request, lo, hi)
    rows: int
    block: tuple                  # arena block
    slot: int
    handle: object = None


class Scheduler:
    def __init__(self, executor, n_models: int, max_batch: int = 8192, chunk: int = 4096, slots: int = 4,
                 clock=time.perf_counter):
        self.ex = executor
        self.pending = [collections.deque() for _ in range(n_models)]   # (request, next row)
        self.inflight = [[None] * slots for _ in range(n_models)]
        self.max_batch, self.chunk = max_batch, chunk
        self.clock = clock
        self.completed = []
        self.n_batches = 0
        self.rows_launched = 0

    def submit(self, req: Request) -> None:
        req.labels = np.empty(req.n, dtype=np.int32)
        self.pending[req.model].append([req, 0])

    def _form(self, m: int):
        """Rows of the oldest pending requests, at most max_batch, each piece
        at most `chunk` rows."""
        parts, rows = [], 0
        q = self.pending[m]
        for item in q:
            req, nxt = item
            while nxt < req.n and rows < self.max_batch:
                take = min(req.n - nxt, self.chunk, self.max_batch - rows)
                parts.append((req, nxt, nxt + take))
                rows += take
                nxt += take
            if rows >= self.max_batch:
                break
        return parts, rows

    def _commit(self, m: int, parts) -> None:
        q = self.pending[m]
        for req, lo, hi in parts:
            q[0][1] = hi
            if hi == req.n:
                q.popleft()

    def step(self) -> list:
        """Launch what fits, collect what finished; returns finished requests."""
        for m in range(len(self.pending)):
            for s, b in enumerate(self.inflight[m]):
                if b is not None or not self.pending[m]:
                    continue
                parts, rows = self._form(m)
                if rows == 0:
                    break
                block = self.ex.reserve(m, rows)
                if block is None:               # not enough free device memory: admit later
                    break
                self._commit(m, parts)
                batch = Batch(m, parts, rows, block, s)
                batch.handle = self.ex.launch(m, s, parts, rows, block)
                self.inflight[m][s] = batch
                self.n_batches += 1
                self.rows_launched += rows
        done = []
        for m in range(len(self.inflight)):
            for s, b in enumerate(self.inflight[m]):
                if b is None or not self.ex.ready(b.handle):
                    continue
                labels = self.ex.labels(b.handle, b.rows)
                t = self.clock()
                off = 0
                for req, lo, hi in b.parts:
                    req.labels[lo:hi] = labels[off:off + hi - lo]
                    off += hi - lo
                    req.done_rows += hi - lo
                    if req.done_rows == req.n:
                        req.t_done = t
                        done.append(req)
                self.ex.release(b.block)
                self.inflight[m][s] = None
        self.completed.extend(done)
        return done

    def idle(self) -> bool:
        return not any(self.pending) and all(b is None for row in self.inflight for b in row)


class GpuExecutor:
    """Runs batches with libhdc: one stream and one pinned label buffer per
    (model, slot); device buffers (rows, labels, workspace) carved from one
    arena tensor.  Request rows in pinned host memory (torch tensors) are
    copied to the device slice by slice; numpy rows go through a pinned
    staging buffer first."""

    def __init__(self, models, pool_bytes: int, max_batch: int, slots: int):
        import torch

        from . import hdc
        self.torch, self.hdc = torch, hdc
        self.models = models
        dev = models[0].device
        self.arena = Arena(pool_bytes)
        self.buf = torch.empty(pool_bytes, dtype=torch.uint8, device=dev)
        self.streams = [[torch.cuda.Stream(device=dev) for _ in range(slots)] for _ in models]
        self.stage_x = [[None] * slots for _ in models]
        self.stage_l = [[torch.empty(max_batch, dtype=torch.int32).pin_memory() for _ in range(slots)]
                        for _ in models]
        self.max_batch = max_batch

    def _layout(self, m: int, rows: int):
        F = self.models[m].m.F
        xb = (rows * F * 4 + ALIGN - 1) // ALIGN * ALIGN
        lb = (rows * 4 + ALIGN - 1) // ALIGN * ALIGN
        wb = self.models[m].workspace_bytes(rows)
        return xb, lb, wb

    def reserve(self, m: int, rows: int):
        xb, lb, wb = self._layout(m, rows)
        return self.arena.alloc(xb + lb + wb)

    def release(self, block) -> None:
        self.arena.free(block)

    def launch(self, m: int, s: int, parts, rows: int, block):
        torch, hdc = self.torch, self.hdc
        model = self.models[m]
        F = model.m.F
        xb, lb, wb = self._layout(m, rows)
        off = block[0]
        X = self.buf[off:off + rows * F * 4].view(torch.float32).view(rows, F)
        L = self.buf[off + xb:off + xb + rows * 4].view(torch.int32)
        ws = self.buf[off + xb + lb:off + xb + lb + wb]
        st = self.streams[m][s]
        blocks, r = [], 0
        for req, lo, hi in parts:
            if isinstance(req.X, torch.Tensor):          # pinned host rows: copied directly
                blocks.append(req.X[lo:hi])
            else:                                        # other host rows: pinned staging first
                if self.stage_x[m][s] is None:
                    self.stage_x[m][s] = torch.empty((self.max_batch, F), dtype=torch.float32).pin_memory()
                stage = self.stage_x[m][s][r:r + hi - lo]
                stage.numpy()[:] = req.X[lo:hi]
                blocks.append(stage)
            r += hi - lo
        # one library call: row copies in, classify, labels out (all on st)
        hdc.classify_host(blocks, model, X, L, self.stage_l[m][s], ws, stream=st)
        ev = torch.cuda.Event()
        ev.record(st)
        return (ev, m, s)

    def ready(self, handle) -> bool:
        return handle[0].query()

    def labels(self, handle, rows: int) -> np.ndarray:
        _, m, s = handle
        return self.stage_l[m][s][:rows].numpy().copy()

    def status(self) -> int:
        """Synchronise every slot stream and return the library's device
        status (0, or the first error code: a bounded device wait that ran
        out makes the labels of that run untrustworthy)."""
        for row in self.streams:
            for st in row:
                rc = self.hdc.stream_status(st)
                if rc != 0:
                    return rc
        return 0


# ------------------------------------------------------------------ load

def poisson_requests(rate: float, duration: float, n_models: int, max_rows: int, seed: int):
    """Open-loop arrivals: exponential gaps at `rate`/s; sizes
    floor(exp(U * ln(max_rows + 1))) clipped to [1, max_rows] (log-uniform);
    model chosen uniformly.  Returns (t_arrive, model, rows) arrays."""
    rng = np.random.default_rng(seed)
    n = int(rate * duration * 1.2) + 16
    t = np.cumsum(rng.exponential(1.0 / rate, n))
    t = t[t < duration]
    k = t.size
    rows = np.clip(np.floor(np.exp(rng.uniform(0, np.log(max_rows + 1), k))), 1, max_rows).astype(np.int64)
    model = rng.integers(0, n_models, k)
    return t, model, rows


class DeviceStatusError(RuntimeError):
    """The executor reported a device-side failure during a serving run."""


def run_open_loop(sched: Scheduler, pools, t_arr, model, rows, warmup: float, clock=time.perf_counter):
    """Feed requests at their arrival times; returns (finished requests in
    the measured window, window seconds, rows classified in it).  Once the
    scheduler is idle the executor's device status is read (if it has one):
    a failure raises DeviceStatusError instead of returning the run."""
    import gc
    gc.collect()
    gc.disable()          # a collection over ~10^5 live requests would stall the loop
    try:
        t0 = clock()
        i, n = 0, t_arr.size
        rid = 0
        while i < n or not sched.idle():
            now = clock() - t0
            while i < n and t_arr[i] <= now:
                m = int(model[i])
                pool = pools[m]
                start = (rid * 7919) % max(1, pool.shape[0] - int(rows[i]))
                sched.submit(Request(rid, m, pool[start:start + int(rows[i])], t0 + t_arr[i]))
                rid += 1
                i += 1
            sched.step()
        end = clock() - t0
    finally:
        gc.enable()
    status = getattr(sched.ex, "status", None)
    rc = status() if status is not None else 0
    if rc != 0:
        raise DeviceStatusError("device status %d after the serving run: its results are not valid" % rc)
    meas = [r for r in sched.completed if r.t_arrive - t0 >= warmup]
    window = max(1e-9, end - warmup)
    return meas, window, sum(r.n for r in meas)


def latency_stats(reqs) -> dict:
    lat = np.array([(r.t_done - r.t_arrive) * 1e3 for r in reqs])
    if lat.size == 0:
        return {"p50_ms": None, "p99_ms": None, "mean_ms": None, "requests": 0}
    return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
            "mean_ms": float(lat.mean()), "max_ms": float(lat.max()), "requests": int(lat.size)}


# ------------------------------------------------------------- benchmark

SERVING_MODELS = ((617, 26, 10000), (784, 10, 8192), (561, 6, 4096))   # (F, C, D), binary classes


def build_models(device, enc: str = "bf16", n_train: int = 5000, epochs: int = 3, seed: int = 9000):
    """The three resident models: Gaussian-mixture training sets of each
    shape, bundling + retraining, then hdc_model_prepare for `enc`."""
    import torch

    from . import hdc, synth
    out = []
    for i, (F, C, D) in enumerate(SERVING_MODELS):
        w = synth.Workload("serve%d" % i, F, D, C, n_train, 0, "gauss", 0.6, epochs, seed + 100 * i)
        d = synth.make(w, n_query=1)
        Bt = torch.from_numpy(d["Bt"]).to(device)
        H = hdc.encode(torch.from_numpy(d["Xtr"]).to(device), hdc.Model(Bt, hdc.ApproxConfig(enc="fp32")))
        acc, _, _ = hdc.train(H, torch.from_numpy(d["ytr"]).to(device), D, C, epochs)
        out.append((w, Bt, acc))
    return out


def query_pools(trained, rows: int, seed: int = 77):
    """Pinned host FP32 query rows per model, drawn from its mixture."""
    import torch

    from . import synth
    pools = []
    for i, (w, _, _) in enumerate(trained):
        X, _ = synth.gauss_mixture(rows, w.F, w.C, w.sigma, seed + i, w.seed)
        pools.append(torch.from_numpy(X).pin_memory())
    return pools


def exact_unbatched_qps(trained, pools, t_arr, model, rows, n_req: int = 300) -> float:
    """Closed loop, one request at a time, FP32 FFMA encode (the plain exact
    form): queries per second."""
    import torch

    from . import hdc
    models = [hdc.Model(Bt, hdc.ApproxConfig(enc="fp32"), acc=acc) for (w, Bt, acc) in trained]
    dev = models[0].device
    n = min(n_req, t_arr.size)
    total = 0
    torch.cuda.synchronize()
    t = time.perf_counter()
    for i in range(n):
        m = int(model[i])
        X = pools[m][:int(rows[i])].to(dev, non_blocking=True)
        hdc.classify(X, models[m]).cpu()
        total += int(rows[i])
    return total / (time.perf_counter() - t)


def main(argv=None):
    import argparse
    import json

    import torch

    from . import hdc
    ap = argparse.ArgumentParser(description="continuous-batching serving benchmark")
    ap.add_argument("--rate", type=float, default=20000.0, help="requests per second (Poisson)")
    ap.add_argument("--seconds", type=float, default=5.0, help="measured window")
    ap.add_argument("--warmup", type=float, default=1.0)
    ap.add_argument("--max-rows", type=int, default=4096)
    ap.add_argument("--max-batch", type=int, default=16384)
    ap.add_argument("--slots", type=int, default=3)
    ap.add_argument("--pool-gb", type=float, default=4.0)
    ap.add_argument("--enc", default="bf16")
    a = ap.parse_args(argv)
    dev = torch.device("cuda")
    hdc.load()
    trained = build_models(dev)
    models = [hdc.Model(Bt, hdc.ApproxConfig(enc=a.enc), acc=acc) for (w, Bt, acc) in trained]
    pools = query_pools(trained, 1 << 16)
    ex = GpuExecutor(models, int(a.pool_gb * (1 << 30)), a.max_batch, a.slots)
    sched = Scheduler(ex, len(models), a.max_batch, chunk=4096, slots=a.slots)
    t_arr, model, rows = poisson_requests(a.rate, a.warmup + a.seconds, len(models), a.max_rows, 1234)
    # warm every model's kernels once
    for m in range(len(models)):
        hdc.classify(pools[m][:256].to(dev), models[m])
    torch.cuda.synchronize()
    reqs, window, qrows = run_open_loop(sched, pools, t_arr, model, rows, a.warmup)
    st = latency_stats(reqs)
    offered = float(rows[t_arr >= a.warmup].sum()) / a.seconds
    exact = exact_unbatched_qps(trained, pools, t_arr, model, rows)
    out = {"metric": "serving latency and throughput (continuous batching, 3 resident models)",
           "rate_req_s": a.rate, "enc": a.enc, "models": [list(x) for x in SERVING_MODELS],
           "offered_queries_s": offered, "achieved_queries_s": qrows / window, **st,
           "batches": sched.n_batches, "mean_batch_rows": sched.rows_launched / max(1, sched.n_batches),
           "unbatched_exact_queries_s": exact,
           "exact_stable": bool(exact >= offered),
           "window_s": window}
    print(json.dumps(out))


if __name__ == "__main__":
    main()
