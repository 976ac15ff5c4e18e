"""Host logic of the continuous-batching server, with a fake executor (no GPU).

The fake executor 'classifies' a row as int(row[0]) and completes a batch
after a given number of polls, so scheduling, slicing, admission by memory
and result reassembly are checked exactly."""
import numpy as np

from paper_2606_26547_gb300 import serve


class FakeExec:
    def __init__(self, capacity, bytes_per_row=100, polls=2):
        self.arena = serve.Arena(capacity)
        self.bpr, self.polls = bytes_per_row, polls
        self.launched = []

    def reserve(self, m, rows):
        return self.arena.alloc(rows * self.bpr)

    def release(self, block):
        self.arena.free(block)

    def launch(self, m, s, parts, rows, block):
        lab = np.concatenate([req.X[lo:hi, 0].astype(np.int32) for req, lo, hi in parts])
        h = {"left": self.polls, "labels": lab, "m": m}
        self.launched.append((m, rows, [(r.rid, lo, hi) for r, lo, hi in parts]))
        return h

    def ready(self, h):
        h["left"] -= 1
        return h["left"] < 0

    def labels(self, h, rows):
        assert len(h["labels"]) == rows
        return h["labels"]


def _req(rid, m, n, t=0.0):
    X = np.zeros((n, 3), np.float32)
    X[:, 0] = np.arange(n) + 1000 * rid
    return serve.Request(rid, m, X, t)


def test_arena_first_fit_and_merge():
    a = serve.Arena(4096)
    b1, b2, b3 = a.alloc(1000), a.alloc(1000), a.alloc(1000)
    assert b1[0] == 0 and b2[0] == 1024 and b3[0] == 2048 and a.alloc(2000) is None
    a.free(b2)
    assert a.alloc(1024)[0] == 1024
    a.free((1024, 1024)); a.free(b1); a.free(b3)
    assert a.free_list == [(0, 4096)] and a.used == 0


def test_all_requests_complete_with_their_rows():
    ex = FakeExec(10 ** 9)
    s = serve.Scheduler(ex, 2, max_batch=500, chunk=300, slots=2, clock=lambda: 1.0)
    reqs = [_req(i, i % 2, n) for i, n in enumerate([1, 700, 50, 299, 301, 1000, 3])]
    for r in reqs:
        s.submit(r)
    for _ in range(1000):
        s.step()
        if s.idle():
            break
    assert s.idle() and len(s.completed) == len(reqs)
    for r in reqs:
        assert np.array_equal(r.labels, r.X[:, 0].astype(np.int32))
    # no batch exceeds max_batch, no piece exceeds chunk, FIFO within a model
    for m, rows, parts in ex.launched:
        assert rows <= 500 and all(hi - lo <= 300 for _, lo, hi in parts)
    for m in (0, 1):
        order = [rid for mm, _, parts in ex.launched if mm == m for rid, _, _ in parts]
        assert order == sorted(order)


def test_admission_waits_for_memory():
    ex = FakeExec(capacity=256 * 4, bytes_per_row=256, polls=3)    # room for 4 rows at a time
    s = serve.Scheduler(ex, 1, max_batch=4, chunk=4, slots=4, clock=lambda: 2.0)
    s.submit(_req(0, 0, 4))
    s.submit(_req(1, 0, 4))
    s.step()
    assert len(ex.launched) == 1 and ex.arena.free_bytes == 0     # second batch not admitted
    while not s.idle():
        s.step()
    assert len(ex.launched) == 2 and ex.arena.free_bytes == 256 * 4


def test_poisson_load_shape():
    t, m, rows = serve.poisson_requests(20000.0, 2.0, 3, 4096, 5)
    assert abs(t.size / 2.0 - 20000) < 5 * np.sqrt(40000) / 2.0
    assert np.all(np.diff(t) > 0) and rows.min() >= 1 and rows.max() <= 4096
    assert set(np.unique(m)) == {0, 1, 2}
    # log-uniform: median near sqrt(4097)
    assert 40 < np.median(rows) < 90


def test_latency_stats():
    rs = []
    for i in range(100):
        r = _req(i, 0, 1, t=0.0)
        r.t_done = (i + 1) / 1000.0
        rs.append(r)
    st = serve.latency_stats(rs)
    assert abs(st["p50_ms"] - 50.5) < 1e-6 and st["requests"] == 100


def test_open_loop_fails_on_device_status():
    """A device-side failure reported by the executor after the run (e.g. a
    bounded wait that ran out) fails the serving run instead of returning
    its latencies."""
    import pytest

    class BadExec(FakeExec):
        def status(self):
            return 5

    pools = [np.zeros((64, 3), np.float32)]
    for ex, raises in ((FakeExec(10 ** 9), False), (BadExec(10 ** 9), True)):
        s = serve.Scheduler(ex, 1, max_batch=64, chunk=64, slots=1)
        t, m, r = np.array([0.0, 0.0]), np.array([0, 0]), np.array([3, 5])
        if raises:
            with pytest.raises(serve.DeviceStatusError):
                serve.run_open_loop(s, pools, t, m, r, 0.0)
        else:
            reqs, _, rows = serve.run_open_loop(s, pools, t, m, r, 0.0)
            assert rows == 8 and len(reqs) == 2
