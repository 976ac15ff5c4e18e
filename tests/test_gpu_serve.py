"""Continuous batching on the GPU: every request's labels inside mixed,
sliced, overlapping batches equal its labels classified alone."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2606_26547_gb300 import build, hdc, serve
    build.build()
    hdc.load()
    dev = torch.device("cuda")
    trained = serve.build_models(dev, n_train=600, epochs=1)
    pools = serve.query_pools(trained, 6000)
    return hdc, serve, dev, trained, pools


@pytest.mark.parametrize("enc", ["bf16", "fp8"])
def test_requests_in_the_mix_equal_alone(setup, enc):
    hdc, serve, dev, trained, pools = setup
    models = [hdc.Model(Bt, hdc.ApproxConfig(enc=enc), acc=acc) for (w, Bt, acc) in trained]
    ex = serve.GpuExecutor(models, 1 << 28, 4096, 3)
    sched = serve.Scheduler(ex, 3, max_batch=4096, chunk=1000, slots=3)
    rng = np.random.default_rng(3)
    reqs = []
    for i in range(90):
        m = int(rng.integers(0, 3))
        n = int(rng.integers(1, 3000))
        lo = int(rng.integers(0, 6000 - n))
        X = pools[m][lo:lo + n] if i % 3 else pools[m][lo:lo + n].numpy()   # pinned torch or numpy rows
        reqs.append(serve.Request(i, m, X, 0.0))
    it = iter(reqs)
    pending = True
    while pending or not sched.idle():
        for _ in range(int(rng.integers(0, 5))):    # arrivals while batches are in flight
            r = next(it, None)
            if r is None:
                pending = False
                break
            sched.submit(r)
        sched.step()
    assert len(sched.completed) == len(reqs)
    for r in reqs:
        Xd = (r.X if isinstance(r.X, torch.Tensor) else torch.from_numpy(r.X)).to(dev)
        alone = hdc.classify(Xd, models[r.model]).cpu().numpy()
        assert np.array_equal(r.labels, alone), r.rid
    assert ex.arena.used == 0
    torch.cuda.synchronize()
    assert hdc.stream_status() == 0
