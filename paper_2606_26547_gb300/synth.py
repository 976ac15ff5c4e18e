"""Seeded synthetic inputs shaped like the HDC classification workloads.

This module holds none of the HDC method's arithmetic: it only draws features,
labels and base hypermatrices from fixed distributions, so that the CUDA path
and the CPU oracle are fed identical inputs.  Every draw is from
``numpy.random.Generator(PCG64(seed))``; the large device-side variant uses a
seeded ``torch.Generator`` and is meant for throughput runs only.

Workloads (sizes follow the HD-Classification application of the paper,
Section 5.1 / Table 1, whose datasets are not available here; the synthetic
class-clustered mixtures stand in for them):

* ``int_exact_F617_D2048_C26``  -- integer features in [-8, 7] around 26
  integer centroids, +-1 base hypermatrix (the shapes of Listing 1).
* ``precision_F784_D10000_C10`` -- FP32 features from a 10-class Gaussian
  mixture (centroids N(0,1), within-class sigma 0.6), N(0,1) base.
* ``sweep_F561_D10000_C6``       -- 6-class Gaussian mixture for the batched
  approximation sweep.
* ``large_F1024_D16384_C100``    -- 100-class mixture, 1e6 queries.
* ``classify_F617_D2048_C26``    -- the approximation-tuning case of
  HD-Classification (Sec. 5.2: D = 2048, 10 training iterations, a float
  baseline near 0.87 accuracy): 26-class mixture with 6238 training and
  1559 validation rows, sigma set so the unapproximated form lands near
  that accuracy.
* ``cluster_F617_D1024_K26``     -- the HD-Clustering case (Sec. 5.2: D =
  1024, 20 training iterations, NMI near 0.72): 7797 points of a 26-class
  mixture clustered into K = 26, sigma set so the binary 20-iteration form
  lands near that NMI.
"""
from __future__ import annotations

import dataclasses

import numpy as np


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    F: int
    D: int
    C: int
    n_train: int
    n_query: int
    kind: str            # "int" (integer mixture, +-1 base) or "gauss"
    sigma: float         # within-class standard deviation
    epochs: int          # retraining epochs after the bundling pass
    seed: int            # base seed; the streams below are derived from it


WORKLOADS = {
    "int_exact_F617_D2048_C26": Workload(
        "int_exact_F617_D2048_C26", 617, 2048, 26, 5000, 2000, "int", 2.0, 3, 1000),
    "precision_F784_D10000_C10": Workload(
        "precision_F784_D10000_C10", 784, 10000, 10, 60000, 10000, "gauss", 0.6, 20, 2000),
    # sigma calibrated so the exact form (FP32 encode at the full D, 10
    # retraining epochs, binary classes) reaches about 0.87 accuracy, the
    # paper's HD-Classification baseline (Sec. 5.2), so the accuracy axis
    # of the sweep is informative
    "sweep_F561_D10000_C6": Workload(
        "sweep_F561_D10000_C6", 561, 10000, 6, 10000, 10000, "gauss", 8.3, 10, 3000),
    "large_F1024_D16384_C100": Workload(
        "large_F1024_D16384_C100", 1024, 16384, 100, 100000, 1000000, "gauss", 0.6, 3, 5000),
    "classify_F617_D2048_C26": Workload(
        "classify_F617_D2048_C26", 617, 2048, 26, 6238, 1559, "gauss", 5.2, 10, 6100),
    # clustering: every point is a "query"; epochs = K-means iterations
    "cluster_F617_D1024_K26": Workload(
        "cluster_F617_D1024_K26", 617, 1024, 26, 0, 7797, "gauss", 4.05, 20, 8000),
}

# stream offsets added to a workload's base seed
_S_CENTROIDS, _S_TRAIN, _S_QUERY, _S_BASE = 0, 1, 2, 3


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def balanced_labels(n: int, C: int) -> np.ndarray:
    """y_n = n mod C (every class equally represented)."""
    return (np.arange(n, dtype=np.int64) % C).astype(np.int32)


def int_centroids(F: int, C: int, seed: int) -> np.ndarray:
    """Centroid components iid uniform integers in [-8, 7]."""
    return _rng(seed).integers(-8, 8, size=(C, F)).astype(np.float64)


def gauss_centroids(F: int, C: int, seed: int) -> np.ndarray:
    return _rng(seed).standard_normal((C, F))


def int_mixture(n: int, F: int, C: int, sigma: float, seed: int, centroid_seed: int):
    """Integer features: clip(round_half_even(mu_y + sigma*eps), -8, 7) as FP32."""
    mu = int_centroids(F, C, centroid_seed)
    y = balanced_labels(n, C)
    eps = _rng(seed).standard_normal((n, F))
    x = np.clip(np.rint(mu[y] + sigma * eps), -8, 7).astype(np.float32)
    return x, y


def gauss_mixture(n: int, F: int, C: int, sigma: float, seed: int, centroid_seed: int):
    """FP32 features x = mu_y + sigma*eps, centroids mu_c ~ N(0, I)."""
    mu = gauss_centroids(F, C, centroid_seed)
    y = balanced_labels(n, C)
    eps = _rng(seed).standard_normal((n, F))
    x = (mu[y] + sigma * eps).astype(np.float32)
    return x, y


def base_bipolar(D: int, F: int, seed: int) -> np.ndarray:
    """Transposed base hypermatrix B^T (D x F) of +-1, Bernoulli(0.5), FP32."""
    bits = _rng(seed).integers(0, 2, size=(D, F))
    return (1 - 2 * bits).astype(np.float32)


def base_gauss(D: int, F: int, seed: int) -> np.ndarray:
    """Transposed base hypermatrix B^T (D x F) with N(0,1) FP32 entries."""
    return _rng(seed).standard_normal((D, F)).astype(np.float32)


def make(workload: str | Workload, n_train: int | None = None, n_query: int | None = None,
         D: int | None = None):
    """Return dict(Bt, Xtr, ytr, Xq, yq) for a workload (sizes overridable)."""
    w = WORKLOADS[workload] if isinstance(workload, str) else workload
    ntr = w.n_train if n_train is None else n_train
    nq = w.n_query if n_query is None else n_query
    Dd = w.D if D is None else D
    cs = w.seed + _S_CENTROIDS
    if w.kind == "int":
        Xtr, ytr = int_mixture(ntr, w.F, w.C, w.sigma, w.seed + _S_TRAIN, cs)
        Xq, yq = int_mixture(nq, w.F, w.C, w.sigma, w.seed + _S_QUERY, cs)
        Bt = base_bipolar(Dd, w.F, w.seed + _S_BASE)
    else:
        Xtr, ytr = gauss_mixture(ntr, w.F, w.C, w.sigma, w.seed + _S_TRAIN, cs)
        Xq, yq = gauss_mixture(nq, w.F, w.C, w.sigma, w.seed + _S_QUERY, cs)
        Bt = base_gauss(Dd, w.F, w.seed + _S_BASE)
    return dict(Bt=Bt, Xtr=Xtr, ytr=ytr, Xq=Xq, yq=yq)


def more_queries(w: Workload, n: int, stream: int = 97):
    """n further query rows of a workload's mixture (same centroids), drawn
    with the seed stream base seed + `stream`; returns (X, y)."""
    cs = w.seed + _S_CENTROIDS
    if w.kind == "int":
        return int_mixture(n, w.F, w.C, w.sigma, w.seed + stream, cs)
    return gauss_mixture(n, w.F, w.C, w.sigma, w.seed + stream, cs)


def levelid_hvs(F: int, D: int, L: int, seed: int):
    """Random draws of a Level-ID encoder: ID hypervector bits (F x D), the
    two level end points (D bits each), Bernoulli(0.5), and the level at
    which each dim switches between them, uniform in 1..L-1."""
    r = _rng(seed + 11)
    ids = r.integers(0, 2, size=(F, D)).astype(np.uint8)
    lo = r.integers(0, 2, size=D).astype(np.uint8)
    hi = r.integers(0, 2, size=D).astype(np.uint8)
    flip = r.integers(1, L, size=D).astype(np.int32)
    return ids, lo, hi, flip


def cluster_init(n: int, K: int, seed: int) -> np.ndarray:
    """K distinct point indices (the initial cluster hypervectors), drawn
    with the workload's init stream (base seed + 7)."""
    return np.sort(_rng(seed + 7).choice(n, K, replace=False)).astype(np.int64)


def device_gauss_queries(n: int, w: Workload, seed: int, device="cuda"):
    """Large query batches drawn on the device (throughput runs only).

    Same mixture as ``gauss_mixture`` / ``int_mixture`` (same centroids) but
    the noise comes from a seeded torch generator on ``device``; integer
    workloads are rounded half to even and clipped to [-8, 7] like
    ``int_mixture``.  Returns (X float32, y int32).
    """
    import torch

    cents = int_centroids if w.kind == "int" else gauss_centroids
    mu = torch.from_numpy(cents(w.F, w.C, w.seed + _S_CENTROIDS)).to(device=device, dtype=torch.float32)
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    y = (torch.arange(n, device=device, dtype=torch.int64) % w.C)
    X = torch.randn(n, w.F, generator=g, device=device, dtype=torch.float32)
    X.mul_(w.sigma).add_(mu[y])
    if w.kind == "int":
        X.round_().clamp_(-8, 7)       # torch.round: half to even
    return X, y.to(torch.int32)
