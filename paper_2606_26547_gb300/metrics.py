"""Quality-of-service metrics of the paper's benchmarks (Sec. 5.1):
classification accuracy and, for HD-Clustering, normalized mutual
information between the true classes and the clusters."""
from __future__ import annotations

import numpy as np


def accuracy(pred, truth) -> float:
    pred, truth = np.asarray(pred), np.asarray(truth)
    return float((pred == truth).mean()) if pred.size else 0.0


def nmi(truth, pred) -> float:
    """I(U; V) / ((H(U) + H(V)) / 2) with natural logarithms (the arithmetic
    normalisation); 1.0 when both labelings have a single cluster."""
    truth, pred = np.asarray(truth).ravel(), np.asarray(pred).ravel()
    n = truth.size
    if n == 0:
        return 1.0
    _, u = np.unique(truth, return_inverse=True)
    _, v = np.unique(pred, return_inverse=True)
    cont = np.zeros((u.max() + 1, v.max() + 1), dtype=np.float64)
    np.add.at(cont, (u, v), 1.0)
    pu, pv, puv = cont.sum(1) / n, cont.sum(0) / n, cont / n
    hu = -np.sum(pu * np.log(pu))
    hv = -np.sum(pv * np.log(pv))
    nz = puv > 0
    mi = np.sum(puv[nz] * (np.log(puv[nz]) - np.log(np.outer(pu, pv)[nz])))
    if hu == 0.0 and hv == 0.0:
        return 1.0
    denom = (hu + hv) / 2.0
    return float(max(mi, 0.0) / denom) if denom > 0 else 0.0
