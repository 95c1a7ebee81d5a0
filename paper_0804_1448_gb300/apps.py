"""The applications of Sec. 2.2 on top of the search: the k-nearest-neighbour
entropy estimate (Eq. entropie_knn, with Eq. digamma and Eq. boule) and
majority-vote classification.

The neighbour searches run on the GPU through the C ABI (knn_search_self for
the entropy, knn_search for classification).  What is left is a reduction of
n numbers and the constants of the estimate, done on the host in float64, and
a vote over k labels per query.

Reading of Eq. entropie_knn.  As printed, the summand is
log((n-1) rho_k(y_i)) + log c_1(d) - Psi(k).  The estimator it names (Goria et
al., after Kozachenko and Leonenko) raises the k-th neighbour distance to the
power d -- log((n-1) rho_k^d) -- which is what makes it consistent (for points
uniform in the unit cube it tends to the true entropy 0, and for a Gaussian
to (d/2) log(2 pi e sigma^2)).  `entropy` uses that form by default; the
printed one is available as form="printed".  Equal points (rho_k = 0) make
either form -inf.
"""
from __future__ import annotations

import math

import numpy as np

EULER_GAMMA = 0.57721566490153286060651209008240243


def digamma_int(k: int) -> float:
    """Psi(k) of Eq. digamma for a positive integer k: -gamma + sum_{j<k} 1/j."""
    if k < 1:
        raise ValueError("k >= 1")
    return -EULER_GAMMA + math.fsum(1.0 / j for j in range(1, k))


def log_unit_ball(d: int) -> float:
    """log c_1(d) of Eq. boule: c_1(d) = 2 pi^(d/2) / (d Gamma(d/2)), the volume of
    the unit ball of R^d."""
    return math.log(2.0) + 0.5 * d * math.log(math.pi) - math.log(d) - math.lgamma(0.5 * d)


def entropy_from_rho(rho, d: int, k: int, form: str = "goria") -> float:
    """H_{n,k} of Eq. entropie_knn from the n distances rho_k(y_i)."""
    rho = np.asarray(rho, dtype=np.float64)
    n = rho.shape[0]
    if n < 2:
        raise ValueError("need at least two points")
    with np.errstate(divide="ignore"):
        lr = np.log(rho)
    if form == "goria":
        s = math.log(n - 1) + d * float(np.mean(lr))
    elif form == "printed":
        s = math.log(n - 1) + float(np.mean(lr))
    else:
        raise ValueError("form is 'goria' or 'printed'")
    return s + log_unit_ball(d) - digamma_int(k)


def entropy(index, k: int, form: str = "goria") -> float:
    """Entropy estimate of the index's reference points (Euclidean k-th
    neighbour distances among the other points, from knn_search_self)."""
    dist, _ = index.search_self(k, "l2")
    index.sync()
    rho = dist[:, k - 1].cpu().numpy()
    return entropy_from_rho(rho, index.d, k, form)


def majority_vote(neighbour_labels) -> np.ndarray:
    """Per row, the label most represented among the k neighbours; equal
    counts go to the smaller label."""
    lab = np.asarray(neighbour_labels)
    if lab.ndim != 2:
        raise ValueError("n x k labels")
    out = np.empty(lab.shape[0], dtype=lab.dtype)
    for i, row in enumerate(lab):
        vals, counts = np.unique(row, return_counts=True)
        out[i] = vals[np.argmax(counts)]          # np.unique sorts: first max = smallest label
    return out


def classify(index, labels, Q, k: int, metric: str = "l2") -> np.ndarray:
    """Label of each query by majority vote of its k nearest reference points
    (the reference points' labels in `labels`)."""
    _, idx = index.search(Q, k, metric)
    index.sync()
    idx = idx.cpu().numpy() if hasattr(idx, "cpu") else np.asarray(idx)
    return majority_vote(np.asarray(labels)[idx])
