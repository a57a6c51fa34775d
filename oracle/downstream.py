"""FP64 oracle of the downstream evaluations of Sec. IV (test infrastructure
only: the test suite, smoke() and bench.py's CPU leg may use it; the product
library never does).

  hadamard        the link-prediction features of Sec. IV ("Link
                  prediction"): z_u * z_v element by element for a pair
  logreg_fit      L2-regularised logistic regression (penalty 1/2 |w|^2 on
                  the weights, the intercept unpenalised; the common default
                  C = 1), fitted by Newton's method
  link_accuracy   the protocol of that paragraph: fit on the training half,
                  accuracy (TP + TN) / (all test pairs) on the other half
  kmeans          Lloyd's k-means (Sec. IV, "Clustering") from given centres
  modularity      the modularity of a clustering (Sec. IV, "Clustering"):
                  the fraction of edges inside clusters minus its expectation
                  when edges are placed at random with the same degrees

Random choices (the train/test split, the initial centres) are inputs.
Readings: Newton stops when the step's max-norm is below 1e-10 or after 100
iterations; k-means assigns a point to the nearest centre (the lowest index
on an exact tie), keeps the centre of a cluster that becomes empty, and
stops when no label changes or after `iters` iterations.
"""
from __future__ import annotations

import numpy as np


def hadamard(Z, pairs) -> np.ndarray:
    Z = np.asarray(Z, dtype=np.float64)
    pairs = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    return Z[pairs[:, 0]] * Z[pairs[:, 1]]


def _sigmoid(t):
    return 0.5 * (1.0 + np.tanh(0.5 * t))


def logreg_fit(X, y, max_iter: int = 100, tol: float = 1e-10):
    """Minimises sum_i log(1 + exp(-s_i (w . x_i + b))) + |w|^2 / 2 with
    s_i = 2 y_i - 1; returns (w, b)."""
    X = np.asarray(X, dtype=np.float64)
    y = np.asarray(y, dtype=np.float64)
    m, d = X.shape
    A = np.hstack([X, np.ones((m, 1))])
    theta = np.zeros(d + 1)
    reg = np.ones(d + 1)
    reg[d] = 0.0                                   # the intercept is not penalised
    for _ in range(max_iter):
        p = _sigmoid(A @ theta)
        g = A.T @ (p - y) + reg * theta
        H = (A * (p * (1.0 - p))[:, None]).T @ A + np.diag(reg)
        step = np.linalg.solve(H, g)
        theta -= step
        if np.abs(step).max() < tol:
            break
    return theta[:d], theta[d]


def link_accuracy(Z, pos_pairs, neg_pairs, train_mask):
    """Hadamard features, label 1 for pos_pairs and 0 for neg_pairs (pos
    first); fit on train_mask, accuracy on the rest.  Returns (accuracy, w, b)."""
    X = np.vstack([hadamard(Z, pos_pairs), hadamard(Z, neg_pairs)])
    y = np.concatenate([np.ones(len(np.asarray(pos_pairs).reshape(-1, 2))),
                        np.zeros(len(np.asarray(neg_pairs).reshape(-1, 2)))])
    tr = np.asarray(train_mask, dtype=bool)
    w, b = logreg_fit(X[tr], y[tr])
    pred = (X[~tr] @ w + b) > 0.0
    return float((pred == (y[~tr] > 0.5)).mean()), w, b


def kmeans(Z, init, iters: int = 100):
    """Lloyd's algorithm from centres Z[init]; returns (labels, centres, iterations)."""
    Z = np.asarray(Z, dtype=np.float64)
    C = Z[np.asarray(init, dtype=np.int64)].copy()
    labels = None
    it = 0
    for it in range(1, iters + 1):
        d2 = ((Z[:, None, :] - C[None, :, :]) ** 2).sum(axis=2)
        new = np.argmin(d2, axis=1)                # lowest index on a tie
        if labels is not None and np.array_equal(new, labels):
            break
        labels = new
        for c in range(C.shape[0]):
            members = labels == c
            if members.any():                      # an empty cluster keeps its centre
                C[c] = Z[members].mean(axis=0)
    return labels, C, it


def modularity(row_ptr, col_idx, labels) -> float:
    """Q = sum_c [ e_c / (2m) - (D_c / (2m))^2 ]: e_c the CSR entries with both
    ends in c (each undirected edge appears twice, so e_c / 2m is the
    fraction of edges inside c), D_c the summed degree of c, 2m = nnz."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col_idx = np.asarray(col_idx, dtype=np.int64)
    labels = np.asarray(labels, dtype=np.int64)
    nnz = int(row_ptr[-1])
    if nnz == 0:
        return 0.0
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(labels.size), deg)
    inside = labels[src] == labels[col_idx]
    K = int(labels.max()) + 1
    e = np.bincount(labels[src][inside], minlength=K).astype(np.float64)
    D = np.bincount(labels, weights=deg, minlength=K)
    return float((e / nnz - (D / nnz) ** 2).sum())
