"""Pins of the downstream-evaluation oracle (Sec. IV: link prediction with
Hadamard features and logistic regression; k-means clustering scored by
modularity) against library routines and closed forms.
"""
import numpy as np
import pytest

from oracle import downstream as ds
from paper_2009_10035_gb300 import graphs


def test_logreg_matches_scikit_learn():
    sk = pytest.importorskip("sklearn.linear_model")
    rng = np.random.default_rng(3)
    X = rng.normal(size=(600, 7))
    w_true = rng.normal(size=7)
    y = (X @ w_true + 0.3 + rng.normal(scale=1.5, size=600) > 0).astype(float)
    w, b = ds.logreg_fit(X, y)
    ref = sk.LogisticRegression(C=1.0, solver="lbfgs", tol=1e-12, max_iter=100000).fit(X, y)
    np.testing.assert_allclose(w, ref.coef_[0], rtol=1e-5, atol=1e-7)
    assert b == pytest.approx(ref.intercept_[0], rel=1e-5, abs=1e-7)


def test_link_accuracy_protocol():
    # pairs whose Hadamard features separate perfectly: every test pair right
    rng = np.random.default_rng(1)
    Z = rng.normal(size=(200, 4))
    Z[:100, 0] = np.abs(Z[:100, 0]) + 1.0     # vertices 0..99: positive first coordinate
    Z[100:, 0] = -np.abs(Z[100:, 0]) - 1.0    # 100..199: negative
    pos = np.array([(i, (i + 1) % 100) for i in range(100)])            # product > 0
    neg = np.array([(i, 100 + (i * 7) % 100) for i in range(100)])      # product < 0
    mask = np.zeros(200, bool)
    mask[::2] = True
    acc, w, b = ds.link_accuracy(Z, pos, neg, mask)
    assert acc == 1.0 and w[0] > 0


def test_kmeans_matches_scikit_learn():
    skc = pytest.importorskip("sklearn.cluster")
    rng = np.random.default_rng(5)
    centres = rng.normal(scale=4.0, size=(6, 5))
    Z = np.vstack([c + rng.normal(size=(80, 5)) for c in centres])
    init = rng.choice(Z.shape[0], 6, replace=False)
    labels, C, _ = ds.kmeans(Z, init, iters=300)
    ref = skc.KMeans(n_clusters=6, init=Z[init], n_init=1, algorithm="lloyd", tol=0.0,
                     max_iter=300).fit(Z)
    np.testing.assert_array_equal(labels, ref.labels_)
    np.testing.assert_allclose(C, ref.cluster_centers_, rtol=1e-10, atol=1e-10)


def test_modularity_matches_networkx():
    nx = pytest.importorskip("networkx")
    g = graphs.erdos_renyi(300, p=0.03, seed=9)
    rng = np.random.default_rng(2)
    labels = rng.integers(0, 5, g.n)
    G = nx.Graph()
    G.add_nodes_from(range(g.n))
    for u in range(g.n):
        for v in g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]:
            if u < v:
                G.add_edge(u, int(v))
    comms = [set(np.flatnonzero(labels == c).tolist()) for c in range(5)]
    want = nx.community.modularity(G, comms)
    assert ds.modularity(g.row_ptr, g.col_idx, labels) == pytest.approx(want, abs=1e-12)


def test_modularity_closed_forms():
    # two disjoint triangles: right split Q = 2 (3/6 - (6/12)^2) = 1/2; one cluster Q = 0
    rp = np.array([0, 2, 4, 6, 8, 10, 12])
    ci = np.array([1, 2, 0, 2, 0, 1, 4, 5, 3, 5, 3, 4])
    assert ds.modularity(rp, ci, [0, 0, 0, 1, 1, 1]) == pytest.approx(0.5, abs=1e-15)
    assert ds.modularity(rp, ci, [0] * 6) == pytest.approx(0.0, abs=1e-15)


def test_kmeans_tie_goes_to_the_lowest_index():
    # 1-D points 0, 2, 1; centres start at 0 and 2; the point at 1 is as far
    # from both and joins centre 0, which moves to 0.5 and keeps it:
    # labels (0, 1, 0).  (Ties to the highest index would end at (0, 1, 1).)
    labels, C, _ = ds.kmeans(np.array([[0.0], [2.0], [1.0]]), [0, 1], iters=10)
    assert labels.tolist() == [0, 1, 0]
    np.testing.assert_allclose(C[:, 0], [0.5, 2.0])


def test_kmeans_empty_cluster_keeps_its_centre():
    # points 5, 5, 20; both centres start at 5: every point ties and joins
    # centre 0 (mean 10) while cluster 1 is empty and stays at 5; then the
    # two 5s move to centre 1: labels (1, 1, 0), centres (20, 5).
    labels, C, _ = ds.kmeans(np.array([[5.0], [5.0], [20.0]]), [0, 1], iters=10)
    assert labels.tolist() == [1, 1, 0]
    np.testing.assert_allclose(C[:, 0], [20.0, 5.0])
