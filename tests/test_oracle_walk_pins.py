"""Pins of the oracle's rForce2Vec path (Algorithm 3, random-walk N(u)).

Each test ties the walk, or the gradient built from it, to a fact outside
the walk code: the graph's own edges, the uniform law of a fair neighbour
choice, a graph on which every walk is forced (a perfect matching, a star, a
one-way chain), and the 1-hop gradient of Algorithm 2, which the closed-form
and finite-difference pins of test_oracle_pins.py fix.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import graphs

MODELS = {"tdist": oracle.TDIST, "sigmoid": oracle.SIGMOID}


def _csr_from_lists(adj):
    rp = np.zeros(len(adj) + 1, np.int32)
    rp[1:] = np.cumsum([len(a) for a in adj])
    ci = np.array([v for a in adj for v in a], np.int32)
    return rp, ci


def _matching(n):
    """Perfect matching 0-1, 2-3, ...: every walk alternates v, u, v, u, ..."""
    return _csr_from_lists([[u ^ 1] for u in range(n)])


def test_every_step_moves_along_an_edge():
    g = graphs.erdos_renyi(300, p=0.03, seed=4)
    rp, ci = g.row_ptr, g.col_idx
    for epoch in (0, 3):
        for u in range(0, 300, 7):
            w = oracle.walk(rp, ci, u, epoch, 9, seed=11)
            if rp[u + 1] == rp[u]:
                assert (w == -1).all()
                continue
            prev = u
            for x in w:
                assert x in ci[rp[prev]:rp[prev + 1]], (u, prev, x)
                prev = x


def test_neighbour_choice_is_uniform_and_fresh_each_epoch():
    # star: centre 0, leaves 1..8; the walk from the centre picks a leaf,
    # comes back, picks a leaf ...
    leaves = 8
    rp, ci = _csr_from_lists([list(range(1, leaves + 1))] + [[0]] * leaves)
    counts = np.zeros(leaves + 1, np.int64)
    walks = []
    for epoch in range(3000):
        w = oracle.walk(rp, ci, 0, epoch, 6, seed=5)
        assert (w[1::2] == 0).all()                 # back at the centre every second step
        for x in w[0::2]:
            counts[x] += 1
        walks.append(tuple(w))
    obs = counts[1:]
    exp = obs.sum() / leaves
    chi2 = float(((obs - exp) ** 2 / exp).sum())
    assert chi2 < 30.0, chi2          # 7 dof: p ~ 1e-4
    # 8^3 = 512 possible walks: all appear, and an epoch repeats the walk of
    # the one before about once in 512
    assert len(set(walks)) >= 500
    repeats = sum(a == b for a, b in zip(walks, walks[1:]))
    assert repeats < 20, repeats


def test_walk_stops_at_a_vertex_without_neighbours():
    # one-way chain 0 -> 1 -> 2, and 2 has no out-neighbours (not symmetric)
    rp, ci = _csr_from_lists([[1], [2], []])
    assert oracle.walk(rp, ci, 0, 0, 5, seed=1).tolist() == [1, 2, -1, -1, -1]
    assert oracle.walk(rp, ci, 2, 0, 5, seed=1).tolist() == [-1] * 5


def test_walk_stream_is_not_the_sample_stream():
    g = graphs.erdos_renyi(200, p=0.5, seed=2)
    n = 200
    same = 0
    for u in range(n):
        w = oracle.walk(g.row_ptr, g.col_idx, u, 0, 1, seed=9)[0]
        lo, hi = g.row_ptr[u], g.row_ptr[u + 1]
        k = int(np.flatnonzero(g.col_idx[lo:hi] == w)[0])
        # the sample of counter (u, 0, 0, 0) taken mod deg(u) would pick index k
        # every time if the two streams coincided
        x = oracle.philox4x32_10([u, 0, 0, 0], [9, 0])[0]
        same += int(x % (hi - lo) == k)
    assert same < n // 4


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_walks_on_a_matching_equal_the_tripled_edges(model):
    """On a perfect matching a walk of 5 steps from u is v, u, v, u, v; the
    steps back at u add nothing, so rForce2Vec's N(u) is v three times: the
    1-hop method on the matching with every CSR entry written three times."""
    n, d, s = 24, 6, 3
    rp, ci = _matching(n)
    rp3, ci3 = _csr_from_lists([[u ^ 1] * 3 for u in range(n)])
    Z = oracle.init_embedding(n, d, seed=3) * 2.0
    m = MODELS[model]
    for u in range(n):
        assert oracle.walk(rp, ci, u, 2, 5, seed=8).tolist() == [u ^ 1, u, u ^ 1, u, u ^ 1]
    g_walk = oracle.grad_minibatch(m, rp, ci, Z, 0, n, s, seed=8, epoch=2, walk=5)
    g_hop = oracle.grad_minibatch(m, rp3, ci3, Z, 0, n, s, seed=8, epoch=2)
    np.testing.assert_array_equal(g_walk, g_hop)
    z_walk = oracle.train(m, rp, ci, Z, s, 5, seed=8, lr=0.05, epochs=3, walk=5)
    z_hop = oracle.train(m, rp3, ci3, Z, s, 5, seed=8, lr=0.05, epochs=3)
    np.testing.assert_array_equal(z_walk, z_hop)


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_walk_gradient_is_the_gradient_of_its_multiset(model):
    """The walk's pairs are ordinary attractive pairs: the gradient equals
    Algorithm 2 on a graph whose row u lists the walk's vertices (self
    visits dropped), with the same negative samples."""
    g = graphs.erdos_renyi(60, p=0.08, seed=6)
    n, d, s, k, ep = 60, 5, 4, 5, 1
    Z = oracle.init_embedding(n, d, seed=2)
    adj = []
    for u in range(n):
        w = oracle.walk(g.row_ptr, g.col_idx, u, ep, k, seed=13)
        adj.append([int(x) for x in w if x >= 0 and x != u])
    rpw, ciw = _csr_from_lists(adj)
    m = MODELS[model]
    got = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, n, s, seed=13, epoch=ep, walk=k)
    want = oracle.grad_minibatch(m, rpw, ciw, Z, 0, n, s, seed=13, epoch=ep)
    np.testing.assert_array_equal(got, want)


def test_isolated_vertex_feels_only_its_samples():
    # vertex 4 has no neighbours: no walk, so only the repulsive terms remain,
    # as in the 1-hop method
    rp, ci = _csr_from_lists([[1], [0, 2], [1, 3], [2], []])
    Z = oracle.init_embedding(5, 4, seed=1)
    for m in (oracle.TDIST, oracle.SIGMOID):
        g_walk = oracle.grad_minibatch(m, rp, ci, Z, 4, 5, 3, seed=2, epoch=0, walk=5)
        g_hop = oracle.grad_minibatch(m, rp, ci, Z, 4, 5, 3, seed=2, epoch=0)
        np.testing.assert_array_equal(g_walk, g_hop)
