"""Pins of the oracle's random-partition option: Algorithm 1's partition
step read literally, a new partition of V into minibatches every epoch.

The partitioned run is tied to the contiguous one, which the other pins fix:
one epoch over the partition of epoch e is one epoch of the contiguous
method on the graph relabelled so that the partition's order becomes id
order (same samples, same neighbour order), mapped back.  The partition is
a permutation, new every epoch, and places a vertex uniformly.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import graphs


def test_partition_is_a_fresh_uniform_permutation():
    n = 40
    firsts = np.zeros(n, np.int64)
    perms = set()
    for e in range(2000):
        p = oracle.partition(n, e, seed=6)
        assert np.array_equal(np.sort(p), np.arange(n))
        perms.add(tuple(p))
        firsts[p[0]] += 1
    assert len(perms) == 2000
    exp = firsts.sum() / n
    chi2 = float(((firsts - exp) ** 2 / exp).sum())
    assert chi2 < 80.0, chi2                  # 39 dof: p ~ 1e-4


def _relabel(g, perm):
    rank = np.empty_like(perm)
    rank[perm] = np.arange(perm.size)
    rows = [rank[g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]] for u in perm]
    rp = np.zeros(perm.size + 1, np.int32)
    rp[1:] = np.cumsum([r.size for r in rows])
    ci = np.concatenate(rows).astype(np.int32) if rp[-1] else np.zeros(0, np.int32)
    return rp, ci, rank


@pytest.mark.parametrize("model", [oracle.TDIST, oracle.SIGMOID, oracle.LINLOG])
def test_partitioned_epoch_is_the_contiguous_epoch_of_the_relabelled_graph(model):
    g = graphs.erdos_renyi(300, p=0.02, seed=7)
    n, d, b, s, e = 300, 6, 64, 3, 4
    Z = oracle.init_embedding(n, d, seed=2)
    rng = np.random.default_rng(1)
    S = [list(rng.integers(0, n, s)) for _ in range(n)]
    got = oracle.train(model, g.row_ptr, g.col_idx, Z, s, b, seed=5, lr=0.05, epochs=1,
                       start_epoch=e, injected=S, partition=True)
    perm = oracle.partition(n, e, seed=5)
    rp, ci, rank = _relabel(g, perm)
    S2 = [[int(rank[w]) for w in S[u]] for u in perm]
    Z2 = oracle.train(model, rp, ci, Z[perm], s, b, seed=5, lr=0.05, epochs=1, start_epoch=e,
                      injected=S2)
    want = np.empty_like(Z2)
    want[perm] = Z2
    np.testing.assert_array_equal(got, want)


def test_first_minibatch_updates_exactly_its_vertices():
    g = graphs.erdos_renyi(500, p=0.02, seed=3)
    Z = oracle.init_embedding(500, 4, seed=1)
    out = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z, 5, 100, seed=8, lr=0.05, epochs=1,
                       start_epoch=2, max_minibatches=1, partition=True)
    changed = np.flatnonzero((out != Z).any(axis=1))
    first = oracle.partition(500, 2, seed=8)[:100]
    assert set(changed) <= set(first)
    assert len(changed) >= 90


def test_shared_samples_follow_the_minibatch_index():
    # with a partition, minibatch k's shared set is still S_k: the gradient
    # of its vertices equals Algorithm 2 with S_k injected for each
    g = graphs.erdos_renyi(200, p=0.03, seed=4)
    Z = oracle.init_embedding(200, 5, seed=3)
    perm = oracle.partition(200, 1, seed=9)
    verts = perm[50:100]                      # minibatch k = 1 of b = 50
    got, _ = oracle.grad_vertices_abs(oracle.TDIST, g.row_ptr, g.col_idx, Z, verts, 4, 9, 1,
                                      shared_k=1)
    Sk = oracle.samples_shared(200, 4, 50, 1, seed=9)[50]
    want = np.stack([oracle.grad_minibatch(oracle.TDIST, g.row_ptr, g.col_idx, Z, int(u),
                                           int(u) + 1, 4, 9, 1,
                                           injected=[list(Sk)] * 200)[0] for u in verts])
    np.testing.assert_array_equal(got, want)
