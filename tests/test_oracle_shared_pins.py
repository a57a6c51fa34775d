"""Pins of the oracle's shared-sample option: Algorithm 1's sampling step
read literally, one set S_b of s negative samples per minibatch used by
every vertex of it.

The shared draw is tied to facts outside its code: the injected-sample path
of Algorithm 2 (pinned by the closed forms of test_oracle_pins.py) must give
the same gradient when handed S_b for every vertex; the draws are uniform,
fresh for every minibatch and epoch, and not the per-vertex stream.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import graphs

MODELS = [oracle.TDIST, oracle.SIGMOID, oracle.FR]


def test_every_vertex_of_a_minibatch_shares_its_set():
    S = oracle.samples_shared(1000, 5, 128, 3, seed=4)
    for k in range(0, 1000, 128):
        blk = S[k:k + 128]
        assert (blk == blk[0]).all()
    firsts = [tuple(S[k]) for k in range(0, 1000, 128)]
    assert len(set(firsts)) == len(firsts)
    assert not np.array_equal(S, oracle.samples_shared(1000, 5, 128, 4, seed=4))


def test_shared_draws_are_uniform_and_not_the_vertex_stream():
    n = 50
    counts = np.zeros(n, np.int64)
    same = 0
    for e in range(40):
        S = oracle.samples_shared(n * 25, 4, 25, e, seed=9) % n   # 50 minibatches of 25
        for k in range(50):
            counts[S[k * 25] % n] += 1
    exp = counts.sum() / n
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 100.0, chi2                # 49 dof: p ~ 3e-5
    per_vertex = oracle.samples(1000, 4, 0, seed=9)
    shared = oracle.samples_shared(1000, 4, 1, 0, seed=9)    # b = 1: k = u
    same = int((per_vertex == shared).sum())
    assert same < 40, same                   # ~4 of 4000 agree by chance


@pytest.mark.parametrize("model", MODELS)
def test_shared_gradient_is_the_injected_gradient(model):
    g = graphs.erdos_renyi(300, p=0.03, seed=2)
    Z = oracle.init_embedding(300, 6, seed=5)
    b, s, ep = 64, 4, 2
    S = oracle.samples_shared(300, s, b, ep, seed=7)
    for k0 in range(0, 300, b):
        k1 = min(300, k0 + b)
        got = oracle.grad_minibatch(model, g.row_ptr, g.col_idx, Z, k0, k1, s, seed=7, epoch=ep,
                                    shared_b=b)
        want = oracle.grad_minibatch(model, g.row_ptr, g.col_idx, Z, k0, k1, s, seed=7,
                                     epoch=ep, injected=[list(r) for r in S])
        np.testing.assert_array_equal(got, want)


def test_shared_training_draws_new_sets_each_epoch():
    g = graphs.erdos_renyi(200, p=0.04, seed=3)
    Z0 = oracle.init_embedding(200, 5, seed=1)
    b, s = 50, 3
    got = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z0, s, b, seed=2, lr=0.05, epochs=3,
                       shared=True)
    Z = Z0.copy()
    for e in range(3):
        S = oracle.samples_shared(200, s, b, e, seed=2)
        Z = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z, s, b, seed=2, lr=0.05, epochs=1,
                         start_epoch=e, injected=[list(r) for r in S])
    np.testing.assert_array_equal(got, Z)
