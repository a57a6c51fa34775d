"""Pins of the oracle's other force models (Table "diffmodels"):
Fruchterman-Reingold, LinLog and ForceAtlas.

The table lists each model's force along the unit vector: -t^2, -log(1 + t)
and -t for a neighbour at distance t, 1/t for a sample.  The pins check the
oracle against facts outside its code:
  - finite differences of the energies whose derivatives are those force
    magnitudes, written here by integrating them: t^3/3, (1+t)log(1+t) - t,
    t^2/2 for the attraction and -log t for the repulsion;
  - single steps worked by hand on two vertices at distance 5;
  - direction: attraction shortens the distance, repulsion lengthens it;
  - invariants: translation and rotation of Z, and Newton's third law.
"""
import math

import numpy as np
import pytest

import oracle

MODELS = {"fr": oracle.FR, "linlog": oracle.LINLOG, "forceatlas": oracle.FORCEATLAS}

E_ATTR = {
    oracle.FR: lambda t: t ** 3 / 3.0,
    oracle.LINLOG: lambda t: (1.0 + t) * math.log1p(t) - t,
    oracle.FORCEATLAS: lambda t: t * t / 2.0,
}


def e_rep(t):
    return -math.log(t)


def _csr(adj):
    rp = np.zeros(len(adj) + 1, np.int32)
    rp[1:] = np.cumsum([len(a) for a in adj])
    ci = np.array([v for a in adj for v in a], np.int32)
    return rp, ci


def _energy(model, Z, u, nbrs, samples):
    e = 0.0
    for v in nbrs:
        e += E_ATTR[model](float(np.linalg.norm(Z[u] - Z[v])))
    for w in samples:
        if w != u:
            e += e_rep(float(np.linalg.norm(Z[u] - Z[w])))
    return e


@pytest.mark.parametrize("name", list(MODELS))
def test_gradient_is_the_derivative_of_the_energy(name):
    model = MODELS[name]
    rng = np.random.default_rng(3)
    n, d = 10, 4
    adj = [[] for _ in range(n)]
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < 0.35:
                adj[u].append(v)
                adj[v].append(u)
    rp, ci = _csr(adj)
    samples = [list(rng.integers(0, n, 3)) for _ in range(n)]
    Z = rng.uniform(-1.0, 1.0, (n, d))
    G = oracle.grad_minibatch(model, rp, ci, Z, 0, n, 3, seed=1, epoch=0, injected=samples)
    h = 1e-6
    for u in range(n):
        for j in range(d):
            Zp, Zm = Z.copy(), Z.copy()
            Zp[u, j] += h
            Zm[u, j] -= h
            fd = (_energy(model, Zp, u, adj[u], samples[u]) -
                  _energy(model, Zm, u, adj[u], samples[u])) / (2 * h)
            assert abs(fd - G[u, j]) <= 1e-6 * max(1.0, abs(fd)), (u, j, fd, G[u, j])


def _pair(model, edge, eta):
    """Two vertices z0 = (0, 0), z1 = (3, 4), minibatch size 1 (vertex 0 is
    updated first, then vertex 1 sees its new row); an edge, or each the
    other's only sample."""
    Z = np.array([[0.0, 0.0], [3.0, 4.0]])
    if edge:
        rp, ci = _csr([[1], [0]])
        return oracle.train(model, rp, ci, Z, 0, 1, seed=1, lr=eta, epochs=1)
    rp, ci = _csr([[], []])
    return oracle.train(model, rp, ci, Z, 1, 1, seed=1, lr=eta, epochs=1,
                        injected=[[1], [0]])


def test_fr_attraction_step_by_hand():
    # vertex 0: force -t^2 = -25 along (z0 - z1)/5 = (-0.6, -0.8): gradient
    # 25 * (-0.6, -0.8) = (-15, -20); z0 = (0.15, 0.20).  Vertex 1 then sits
    # at (2.85, 3.8) from it, t = 4.75: gradient 4.75 * (2.85, 3.8) =
    # (13.5375, 18.05); z1 = (3 - 0.135375, 4 - 0.1805).
    Z = _pair(oracle.FR, True, 0.01)
    np.testing.assert_allclose(Z, [[0.15, 0.20], [2.864625, 3.8195]], rtol=0, atol=1e-12)


def test_forceatlas_attraction_step_by_hand():
    # force -t: gradient t * unit = z0 - z1 = (-3, -4): z0 = (0.03, 0.04);
    # then z1 - z0 = (2.97, 3.96): z1 = (2.9703, 3.9604)
    Z = _pair(oracle.FORCEATLAS, True, 0.01)
    np.testing.assert_allclose(Z, [[0.03, 0.04], [2.9703, 3.9604]], rtol=0, atol=1e-12)


def test_linlog_attraction_step_by_hand():
    # force -log(1 + 5) = -log 6 along (-0.6, -0.8): z0 moves 0.01 log 6
    # toward z1; then vertex 1 moves 0.01 log(1 + t') toward z0, with
    # t' = 5 - 0.01 log 6, the two moves along the same line
    Z = _pair(oracle.LINLOG, True, 0.01)
    a = 0.01 * math.log(6.0)
    t1 = 5.0 - a
    b = 0.01 * math.log(1.0 + t1)
    np.testing.assert_allclose(Z[0], [0.6 * a, 0.8 * a], rtol=0, atol=1e-12)
    np.testing.assert_allclose(Z[1], [3.0 - 0.6 * b, 4.0 - 0.8 * b], rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", list(MODELS))
def test_repulsion_step_by_hand_and_the_bound(name):
    # force 1/t = 0.2 away from z1: gradient -(1/t) * (-0.6, -0.8) =
    # (0.12, 0.16); z0 = (-0.0012, -0.0016).  Vertex 1 is then pushed
    # along (3.0012, 4.0016) / t^2 with t^2 = 25.020004: its second
    # coordinate passes 4 and is held at the bound.
    Z = _pair(MODELS[name], False, 0.01)
    np.testing.assert_allclose(Z[0], [-0.0012, -0.0016], rtol=0, atol=1e-15)
    assert Z[1, 0] == pytest.approx(3.0 + 0.01 * 3.0012 / 25.020004, abs=1e-15)
    assert Z[1, 1] == 4.0


@pytest.mark.parametrize("name", list(MODELS))
def test_attraction_shortens_and_repulsion_lengthens(name):
    model = MODELS[name]
    rng = np.random.default_rng(8)
    for _ in range(20):
        Z = rng.uniform(-0.5, 0.5, (2, 6))
        t0 = np.linalg.norm(Z[0] - Z[1])
        rp, ci = _csr([[1], [0]])
        Za = oracle.train(model, rp, ci, Z, 0, 2, seed=1, lr=0.01, epochs=1)
        assert np.linalg.norm(Za[0] - Za[1]) < t0
        rp, ci = _csr([[], []])
        Zr = oracle.train(model, rp, ci, Z, 1, 2, seed=1, lr=0.01, epochs=1, injected=[[1], [0]])
        assert np.linalg.norm(Zr[0] - Zr[1]) > t0


def _random_graph(n, p, seed):
    rng = np.random.default_rng(seed)
    adj = [[] for _ in range(n)]
    for u in range(n):
        for v in range(u + 1, n):
            if rng.random() < p:
                adj[u].append(v)
                adj[v].append(u)
    return _csr(adj)


@pytest.mark.parametrize("name", list(MODELS))
def test_translation_and_rotation_commute_with_training(name):
    model = MODELS[name]
    rp, ci = _random_graph(20, 0.2, 4)
    rng = np.random.default_rng(5)
    Z = rng.uniform(-0.3, 0.3, (20, 3))
    samples = [list(rng.integers(0, 20, 2)) for _ in range(20)]
    base = oracle.train(model, rp, ci, Z, 2, 5, seed=1, lr=0.002, epochs=2, injected=samples)
    assert np.abs(base).max() < 3.0           # away from the coordinate bound
    shift = np.array([0.4, -0.2, 0.3])
    moved = oracle.train(model, rp, ci, Z + shift, 2, 5, seed=1, lr=0.002, epochs=2,
                         injected=samples)
    np.testing.assert_allclose(moved - shift, base, rtol=0, atol=1e-12)
    Q, _ = np.linalg.qr(rng.normal(size=(3, 3)))
    rot = oracle.train(model, rp, ci, Z @ Q, 2, 5, seed=1, lr=0.002, epochs=2,
                       injected=samples)
    np.testing.assert_allclose(rot @ Q.T, base, rtol=0, atol=1e-12)


@pytest.mark.parametrize("name", list(MODELS))
def test_attractive_forces_balance(name):
    # with no samples the attraction on u from v is minus that on v from u
    rp, ci = _random_graph(15, 0.3, 6)
    Z = np.random.default_rng(7).uniform(-1, 1, (15, 4))
    G = oracle.grad_minibatch(MODELS[name], rp, ci, Z, 0, 15, 0, seed=1, epoch=0)
    np.testing.assert_allclose(G.sum(axis=0), 0.0, atol=1e-12)


def test_models_differ_only_in_the_attraction():
    rp, ci = _random_graph(12, 0.3, 9)
    Z = np.random.default_rng(1).uniform(-1, 1, (12, 5))
    samples = [[int((u * 7 + 3) % 12)] for u in range(12)]
    rep_only = [oracle.grad_minibatch(m, np.zeros(13, np.int32), np.zeros(0, np.int32), Z, 0,
                                      12, 1, seed=1, epoch=0, injected=samples)
                for m in MODELS.values()]
    np.testing.assert_array_equal(rep_only[0], rep_only[1])
    np.testing.assert_array_equal(rep_only[0], rep_only[2])
    att = [oracle.grad_minibatch(m, rp, ci, Z, 0, 12, 0, seed=1, epoch=0) for m in MODELS.values()]
    assert not np.allclose(att[0], att[1]) and not np.allclose(att[1], att[2])
