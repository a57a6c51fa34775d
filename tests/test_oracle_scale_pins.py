"""Pins of the oracle's per-minibatch error scale (grad_abs), CPU only.

Every per-launch parity test divides the GPU's error by a scale that the
oracle returns beside its gradient: per pair, (|c| + |dc/dr| r_abs) |x_j|,
where the pair's term is c(r) x_j, r is the reduced scalar (the dot product
z_u . z_x for the sigmoid model, the squared distance q = |z_u - z_x|^2 for
the others), r_abs the same reduction over absolute values, and x the
partner row (sigmoid) or the difference z_u - z_x.  That is the first-order
size of the rounding error of an FP32 evaluation, so a scale that is too
large would loosen every such test without failing any.

These tests find c and dc/dr without the oracle's scale code: c from the
oracle's gradient of a single pair (g = c x), and dc/dr from central finite
differences of that gradient along a direction that changes r by a known
amount.  The scale the oracle returns must then equal (|c| + |dc/dr| r_abs)
|x| element by element.  The gradient itself is pinned separately (finite
differences of the loss of Eq. 2 and of the energies of Table
"diffmodels"), so a wrong factor anywhere in the scale fails here.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import graphs

ALL_MODELS = {"tdist": oracle.TDIST, "sigmoid": oracle.SIGMOID, "fr": oracle.FR,
              "linlog": oracle.LINLOG, "forceatlas": oracle.FORCEATLAS}


def _pair_case(kind, d, rng):
    """Two vertices; vertex 0's only pair is with vertex 1, as a neighbour
    (kind 'attr': one edge, s = 0) or as an injected negative sample (kind
    'rep': no edge, S(0) = [1])."""
    if kind == "attr":
        g = graphs.from_edges(2, [0], [1])
        injected = None
        s = 0
    else:
        g = graphs.from_edges(2, [], [])
        injected = [[1], []]
        s = 1
    Z = rng.uniform(-0.6, 0.6, size=(2, d))
    return g, Z, s, injected


def _grad(model, g, Z, s, injected):
    G, A = oracle.grad_minibatch_abs(model, g.row_ptr, g.col_idx, Z, 0, 1, s, 7, 0,
                                     injected=injected)
    return G[0], A[0]


@pytest.mark.parametrize("kind", ["attr", "rep"])
@pytest.mark.parametrize("name", list(ALL_MODELS))
def test_error_scale_from_finite_differences(name, kind):
    model = ALL_MODELS[name]
    rng = np.random.default_rng([list(ALL_MODELS).index(name), kind == "rep"])
    d = 6
    for trial in range(4):
        g, Z, s, injected = _pair_case(kind, d, rng)
        zu, zx = Z[0].copy(), Z[1].copy()
        G, A = _grad(model, g, Z, s, injected)
        if model == oracle.SIGMOID:
            x = zx
            r = float(zu @ zx)
            r_abs = float(np.abs(zu * zx).sum())
            # moving z_u along z_x / |z_x|^2 changes r by exactly h, x not at all
            direction = zx / float(zx @ zx)
            h = 1e-5

            def g_at(t):
                Zt = Z.copy()
                Zt[0] = zu + t * direction
                return _grad(model, g, Zt, s, injected)[0]
            dgdr = (g_at(h) - g_at(-h)) / (2 * h)
            c = G / x
            dc = dgdr / x
        else:
            x = zu - zx
            q = float(x @ x)
            r_abs = q
            # moving z_u to z_x + (1 + t) x scales x by (1 + t) and q by (1 + t)^2:
            # dg/dt at 0 = (c + 2 q dc/dq) x
            h = 1e-5

            def g_at(t):
                Zt = Z.copy()
                Zt[0] = zx + (1 + t) * x
                return _grad(model, g, Zt, s, injected)[0]
            dgdt = (g_at(h) - g_at(-h)) / (2 * h)
            c = G / x
            dc = (dgdt / x - c) / (2 * q)
        # c and dc/dr are one scalar each, the same for every element
        assert np.allclose(c, c[0], rtol=1e-9, atol=1e-12), (trial, c)
        assert np.allclose(dc, dc[0], rtol=1e-5, atol=1e-9), (trial, dc)
        want = (abs(c[0]) + abs(dc[0]) * r_abs) * np.abs(x)
        np.testing.assert_allclose(A, want, rtol=1e-6, atol=1e-12)


@pytest.mark.parametrize("name", ["tdist", "sigmoid"])
def test_error_scale_adds_over_pairs(name):
    """With several pairs the scale is the sum of the pairs' scales: a vertex
    with two neighbours and one injected sample against the three pairs
    evaluated one at a time (each alone in its own two-vertex graph)."""
    model = ALL_MODELS[name]
    rng = np.random.default_rng(3)
    d = 5
    Z = rng.uniform(-0.6, 0.6, size=(4, d))
    g = graphs.from_edges(4, [0, 0], [1, 2])
    _, A = oracle.grad_minibatch_abs(model, g.row_ptr, g.col_idx, Z, 0, 1, 1, 7, 0,
                                     injected=[[3], [], [], []])
    parts = []
    for v, kind in ((1, "attr"), (2, "attr"), (3, "rep")):
        Z2 = np.stack([Z[0], Z[v]])
        if kind == "attr":
            g2 = graphs.from_edges(2, [0], [1])
            parts.append(_grad(model, g2, Z2, 0, None)[1])
        else:
            g2 = graphs.from_edges(2, [], [])
            parts.append(_grad(model, g2, Z2, 1, [[1], []])[1])
    np.testing.assert_allclose(A[0], np.sum(parts, axis=0), rtol=1e-12)


def test_error_scale_bounds_an_fp32_evaluation():
    """The scale does what the parity tests use it for: an FP32 evaluation of
    z_u - eta * g (every product, reduction and sum rounded to FP32, pairs
    added in random orders) stays within a small multiple of FP32's unit
    roundoff times the scale, on a vertex with many pairs."""
    rng = np.random.default_rng(11)
    n, d, eta = 300, 16, 0.05
    g = graphs.erdos_renyi(n, p=0.3, seed=2)
    Z = rng.uniform(-0.5, 0.5, size=(n, d)).astype(np.float32).astype(np.float64)
    u = int(np.argmax(g.degrees()))
    G, A = oracle.grad_minibatch_abs(oracle.TDIST, g.row_ptr, g.col_idx, Z, u, u + 1, 0, 7, 0)
    want = Z[u] - eta * G[0]
    scale = np.abs(Z[u]) + eta * A[0]
    nbrs = g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]
    z32 = Z.astype(np.float32)
    worst = 0.0
    for _ in range(20):
        acc = np.zeros(d, np.float32)
        for v in rng.permutation(nbrs):
            df = z32[u] - z32[v]
            q = np.float32(np.sum(df * df, dtype=np.float32))
            c = np.float32(2) / (np.float32(1) + q)
            acc = acc + c * df
        got = z32[u] - np.float32(eta) * acc
        worst = max(worst, float((np.abs(got - want) / scale).max()))
    u32 = 2.0 ** -24
    assert worst <= 8 * u32 * 4, worst
