"""Pins of the FP64 oracle against facts fixed outside it.

Each test checks the oracle against something it cannot agree with by
construction: a library routine (cuRAND's host Philox), hand-derived closed
forms (tests/golden/closed_form_steps.json), finite differences of the
paper's objective, a brute-force all-pairs objective written separately here,
and invariants of the mathematics (relabelling, rotation, translation,
Newton's third law of the t-model forces).
"""
import ctypes
import ctypes.util
import json
import math
import os

import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import graphs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "closed_form_steps.json")
MODELS = {"tdist": oracle.TDIST, "sigmoid": oracle.SIGMOID}


# --------------------------------------------------------------------------
# Philox4x32-10 against cuRAND's host generator
# --------------------------------------------------------------------------

def _curand():
    cands = ["/usr/local/cuda/lib64/libcurand.so", ctypes.util.find_library("curand")]
    for c in cands:
        if c and (os.path.exists(c) or not c.startswith("/")):
            try:
                return ctypes.CDLL(c)
            except OSError:
                continue
    return None


def _curand_block(lib, seed, c0, c1, c2):
    """cuRAND's host PHILOX4_32_10 generator emits, at output offset
    4 * ((c1:c0) * 65536 + c2), the four words of Philox(ctr=(c0,c1,c2,0),
    key=(seed lo, seed hi)).  (Counter layout of its 65536 interleaved
    subsequences, established against the library's own output.)"""
    gen = ctypes.c_void_p()
    assert lib.curandCreateGeneratorHost(ctypes.byref(gen), ctypes.c_int(161)) == 0   # CURAND_RNG_PSEUDO_PHILOX4_32_10
    try:
        assert lib.curandSetPseudoRandomGeneratorSeed(gen, ctypes.c_ulonglong(seed)) == 0
        off = 4 * ((((c1 << 32) | c0) << 16) + c2)
        assert lib.curandSetGeneratorOffset(gen, ctypes.c_ulonglong(off)) == 0
        out = (ctypes.c_uint * 4)()
        assert lib.curandGenerate(gen, out, ctypes.c_size_t(4)) == 0
        return [int(x) for x in out]
    finally:
        lib.curandDestroyGenerator(gen)


def test_philox_matches_curand_host_generator():
    lib = _curand()
    if lib is None:
        pytest.skip("libcurand not available")
    rng = np.random.default_rng(3)
    cases = [(0, 0, 0, 0), (1, 0, 0, 0), (0x123456789abcdef, 5, 1, 3),
             (2**64 - 1, 2**32 - 1, 7, 65535), (42, 999_999, 19, 0xFFFF)]
    for _ in range(40):
        cases.append((int(rng.integers(0, 2**63)), int(rng.integers(0, 2**32)),
                      int(rng.integers(0, 64)), int(rng.integers(0, 65536))))
    for seed, c0, c1, c2 in cases:
        want = _curand_block(lib, seed, c0, c1, c2)
        got = oracle.philox4x32_10([c0, c1, c2, 0], [seed & 0xFFFFFFFF, seed >> 32])
        assert [int(x) for x in got] == want, (seed, c0, c1, c2)


def test_sample_and_init_use_their_counters():
    seed = 0xDEADBEEF12345
    key = [seed & 0xFFFFFFFF, seed >> 32]
    n = 1000
    for u, e, k in [(0, 0, 0), (17, 3, 4), (999, 19, 9)]:
        x0 = int(oracle.philox4x32_10([u, e, k, 0], key)[0])
        assert int(oracle.samples(n, k + 1, e, seed)[u, k]) == x0 % n
    Z = oracle.init_embedding(5, 3, seed)
    for i in range(5):
        for j in range(3):
            x0 = int(oracle.philox4x32_10([i, j, 0xFFFF, 0], key)[0])
            assert Z[i, j] == (x0 >> 8) * 2.0**-24 - 0.5


def test_init_embedding_range_and_uniformity():
    Z = oracle.init_embedding(4000, 32, 1)
    assert Z.min() >= -0.5 and Z.max() < 0.5
    scaled = (Z + 0.5) * 2**24
    assert np.array_equal(scaled, np.round(scaled))      # exact in FP32 as well
    assert np.array_equal(Z.astype(np.float32).astype(np.float64), Z)
    hist, _ = np.histogram(Z, bins=32, range=(-0.5, 0.5))
    expected = Z.size / 32
    chi2 = float(((hist - expected) ** 2 / expected).sum())
    assert chi2 < 80.0          # 31 dof: p ~ 1e-5 threshold


def test_negative_samples_uniform_and_fresh_each_epoch():
    n, s = 997, 8
    S0 = oracle.samples(n, s, 0, 5)
    S1 = oracle.samples(n, s, 1, 5)
    assert S0.min() >= 0 and S0.max() < n
    assert (S0 != S1).mean() > 0.99
    allS = np.concatenate([oracle.samples(n, s, e, 5).ravel() for e in range(40)])
    hist = np.bincount(allS, minlength=n)
    expected = allS.size / n
    chi2 = float(((hist - expected) ** 2 / expected).sum())
    assert chi2 < n + 6 * math.sqrt(2 * n)


# --------------------------------------------------------------------------
# Hand-derived closed forms
# --------------------------------------------------------------------------

def _golden():
    with open(GOLDEN) as f:
        return json.load(f)


def _graph_from_case(case):
    e = np.asarray(case["edges"], dtype=np.int64).reshape(-1, 2)
    return graphs.from_edges(case["n"], e[:, 0], e[:, 1])


@pytest.mark.parametrize("case", _golden()["cases"], ids=lambda c: c["name"])
def test_closed_form_single_epoch(case):
    g = _graph_from_case(case)
    Z = oracle.train(MODELS[case["model"]], g.row_ptr, g.col_idx, np.array(case["z0"]),
                     s=0, b=case["b"], seed=1, lr=case["lr"], epochs=1,
                     injected=case["samples"])
    np.testing.assert_allclose(Z, np.array(case["z1"]), rtol=1e-14, atol=1e-15)


@pytest.mark.parametrize("case", _golden()["losses"], ids=lambda c: c["name"])
def test_closed_form_losses(case):
    g = graphs.from_edges(2, [0], [1])
    Z = np.array([case["zu"], case["zv"]])
    m = MODELS[case["model"]]
    att = oracle.loss_vertex(m, g.row_ptr, g.col_idx, Z, 0, 0, 1, 0, injected=[[], []])
    empty = graphs.from_edges(2, [], [])
    rep = oracle.loss_vertex(m, empty.row_ptr, empty.col_idx, Z, 0, 0, 1, 0,
                             injected=[[1], []])
    assert att == pytest.approx(case["attractive"], rel=1e-14)
    assert rep == pytest.approx(case["repulsive"], rel=1e-14)


def test_sigmoid_gradient_vanishes_at_zero_embedding():
    g = graphs.erdos_renyi(40, p=0.2, seed=3)
    Z = np.zeros((40, 6))
    G = oracle.grad_minibatch(oracle.SIGMOID, g.row_ptr, g.col_idx, Z, 0, 40, 5, 9, 0)
    assert np.all(G == 0.0)
    # and the loss there is (deg + |S|) log 2 per vertex
    L = oracle.loss_vertex(oracle.SIGMOID, g.row_ptr, g.col_idx, Z, 3, 0, 9, 0,
                           injected=[[7, 8]] * 40)
    assert L == pytest.approx((g.degrees()[3] + 2) * math.log(2.0), rel=1e-14)


# --------------------------------------------------------------------------
# Finite differences of the objective (Eq. 2 with Eq. 3 / Eq. 7)
# --------------------------------------------------------------------------

def _random_case(n=14, d=5, seed=0, scale=0.6):
    rng = np.random.default_rng(seed)
    g = graphs.erdos_renyi(n, p=0.35, seed=seed + 1)
    Z = rng.normal(scale=scale, size=(n, d))
    nbr = [set(g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]].tolist()) for u in range(n)]
    samp = [[int(w) for w in rng.choice(n, size=4, replace=False) if w != u] for u in range(n)]
    return g, Z, nbr, samp


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_gradient_matches_finite_differences_of_loss(model):
    m = MODELS[model]
    g, Z, _, samp = _random_case(seed=11)
    n, d = Z.shape
    G = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, n, 0, 1, 0, injected=samp)
    h = 1e-5
    for u in range(n):
        fd = np.zeros(d)
        for j in range(d):
            Zp = Z.copy(); Zp[u, j] += h
            Zm = Z.copy(); Zm[u, j] -= h
            lp = oracle.loss_vertex(m, g.row_ptr, g.col_idx, Zp, u, 0, 1, 0, injected=samp)
            lm = oracle.loss_vertex(m, g.row_ptr, g.col_idx, Zm, u, 0, 1, 0, injected=samp)
            fd[j] = (lp - lm) / (2 * h)
        np.testing.assert_allclose(G[u], fd, rtol=1e-6, atol=1e-8)


def _bruteforce_eq1_loss(model, Z, u, nbr):
    """Eq. 1 written out directly: attractive over N(u), repulsive over every
    other vertex that is not a neighbour."""
    n = Z.shape[0]
    L = 0.0
    for w in range(n):
        if w == u:
            continue
        if model == "sigmoid":
            delta = 1.0 / (1.0 + math.exp(-float(Z[u] @ Z[w])))
        else:
            delta = 1.0 / (1.0 + float(((Z[u] - Z[w]) ** 2).sum()))
        L += -math.log(delta) if w in nbr[u] else -math.log(1.0 - delta)
    return L


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_all_pairs_negative_set_matches_bruteforce_eq1(model):
    m = MODELS[model]
    g, Z, nbr, _ = _random_case(n=10, d=4, seed=5)
    n, d = Z.shape
    comp = [[w for w in range(n) if w != u and w not in nbr[u]] for u in range(n)]
    G = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, n, 0, 1, 0, injected=comp)
    h = 1e-5
    for u in range(n):
        L0 = oracle.loss_vertex(m, g.row_ptr, g.col_idx, Z, u, 0, 1, 0, injected=comp)
        assert L0 == pytest.approx(_bruteforce_eq1_loss(model, Z, u, nbr), rel=1e-12)
        fd = np.zeros(d)
        for j in range(d):
            Zp = Z.copy(); Zp[u, j] += h
            Zm = Z.copy(); Zm[u, j] -= h
            fd[j] = (_bruteforce_eq1_loss(model, Zp, u, nbr)
                     - _bruteforce_eq1_loss(model, Zm, u, nbr)) / (2 * h)
        np.testing.assert_allclose(G[u], fd, rtol=1e-6, atol=1e-8)


# --------------------------------------------------------------------------
# Structure of Algorithm 2: which rows a gradient reads (Fig. "gradla")
# --------------------------------------------------------------------------

@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_gradient_reads_exactly_neighbours_and_samples(model):
    """The linear-algebra example of Sec. III-D: v0 has neighbours {v1, v3, v7}
    and negative samples {v2, v5}; its gradient depends on those rows and on
    z0 only."""
    m = MODELS[model]
    g = graphs.from_edges(8, [0, 0, 0, 4], [1, 3, 7, 6])
    samp = [[2, 5]] + [[] for _ in range(7)]
    rng = np.random.default_rng(2)
    Z = rng.normal(size=(8, 3))
    g0 = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, 1, 0, 1, 0, injected=samp)
    for w in range(1, 8):
        Zp = Z.copy(); Zp[w] += 0.25
        gp = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Zp, 0, 1, 0, 1, 0, injected=samp)
        changed = not np.array_equal(g0, gp)
        assert changed == (w in (1, 2, 3, 5, 7)), w


# --------------------------------------------------------------------------
# Invariants of the whole iteration
# --------------------------------------------------------------------------

@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_relabelling_permutes_the_result(model):
    m = MODELS[model]
    n, d = 30, 4
    g = graphs.erdos_renyi(n, p=0.2, seed=4)
    rng = np.random.default_rng(8)
    pi = rng.permutation(n)                       # new id of old vertex i
    samp = [[int(w) for w in rng.integers(0, n, 3)] for _ in range(n)]
    Z0 = oracle.init_embedding(n, d, 3)
    Z = oracle.train(m, g.row_ptr, g.col_idx, Z0, 0, n, 1, 0.05, 3, injected=samp)
    src = np.repeat(np.arange(n), g.degrees())
    gp = graphs.from_edges(n, pi[src], pi[g.col_idx])
    samp_p = [None] * n
    for i in range(n):
        samp_p[pi[i]] = [int(pi[w]) for w in samp[i]]
    Z0p = np.zeros_like(Z0); Z0p[pi] = Z0
    Zp = oracle.train(m, gp.row_ptr, gp.col_idx, Z0p, 0, n, 1, 0.05, 3, injected=samp_p)
    np.testing.assert_allclose(Zp[pi], Z, rtol=0, atol=1e-12)


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_rotation_commutes_with_training(model):
    m = MODELS[model]
    n, d = 60, 6
    g = graphs.erdos_renyi(n, p=0.1, seed=6)
    Q, _ = np.linalg.qr(np.random.default_rng(1).normal(size=(d, d)))
    Z0 = oracle.init_embedding(n, d, 2)
    Z = oracle.train(m, g.row_ptr, g.col_idx, Z0, 3, 16, 77, 0.05, 2)
    ZQ = oracle.train(m, g.row_ptr, g.col_idx, Z0 @ Q, 3, 16, 77, 0.05, 2)
    np.testing.assert_allclose(ZQ, Z @ Q, rtol=0, atol=1e-12)


def test_translation_commutes_with_training_t_model():
    n, d = 60, 5
    g = graphs.erdos_renyi(n, p=0.1, seed=7)
    c = np.array([0.3, -1.2, 2.0, 0.0, 0.7])
    Z0 = oracle.init_embedding(n, d, 4)
    Z = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z0, 3, 16, 5, 0.05, 2)
    Zc = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z0 + c, 3, 16, 5, 0.05, 2)
    np.testing.assert_allclose(Zc, Z + c, rtol=0, atol=1e-12)


def test_t_model_attractive_forces_balance():
    """With no negative samples and one minibatch, the t-model attractive
    forces are pairwise equal and opposite, so the gradients sum to zero."""
    n, d = 50, 3
    g = graphs.erdos_renyi(n, p=0.15, seed=9)
    Z0 = oracle.init_embedding(n, d, 6)
    G = oracle.grad_minibatch(oracle.TDIST, g.row_ptr, g.col_idx, Z0, 0, n, 0, 1, 0)
    assert np.abs(G.sum(axis=0)).max() < 1e-12
    assert np.abs(G).max() > 0.1


def test_minibatch_uses_snapshot_then_next_sees_update():
    """Within a minibatch every gradient uses the minibatch-start Z; the next
    minibatch uses the updated rows (Sec. III-B)."""
    n, d = 20, 3
    g = graphs.erdos_renyi(n, p=0.3, seed=10)
    Z0 = oracle.init_embedding(n, d, 1)
    b = 8
    Z = oracle.train(oracle.TDIST, g.row_ptr, g.col_idx, Z0, 2, b, 3, 0.1, 1)
    # redo by hand with the oracle's Algorithm 2
    W = Z0.copy()
    for u0 in range(0, n, b):
        u1 = min(u0 + b, n)
        G = oracle.grad_minibatch(oracle.TDIST, g.row_ptr, g.col_idx, W, u0, u1, 2, 3, 0)
        W[u0:u1] -= 0.1 * G
    np.testing.assert_array_equal(Z, W)


def test_learning_rate_schedule():
    assert oracle.learning_rate(0.02, 0, 20, 7) == 0.02
    assert oracle.learning_rate(0.02, 1, 20, 0) == 0.02
    assert oracle.learning_rate(0.02, 1, 20, 10) == pytest.approx(0.01, rel=1e-15)
    assert oracle.learning_rate(0.02, 1, 20, 19) == pytest.approx(0.001, rel=1e-13)


def test_thread_count_does_not_change_result():
    g = graphs.erdos_renyi(300, p=0.05, seed=12)
    Z0 = oracle.init_embedding(300, 16, 1)
    before = oracle.set_threads(0)
    try:
        oracle.set_threads(1)
        A = oracle.train(oracle.SIGMOID, g.row_ptr, g.col_idx, Z0, 5, 64, 1, 0.02, 2)
        oracle.set_threads(4)
        B = oracle.train(oracle.SIGMOID, g.row_ptr, g.col_idx, Z0, 5, 64, 1, 0.02, 2)
    finally:
        oracle.set_threads(before)
    np.testing.assert_array_equal(A, B)


@pytest.mark.parametrize("model", ["tdist", "sigmoid"])
def test_loss_decreases_over_first_epochs(model):
    g = graphs.er1000_graph()
    m = MODELS[model]
    Z = oracle.init_embedding(g.n, 32, 1)
    # loss over a fixed sample set so that the comparisons are like for like
    samp = [list(r) for r in oracle.samples(g.n, 5, 0, 1)]
    losses = [oracle.loss_total(m, g.row_ptr, g.col_idx, Z, 0, 1, 0, injected=samp)]
    for e in range(5):
        Z = oracle.train(m, g.row_ptr, g.col_idx, Z, 5, 256, 1, 0.02, 1, start_epoch=e)
        losses.append(oracle.loss_total(m, g.row_ptr, g.col_idx, Z, 0, 1, 0, injected=samp))
    assert all(b < a for a, b in zip(losses, losses[1:])), losses


# --------------------------------------------------------------------------
# AUC (Mann-Whitney with ties counted one half)
# --------------------------------------------------------------------------

def test_auc_matches_pair_counting():
    rng = np.random.default_rng(0)
    for _ in range(5):
        pos = rng.integers(0, 20, size=37).astype(float)
        neg = rng.integers(0, 20, size=53).astype(float)
        want = sum((p > q) + 0.5 * (p == q) for p in pos for q in neg) / (pos.size * neg.size)
        assert oracle.auc(pos, neg) == pytest.approx(want, abs=1e-15)
    assert oracle.auc([1.0, 2.0], [0.0, 0.5]) == 1.0
    assert oracle.auc([0.0], [1.0]) == 0.0


def test_auc_matches_sklearn():
    metrics = pytest.importorskip("sklearn.metrics")
    rng = np.random.default_rng(1)
    pos = rng.normal(0.5, 1.0, 400)
    neg = rng.normal(0.0, 1.0, 500)
    y = np.r_[np.ones(400), np.zeros(500)]
    want = metrics.roc_auc_score(y, np.r_[pos, neg])
    assert oracle.auc(pos, neg) == pytest.approx(want, abs=1e-12)


def test_philox_self_samples_are_skipped():
    """With Philox draws, a sample that lands on u itself adds nothing: the
    gradient equals the one with that draw removed from an injected S(u)."""
    n, s, seed = 7, 6, 3
    g = graphs.erdos_renyi(n, p=0.4, seed=2)
    S = oracle.samples(n, s, 0, seed)
    assert any(u in S[u] for u in range(n))           # the case occurs here
    Z = oracle.init_embedding(n, 3, 1)
    for m in (oracle.TDIST, oracle.SIGMOID):
        G = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, n, s, seed, 0)
        inj = [[int(w) for w in S[u] if w != u] for u in range(n)]
        Gi = oracle.grad_minibatch(m, g.row_ptr, g.col_idx, Z, 0, n, 0, seed, 0, injected=inj)
        np.testing.assert_array_equal(G, Gi)


def test_sigmoid_coordinates_are_bounded_t_model_is_not():
    """Sigmoid model: each coordinate of an updated row is clamped to [-4, 4]
    (worked by hand: one edge, s = 0, b = 2, eta = 10, d = 1, z = (3.9, 0.1);
    grad_u = (sigma(0.39) - 1) * 0.1, grad_v = (sigma(0.39) - 1) * 3.9, both
    negative, so both rows move up past 4 and stop there).  The t model is not
    bounded: z_v = 0.1 + 10 * 2 * 3.8 / (1 + 3.8^2) = 5.0223..."""
    rp = np.array([0, 1, 2], np.int32)
    ci = np.array([1, 0], np.int32)
    Z0 = np.array([[3.9], [0.1]])
    zs = oracle.train(1, rp, ci, Z0, 0, 2, 1, 10.0, 1)
    assert zs[0, 0] == 4.0 and zs[1, 0] == 4.0
    zt = oracle.train(0, rp, ci, Z0, 0, 2, 1, 10.0, 1)
    step = 10.0 * 2.0 * 3.8 / (1.0 + 3.8 ** 2)
    assert abs(zt[0, 0] - (3.9 - step)) < 1e-12
    assert abs(zt[1, 0] - (0.1 + step)) < 1e-12 and zt[1, 0] > 4.0
    # below the bound the update is the plain Eq. 10 step
    zs2 = oracle.train(1, rp, ci, np.array([[0.3], [-0.2]]), 0, 2, 1, 0.5, 1)
    g_u = (1.0 / (1.0 + math.exp(0.06)) - 1.0) * -0.2
    assert abs(zs2[0, 0] - (0.3 - 0.5 * g_u)) < 1e-12


def test_sigmoid_loss_stays_finite_at_the_coordinate_bound():
    """Eq. 3's terms at dot products far beyond FP64's exp range: with every
    coordinate at the bound 4 and d = 128, z_u . z_w = 2048, so the repulsive
    term -log(1 - sigma(2048)) = log(1 + e^2048) equals 2048 to FP64
    precision and the attractive -log sigma(2048) = log(1 + e^-2048) is 0
    (e^-2048 underflows); at -2048 the roles swap."""
    d = 128
    Z = np.full((2, d), 4.0)
    edge = graphs.from_edges(2, [0], [1])
    none = graphs.from_edges(2, [], [])
    rep = oracle.loss_vertex(oracle.SIGMOID, none.row_ptr, none.col_idx, Z, 0, 0, 1, 0,
                             injected=[[1], []])
    att = oracle.loss_vertex(oracle.SIGMOID, edge.row_ptr, edge.col_idx, Z, 0, 0, 1, 0)
    assert rep == 2048.0 and att == 0.0
    Z[1] = -4.0
    rep = oracle.loss_vertex(oracle.SIGMOID, none.row_ptr, none.col_idx, Z, 0, 0, 1, 0,
                             injected=[[1], []])
    att = oracle.loss_vertex(oracle.SIGMOID, edge.row_ptr, edge.col_idx, Z, 0, 0, 1, 0)
    assert rep == 0.0 and att == 2048.0
