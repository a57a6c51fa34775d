"""CPU checks of the batched form's host side: the SBM batch generator's
output, and argument validation of f2v_batch_create before any device work."""
import ctypes

import numpy as np
import pytest

from paper_2009_10035_gb300 import build, f2v, graphs


def _check_csr(g):
    rp, ci = g.row_ptr, g.col_idx
    assert rp[0] == 0 and rp[-1] == ci.size and np.all(np.diff(rp) >= 0)
    u = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    assert np.all((ci >= 0) & (ci < g.n)) and np.all(u != ci)
    keys = u * g.n + ci
    assert np.all(np.diff(keys) > 0)                      # rows sorted, no duplicates
    assert np.array_equal(np.sort(ci.astype(np.int64) * g.n + u), keys)   # symmetric


def test_sbm_batch_is_valid_and_deterministic():
    a = graphs.sbm_batch(40, seed=4, n_range=(50, 3000))
    b = graphs.sbm_batch(40, seed=4, n_range=(50, 3000))
    assert np.array_equal(a.row_ptr, b.row_ptr) and np.array_equal(a.col_idx, b.col_idx)
    assert np.array_equal(a.seed, b.seed) and np.array_equal(a.d, b.d)
    assert a.row_ptr.size == int(a.n.sum()) + a.num_graphs
    for i in range(a.num_graphs):
        _check_csr(a.graph(i))
    assert set(a.d.tolist()) == {2, 16, 64}
    assert a.n.min() >= 50 and a.n.max() <= 3000
    assert a.blocks.min() >= 2 and a.blocks.max() <= 16
    c = graphs.sbm_batch(40, seed=5, n_range=(50, 3000))
    assert not np.array_equal(a.n, c.n)


def test_sbm_edge_densities_match_p_in_and_p_out():
    n, B, p_in, p_out = 4000, 4, 0.05, 0.002
    rp, ci, roff, coff = graphs.sbm_graphs([n], [B], p_in, p_out, seed=9)
    g = graphs.Graph(n, rp, ci)
    _check_csr(g)
    bounds = (np.arange(B + 1, dtype=np.int64) * n) // B
    blk = np.searchsorted(bounds, np.arange(n), side="right") - 1
    u = np.repeat(np.arange(n), np.diff(rp))
    same = blk[u] == blk[ci]
    sizes = np.diff(bounds)
    pin_pairs = int((sizes * (sizes - 1)).sum())
    pout_pairs = n * (n - 1) - pin_pairs
    # binomial standard errors: 5 sigma
    est_in = same.sum() / pin_pairs
    est_out = (~same).sum() / pout_pairs
    assert abs(est_in - p_in) < 5 * np.sqrt(p_in * (1 - p_in) / (pin_pairs / 2))
    assert abs(est_out - p_out) < 5 * np.sqrt(p_out * (1 - p_out) / (pout_pairs / 2))


def test_sbm_extremes():
    rp, ci, _, _ = graphs.sbm_graphs([5, 6], [1, 3], 1.0, 0.0, seed=1)
    g0 = graphs.Graph(5, rp[:6], ci[:20])
    _check_csr(g0)
    assert g0.nnz == 20                                  # complete graph K5
    g1 = graphs.Graph(6, rp[6:], ci[20:])
    _check_csr(g1)
    assert g1.nnz == 6                                   # three disjoint edges


@pytest.fixture(scope="module")
def lib():
    build.build()
    return f2v.load_library()


@pytest.mark.parametrize("case,needle", [
    (dict(G=0), "num_graphs"),
    (dict(d=[3]), "d = 3"),
    (dict(d=[256]), "d = 256"),
    (dict(n=[0]), "n = 0"),
    (dict(s=-1), "s = -1"),
    (dict(b=0), "minibatch"),
    (dict(lr=0.0), "lr"),
])
def test_batch_create_rejects_invalid_arguments(lib, case, needle):
    G = case.get("G", 1)
    n = np.asarray(case.get("n", [2]), np.int32)
    d = np.asarray(case.get("d", [16]), np.int32)
    seed = np.ones(1, np.uint64)
    rp = np.asarray([0, 1, 2], np.int32)
    ci = np.asarray([1, 0], np.int32)
    h = ctypes.c_void_p()
    vp = lambda a: a.ctypes.data_as(ctypes.c_void_p)
    rc = lib.f2v_batch_create(G, vp(n), vp(d), vp(seed), vp(rp), vp(ci), 0, case.get("s", 5),
                              case.get("lr", 0.02), case.get("b", 128), 0, None,
                              ctypes.byref(h))
    assert rc == f2v.EINVAL
    assert not h.value
    assert needle in lib.f2v_last_error_global().decode()


def test_batch_null_handle_calls_fail_cleanly(lib):
    assert lib.f2v_batch_epoch(None) == f2v.EINVAL
    assert lib.f2v_batch_synchronize(None) == f2v.EINVAL
    lib.f2v_batch_destroy(None)
