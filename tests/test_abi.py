"""CPU checks of the C ABI: the library builds, loads and exports every
function include/f2v.h declares, and host-side validation rejects bad input
before any device work."""
import ctypes

import numpy as np
import pytest

from paper_2009_10035_gb300 import build, f2v, graphs


@pytest.fixture(scope="module")
def lib():
    build.build()
    return f2v.load_library()


def test_header_declares_the_boundary():
    names = f2v.header_functions()
    for core in ("f2v_create", "f2v_epoch", "f2v_get_embedding", "f2v_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in f2v.header_functions():
        assert hasattr(lib, name), name


def _create(lib, rp, ci, n, d=8, s=5, lr=0.02, b=4, model=0):
    rp = np.ascontiguousarray(rp, np.int32)
    ci = np.ascontiguousarray(ci if len(ci) else [0], np.int32)
    h = ctypes.c_void_p()
    rc = lib.f2v_create(rp.ctypes.data_as(ctypes.c_void_p), ci.ctypes.data_as(ctypes.c_void_p),
                        n, d, model, s, lr, b, 1, ctypes.byref(h))
    return rc, h, lib.f2v_last_error_global().decode()


@pytest.mark.parametrize("case,needle", [
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, d=0), "d ="),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, d=2000), "d ="),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, s=-1), "s ="),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, s=70000), "s ="),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, b=0), "minibatch"),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, lr=0.0), "lr"),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, lr=float("nan")), "lr"),
    (dict(rp=[0, 1, 2], ci=[1, 0], n=2, model=7), "model"),
    (dict(rp=[0], ci=[], n=0), "n ="),
    (dict(rp=[1, 1, 2], ci=[1, 0], n=2), "row_ptr[0]"),
    (dict(rp=[0, 2, 1], ci=[1, 0], n=2), "monotone"),
    (dict(rp=[0, 1, 2], ci=[1, 5], n=2), "out of range"),
    (dict(rp=[0, 1, 2], ci=[0, 0], n=2), "self-loop"),
    (dict(rp=[0, 2, 4, 4], ci=[1, 1, 0, 0], n=3), "duplicate"),
])
def test_create_rejects_invalid_input(lib, case, needle):
    rc, h, msg = _create(lib, **case)
    assert rc == f2v.EINVAL
    assert not h.value
    assert needle in msg


def test_null_context_calls_fail_cleanly(lib):
    assert lib.f2v_epoch(None) == f2v.EINVAL
    assert lib.f2v_train(None, 1) == f2v.EINVAL
    lib.f2v_destroy(None)


def test_python_binding_refuses_missing_library(tmp_path):
    with pytest.raises(RuntimeError):
        f2v.load_library(str(tmp_path / "missing.so"))


def test_graph_generators_give_valid_symmetric_csr():
    for g in (graphs.er1000_graph(), graphs.rmat(10, 8, seed=3), graphs.sbm(500, 4, 0.05, 0.002),
              graphs.star(50)):
        n = g.n
        deg = g.degrees()
        src = np.repeat(np.arange(n), deg)
        assert (g.col_idx >= 0).all() and (g.col_idx < n).all()
        assert (src != g.col_idx).all()
        keys = src.astype(np.int64) * n + g.col_idx
        assert np.unique(keys).size == keys.size
        rkeys = g.col_idx.astype(np.int64) * n + src
        assert np.array_equal(np.sort(keys), np.sort(rkeys))
        for u in range(0, n, max(1, n // 50)):
            row = g.col_idx[g.row_ptr[u]:g.row_ptr[u + 1]]
            assert (np.diff(row) > 0).all()


def test_er1000_graph_shape():
    g = graphs.er1000_graph()
    assert g.n == 1000
    assert 9000 < g.nnz // 2 < 11000


def test_holdout_split_is_disjoint_and_balanced():
    g0 = graphs.erdos_renyi(500, m=3000, seed=1)
    g = graphs.holdout(g0, 0.05, seed=2)
    full = set(graphs.undirected_keys(g0).tolist())
    train = set(graphs.undirected_keys(g).tolist())
    pos = {int(a) * g.n + int(b) for a, b in g.test_pos}
    neg = {int(a) * g.n + int(b) for a, b in g.test_neg}
    assert len(pos) == round(0.05 * len(full)) == len(neg)
    assert pos.isdisjoint(train) and pos | train == full
    assert neg.isdisjoint(full)
    assert all(a < b for a, b in g.test_neg)


def test_output_buffers_are_checked_before_the_call():
    ok = np.zeros(12, np.float32)
    assert f2v._host_out(ok, 12) is ok
    assert f2v._host_out(np.zeros(20, np.float32), 12, exact=False) is not None
    ro = np.zeros(12, np.float32)
    ro.flags.writeable = False
    bad = [np.zeros(12, np.float64), np.zeros((4, 6), np.float32)[:, :3], ro,
           np.zeros(11, np.float32), [0.0] * 12]
    for out in bad:
        with pytest.raises(ValueError):
            f2v._host_out(out, 12)
    with pytest.raises(ValueError):
        f2v._host_out(np.zeros(11, np.float32), 12, exact=False)


@pytest.mark.parametrize("d,zoff,csr_off,ok", [
    (128, 8, 0, False),      # 16-byte vectors: an 8-byte offset is refused
    (128, 4, 0, False),
    (2, 4, 0, False),        # 8-byte vectors at d = 2
    (128, 0, 2, False),      # CSR words must be 4-byte aligned
    (2, 8, 0, True),         # 8 bytes is enough at d = 2 (passes the check)
    (48, 4, 0, True),        # scalar shape: 4 bytes is enough (passes the check)
])
def test_noalloc_rejects_misaligned_buffers_before_device_work(lib, d, zoff, csr_off, ok):
    """f2v_minibatch_noalloc takes Z and the CSR from the caller's allocator;
    a pointer that the kernel's vector accesses cannot use is refused on the
    host.  The pointers here are never dereferenced: the call must return
    before any device work (a call that passes the alignment check then
    fails later with another message, since mb_begin >= mb_end)."""
    base = 1 << 20
    rc = lib.f2v_minibatch_noalloc(
        ctypes.c_void_p(base + csr_off), ctypes.c_void_p(base + 4096 + csr_off), 10, d, 0, 5,
        ctypes.c_float(0.02), 1, 0, 3, 3 if ok else 4,
        ctypes.c_void_p(base + 8192 + zoff), ctypes.c_void_p(base + 65536 + zoff), None)
    assert rc == f2v.EINVAL
    msg = lib.f2v_noalloc_last_error().decode()
    if ok:
        assert "aligned" not in msg and "mb_begin" in msg
    else:
        assert "aligned" in msg


def test_library_rebuild_depends_on_every_header():
    """An edit to any public header makes the library out of date."""
    import os
    deps = set(build._deps())
    for h in os.listdir(build.INCLUDE):
        if h.endswith(".h"):
            assert os.path.join(build.INCLUDE, h) in deps, h
