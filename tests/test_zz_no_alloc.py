"""f2v_minibatch_noalloc: the minibatch step for callers that cannot allocate.

Some callers own all device memory through their own allocator or arena, or
plan it for a whole run, and must not have a library call cudaMalloc while
the step runs.  f2v_minibatch_noalloc serves them: it takes the graph and
both embedding buffers as device pointers and keeps its scratch in a fixed
array inside the library.  This test calls it through the C ABI, twice in a
row (two consecutive minibatches), and checks each result against the same
minibatches run through a context (f2v_create / f2v_run_minibatches), with
the element-wise tolerance the parity tests use.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

from paper_2009_10035_gb300 import f2v, graphs

pytestmark = pytest.mark.gpu

TOL = 1e-5
FLOOR = 1e-3


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float((np.abs(a - b) / np.maximum(np.abs(b), FLOOR)).max())


@pytest.mark.parametrize("model", [f2v.TDIST, f2v.SIGMOID], ids=["tdist", "sigmoid"])
def test_noalloc_minibatch_matches_context(model):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lib = f2v.load_library()
    g = graphs.er1000_graph()                 # n=1000, ~10,000 edges
    d, s, b, lr, seed = 32, 5, 256, 0.02, 1

    # the existing entry points: a context, one minibatch at a time
    with f2v.Context(g.row_ptr, g.col_idx, g.n, d, model=model, s=s, lr=lr, minibatch=b,
                     seed=seed) as ctx:
        z0 = ctx.embedding()
        ctx.run_minibatches(1)
        want1 = ctx.embedding()
        ctx.run_minibatches(1)
        want2 = ctx.embedding()

    # the same two minibatches on caller-owned device buffers
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(g.col_idx.astype(np.int32)).to(dev)
    zcur = torch.from_numpy(z0).to(dev)
    znext = torch.zeros_like(zcur)
    stream = torch.cuda.current_stream()

    def step(k):
        u0, u1 = k * b, min(g.n, (k + 1) * b)
        rc = lib.f2v_minibatch_noalloc(
            ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()), g.n, d, model, s,
            ctypes.c_float(lr), seed, 0, u0, u1, ctypes.c_void_p(zcur.data_ptr()),
            ctypes.c_void_p(znext.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == f2v.OK, lib.f2v_noalloc_last_error().decode()
        torch.cuda.synchronize()
        # Z after minibatch k: updated rows from z_next, the rest from z_cur
        cur = zcur.cpu().numpy().copy()
        cur[:u1] = znext[:u1].cpu().numpy()
        return cur

    got1 = step(0)
    assert _rel(got1, want1) <= TOL
    got2 = step(1)
    assert _rel(got2, want2) <= TOL
    assert np.array_equal(got2[2 * b:], z0[2 * b:])


def test_noalloc_rejects_oversized_minibatch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    lib = f2v.load_library()
    # a star whose hub alone has 200,000 neighbours: at d = 256 its partial
    # sums need far more than the fixed scratch holds
    g = graphs.star(200_000)
    dev = torch.device("cuda", 0)
    rp = torch.from_numpy(g.row_ptr.astype(np.int32)).to(dev)
    ci = torch.from_numpy(g.col_idx.astype(np.int32)).to(dev)
    z = torch.zeros((g.n, 256), dtype=torch.float32, device=dev)
    zn = torch.zeros_like(z)
    rc = lib.f2v_minibatch_noalloc(
        ctypes.c_void_p(rp.data_ptr()), ctypes.c_void_p(ci.data_ptr()), g.n, 256, f2v.TDIST, 5,
        ctypes.c_float(0.02), 1, 0, 0, 1, ctypes.c_void_p(z.data_ptr()),
        ctypes.c_void_p(zn.data_ptr()), None)
    assert rc == f2v.EINVAL
    assert "scratch" in lib.f2v_noalloc_last_error().decode()
    torch.cuda.synchronize()
    assert not bool(zn.any())
