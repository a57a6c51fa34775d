"""f2v_minibatch_noalloc: the minibatch step for callers that cannot allocate.

Some callers own all device memory through their own allocator or arena, or
plan it for a whole run, and must not have a library call cudaMalloc while
the step runs.  f2v_minibatch_noalloc serves them: it takes the graph and
both embedding buffers as device pointers and keeps its scratch in a fixed
array inside the library.  These tests call it through the C ABI, twice in a
row (two consecutive minibatches), and check each result two ways: against
the same minibatches run through a context (f2v_create /
f2v_run_minibatches), element by element with the tolerance the parity
tests use, and against the FP64 oracle's Algorithm 2 + Eq. 10 computed from
the same Z, with the per-minibatch bound of the parity tests.  The row sizes
cover every kernel shape the call can pick (one lane per row at d = 2, lane
groups at d = 32, the masked shape at d = 48, whole warps at d = 128 and
two vectors per lane at d = 256), and epoch 1 checks the epoch part of the
sample counters.

The file is named so that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import f2v, graphs

pytestmark = pytest.mark.gpu

TOL = 1e-5
FLOOR = 1e-3


def _rel(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float((np.abs(a - b) / np.maximum(np.abs(b), FLOOR)).max())


@pytest.fixture(scope="module")
def torch_cuda():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    return torch


@pytest.mark.parametrize("epoch", [0, 1])
@pytest.mark.parametrize("d", [2, 32, 48, 128, 256])
@pytest.mark.parametrize("model", [f2v.TDIST, f2v.SIGMOID], ids=["tdist", "sigmoid"])
def test_noalloc_minibatch_matches_context_and_oracle(torch_cuda, model, d, epoch):
    torch = torch_cuda
    lib = f2v.load_library()
    g = graphs.er1000_graph()                 # n=1000, ~10,000 edges
    s, b, lr, seed = 5, 256, 0.02, 1

    # the existing entry points: a context, one minibatch at a time, after
    # `epoch` whole epochs
    with f2v.Context(g.row_ptr, g.col_idx, g.n, d, model=model, s=s, lr=lr, minibatch=b,
                     seed=seed) as ctx:
        ctx.train(epoch)
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
            ctypes.c_float(lr), seed, epoch, u0, u1, ctypes.c_void_p(zcur.data_ptr()),
            ctypes.c_void_p(znext.data_ptr()), ctypes.c_void_p(stream.cuda_stream))
        assert rc == f2v.OK, lib.f2v_noalloc_last_error().decode()
        torch.cuda.synchronize()
        # Z after minibatch k: updated rows from z_next, the rest from z_cur
        cur = zcur.cpu().numpy().copy()
        cur[:u1] = znext[:u1].cpu().numpy()
        return cur

    def oracle_check(before, after, k):
        u0, u1 = k * b, min(g.n, (k + 1) * b)
        before = before.astype(np.float64)
        G, A = oracle.grad_minibatch_abs(model, g.row_ptr, g.col_idx, before, u0, u1, s, seed,
                                         epoch)
        want = before[u0:u1] - np.float64(np.float32(lr)) * G
        if model != f2v.TDIST:
            want = np.clip(want, -4.0, 4.0)
        scale = np.maximum(np.abs(before[u0:u1]) + lr * A, FLOOR)
        err = np.abs(after[u0:u1].astype(np.float64) - want) / scale
        assert err.max() <= TOL, (k, float(err.max()))

    got1 = step(0)
    assert _rel(got1, want1) <= TOL
    oracle_check(z0, got1, 0)
    got2 = step(1)
    assert _rel(got2, want2) <= TOL
    oracle_check(got1, got2, 1)
    assert np.array_equal(got2[2 * b:], z0[2 * b:])


def test_noalloc_rejects_oversized_minibatch(torch_cuda):
    torch = torch_cuda
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
