"""Parity of the batched form (include/f2v_batch.h) with the FP64 oracle.

Every graph of a batch must compute what the oracle computes for that graph
alone (Algorithm 1 per graph, its own seed).  As for the single-graph form,
the runs are compared minibatch by minibatch: the batch advances one
minibatch position at a time and the oracle computes each graph's update
(Algorithm 2 + Eq. 10) from the batch's own Z before it; the error of FP32
accumulation of z_u - eta * sum(terms) is bounded relative to |z_u| + eta *
sum|terms| (the oracle's absolute-value sum), so it is measured against that
scale, floor 1e-3, bound 1e-5.  Rows outside the minibatch must not move.
A whole-epoch element-wise check (1e-5 relative, floor 1e-3) is kept for
well-conditioned cases.
"""
import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import f2v, graphs

pytestmark = pytest.mark.gpu

TOL = 1e-5
FLOOR = 1e-3
MODELS = [pytest.param(f2v.TDIST, id="tdist"), pytest.param(f2v.SIGMOID, id="sigmoid")]


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    f2v.load_library()


def rel_err(got, want):
    return np.abs(np.asarray(got, np.float64) - want) / np.maximum(np.abs(want), FLOOR)


def concat(graph_list, dims, seeds):
    """Concatenated layout of f2v_batch_create from a list of graphs.Graph."""
    n = np.array([g.n for g in graph_list], np.int32)
    rp = np.concatenate([g.row_ptr for g in graph_list]).astype(np.int32)
    ci = np.concatenate([g.col_idx for g in graph_list] + [np.zeros(0, np.int32)]).astype(np.int32)
    return n, np.asarray(dims, np.int32), np.asarray(seeds, np.uint64), rp, ci


def oracle_epochs(g, d, model, s, b, lr, seed, epochs, start_epoch=0, z0=None,
                  schedule=0, total_epochs=0):
    Z0 = oracle.init_embedding(g.n, d, seed) if z0 is None else np.asarray(z0, np.float64)
    return oracle.train(model, g.row_ptr, g.col_idx, Z0, s, b, seed, lr, epochs,
                        start_epoch=start_epoch, schedule=schedule, total_epochs=total_epochs)


def check_batch_one_epoch(glist, dims, model, s=5, b=128, lr=0.02, tilings=()):
    """Whole epoch against the oracle, element by element (well-conditioned
    cases)."""
    seeds = [1000 + 17 * i for i in range(len(glist))]
    n, d, sd, rp, ci = concat(glist, dims, seeds)
    worst = 0.0
    with f2v.Batch(n, d, sd, rp, ci, model=model, s=s, lr=lr, minibatch=b) as bt:
        for t in tilings:
            bt.set_tiling(*t)
        bt.epoch()
        bt.synchronize()
        for i, g in enumerate(glist):
            got = bt.embedding(i)
            want = oracle_epochs(g, int(d[i]), model, s, b, lr, seeds[i], 1)
            assert np.isfinite(got).all()
            err = rel_err(got, want)
            assert err.max() <= TOL, (f"graph {i} (n={g.n}, d={d[i]}): max rel err "
                                      f"{err.max():.3e} at {np.unravel_index(err.argmax(), err.shape)}")
            worst = max(worst, float(err.max()))
    return worst


def bf16_round(x):
    """FP32 -> BF16 (round to nearest even) -> FP64, for finite x."""
    u = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def check_step(bt, glist, dims, seeds, model, s, b, lr, e, k, before, which,
               schedule=0, total_epochs=0, bf16=False):
    """Minibatch position k of epoch e has just run on `bt`; `before` holds
    each checked graph's Z before it (the FP32 master in the BF16 form, whose
    partner rows are read as stored: rounded to BF16)."""
    worst = 0.0
    eta = oracle.learning_rate(lr, schedule, total_epochs, e)
    for i in which:
        g = glist[i]
        after = bt.embedding(int(i)).astype(np.float64)
        M = -(-g.n // b)
        if k >= M:
            assert np.array_equal(after, before[i]), f"graph {i} moved at position {k} >= M"
            continue
        u0, u1 = k * b, min(g.n, (k + 1) * b)
        G, A = oracle.grad_minibatch_abs(model, g.row_ptr, g.col_idx, before[i], u0, u1, s,
                                         int(seeds[i]), e,
                                         gather=bf16_round(before[i]) if bf16 else None)
        want = before[i][u0:u1] - eta * G
        if model == f2v.SIGMOID:
            want = np.clip(want, -4.0, 4.0)
        scale = np.maximum(np.abs(before[i][u0:u1]) + eta * A, FLOOR)
        err = np.abs(after[u0:u1] - want) / scale
        assert np.isfinite(after).all()
        assert err.max() <= TOL, (f"epoch {e} position {k} graph {i} (n={g.n}, d={dims[i]}): "
                                  f"scaled err {err.max():.3e}")
        assert np.array_equal(after[:u0], before[i][:u0])
        assert np.array_equal(after[u1:], before[i][u1:])
        worst = max(worst, float(err.max()))
    return worst


def check_batch_steps(glist, dims, model, s=5, b=128, lr=0.02, epochs=1, tilings=(),
                      schedule=None, total_epochs=0):
    """Every minibatch position of every epoch, every graph, against the oracle."""
    seeds = [1000 + 17 * i for i in range(len(glist))]
    n, d, sd, rp, ci = concat(glist, dims, seeds)
    M = max(-(-g.n // b) for g in glist)
    worst = 0.0
    with f2v.Batch(n, d, sd, rp, ci, model=model, s=s, lr=lr, minibatch=b) as bt:
        for t in tilings:
            bt.set_tiling(*t)
        if schedule is not None:
            bt.set_schedule(schedule, total_epochs)
        which = range(len(glist))
        for e in range(epochs):
            for k in range(M):
                assert bt.progress == (e, k)
                before = [bt.embedding(i).astype(np.float64) for i in which]
                bt.run_minibatches(1)
                worst = max(worst, check_step(bt, glist, d, seeds, model, s, b, lr, e, k, before,
                                              which, 0 if schedule is None else schedule,
                                              total_epochs))
        assert bt.progress == (epochs, 0)
    return worst


def small_sbm_batch(count, seed, n_range=(50, 1500), dims=(2, 16, 64)):
    return graphs.sbm_batch(count, seed=seed, n_range=n_range, dims=dims)


@pytest.mark.parametrize("model", MODELS)
def test_mixed_sbm_batch_steps(model):
    gb = small_sbm_batch(12, seed=5)
    glist = [gb.graph(i) for i in range(gb.num_graphs)]
    check_batch_steps(glist, gb.d, model)


@pytest.mark.parametrize("model", MODELS)
def test_whole_epoch_well_conditioned(model):
    # d >= 32 and modest degrees: one FP32 epoch stays within 1e-5 of FP64
    glist = [graphs.erdos_renyi(1000, m=10000, seed=1), graphs.sbm(1500, 4, 0.02, 0.002, seed=2),
             graphs.erdos_renyi(400, m=1500, seed=3)]
    check_batch_one_epoch(glist, [32, 64, 128], model)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("d,L", [(2, 1), (4, 1), (4, 2), (8, 2), (8, 4), (16, 4), (16, 8),
                                 (32, 8), (32, 16), (64, 16), (64, 32), (128, 32)])
def test_every_shape(model, d, L):
    glist = [graphs.sbm(300, 3, 0.05, 0.01, seed=2), graphs.erdos_renyi(700, m=3000, seed=3)]
    check_batch_steps(glist, [d, d], model, tilings=[(d, L, 64)])


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("C", [32, 64, 1024])
def test_item_sizes_and_split_hubs(model, C):
    # a star with 3000 leaves spans ~100 items of 32 pairs: a two-level combine tree
    glist = [graphs.star(3000), graphs.sbm(900, 4, 0.05, 0.004, seed=4)]
    check_batch_steps(glist, [16, 64], model, b=1024, tilings=[(16, 4, C), (64, 16, C)])


@pytest.mark.parametrize("model", MODELS)
def test_edge_cases(model):
    # one vertex; an edgeless graph; n < b; isolated vertices; s = 0 below
    glist = [graphs.from_edges(1, np.zeros(0, np.int64), np.zeros(0, np.int64)),
             graphs.from_edges(40, np.zeros(0, np.int64), np.zeros(0, np.int64)),
             graphs.erdos_renyi(90, m=200, seed=6),
             graphs.from_edges(300, np.arange(0, 100, 2), np.arange(1, 101, 2))]
    check_batch_steps(glist, [2, 16, 32, 8], model)
    check_batch_steps(glist, [2, 16, 32, 8], model, s=0)


def test_many_minibatches_per_graph():
    # 8000 vertices at b = 64: a chain of 125 minibatch barriers in one launch
    glist = [graphs.sbm(8000, 8, 0.02, 0.001, seed=8), graphs.sbm(120, 2, 0.1, 0.01, seed=9)]
    seeds = [5, 6]
    n, d, sd, rp, ci = concat(glist, [16, 2], seeds)
    with f2v.Batch(n, d, sd, rp, ci, model=f2v.TDIST, s=5, lr=0.02, minibatch=64) as bt:
        # positions 0..99 in one launch, then the last 25 one at a time
        bt.run_minibatches(100)
        for k in range(100, 125):
            before = [bt.embedding(i).astype(np.float64) for i in range(2)]
            bt.run_minibatches(1)
            check_step(bt, glist, d, seeds, f2v.TDIST, 5, 64, 0.02, 0, k, before, [0, 1])
        assert bt.progress == (1, 0)


@pytest.mark.parametrize("model", MODELS)
def test_steps_across_epochs_with_linear_schedule(model):
    gb = small_sbm_batch(6, seed=11, n_range=(60, 900))
    glist = [gb.graph(i) for i in range(gb.num_graphs)]
    check_batch_steps(glist, gb.d, model, epochs=3, schedule=f2v.LR_LINEAR, total_epochs=5)


def test_epoch_after_partial_steps_equals_whole_epoch():
    gb = small_sbm_batch(7, seed=12, n_range=(60, 2000))
    with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=5, lr=0.02, minibatch=128) as a:
        a.train(2)
        whole = [a.embedding(i) for i in range(gb.num_graphs)]
    with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=5, lr=0.02, minibatch=128) as b:
        b.run_minibatches(3)
        b.run_minibatches(2)
        b.epoch()           # finishes the begun epoch
        assert b.progress == (1, 0)
        b.epoch()
        for i in range(gb.num_graphs):
            assert np.array_equal(b.embedding(i), whole[i])


def test_bit_reproducible_and_concatenated_readout():
    gb = small_sbm_batch(9, seed=13)
    outs = []
    for _ in range(2):
        with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=5, lr=0.02, minibatch=128) as bt:
            bt.train(3)
            allz = np.empty(int(bt.z_off[-1]), np.float32)
            bt.embeddings_into_host(allz)
            for i in range(gb.num_graphs):
                zi = bt.embedding(i).ravel()
                assert np.array_equal(zi, allz[bt.z_off[i]:bt.z_off[i + 1]])
            outs.append(allz)
    assert np.array_equal(outs[0], outs[1])


def test_set_embedding_resumes_bit_identically():
    gb = small_sbm_batch(5, seed=17)
    with f2v.Batch.from_graphs(gb, model=f2v.SIGMOID, s=5, lr=0.02, minibatch=128) as a:
        a.train(2)
        mid = [a.embedding(i) for i in range(gb.num_graphs)]
        a.train(1)
        end = [a.embedding(i) for i in range(gb.num_graphs)]
    with f2v.Batch.from_graphs(gb, model=f2v.SIGMOID, s=5, lr=0.02, minibatch=128) as b:
        b.train(2)      # the epoch counter advances with training
        for i in range(gb.num_graphs):
            b.set_embedding(i, mid[i] * 0 + mid[i])
        b.train(1)
        for i in range(gb.num_graphs):
            assert np.array_equal(b.embedding(i), end[i])


def test_autotune_restores_state_and_applies_tiling(tmp_path):
    gb = small_sbm_batch(10, seed=19)
    cache = str(tmp_path / "tune.json")
    with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=5, lr=0.02, minibatch=128) as bt:
        bt.train(1)
        z1 = [bt.embedding(i) for i in range(gb.num_graphs)]
        chosen = bt.autotune(1, cache=cache, key="k")
        assert sorted({t[0] for t in chosen}) == sorted(set(int(x) for x in gb.d))
        for d, L, C in chosen:
            assert bt.tiling(d) == (d, L, C)
        # tuning ran epochs, then put Z and the epoch counter back
        assert bt.epoch_counter == 1
        for i in range(gb.num_graphs):
            assert np.array_equal(bt.embedding(i), z1[i])
    # the cached tiling is applied without timing, and fixes the result
    runs = []
    for use_cache in (True, False):
        with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=5, lr=0.02, minibatch=128) as bt:
            if use_cache:
                assert bt.autotune(1, cache=cache, key="k") == chosen
            else:
                for d, L, C in chosen:
                    bt.set_tiling(d, L, C)
            bt.train(2)
            runs.append([bt.embedding(i) for i in range(gb.num_graphs)])
    for a, b in zip(*runs):
        assert np.array_equal(a, b)


@pytest.mark.parametrize("model", MODELS)
def test_bf16_batch_steps_against_oracle(model):
    """BF16 storage in the batched form, every minibatch position of two
    epochs and every graph against the oracle fed the same BF16-rounded
    partner rows and FP32 master own rows, with the per-minibatch bound."""
    gb = small_sbm_batch(6, seed=23, dims=(16, 64, 128))
    glist = [gb.graph(i) for i in range(gb.num_graphs)]
    dims = [int(x) for x in gb.d]
    seeds = [1000 + 17 * i for i in range(len(glist))]
    n, d, sd, rp, ci = concat(glist, dims, seeds)
    s, b, lr = 5, 128, 0.02
    M = max(-(-g.n // b) for g in glist)
    with f2v.Batch(n, d, sd, rp, ci, model=model, s=s, lr=lr, minibatch=b,
                   precision=f2v.BF16) as bt:
        which = range(len(glist))
        for e in range(2):
            for k in range(M):
                before = [bt.embedding(i).astype(np.float64) for i in which]
                bt.run_minibatches(1)
                check_step(bt, glist, d, seeds, model, s, b, lr, e, k, before, which, bf16=True)


@pytest.mark.parametrize("model", MODELS)
def test_bf16_batch_matches_bf16_context(model):
    """BF16 storage: the batch and the single-graph BF16 context apply the same
    rounding (partner rows rounded to nearest even, FP32 master); they differ
    only in FP32 summation order, which can move a master value across a BF16
    rounding boundary, so the bound is a few BF16 steps of eta * force."""
    gb = small_sbm_batch(6, seed=23, dims=(16, 64, 128))
    s, b, lr = 5, 128, 0.02
    with f2v.Batch.from_graphs(gb, model=model, s=s, lr=lr, minibatch=b,
                               precision=f2v.BF16) as bt:
        bt.train(2)
        for i in range(gb.num_graphs):
            g = gb.graph(i)
            with f2v.Context(g.row_ptr, g.col_idx, g.n, int(gb.d[i]), model=model, s=s, lr=lr,
                             minibatch=b, seed=int(gb.seed[i]), precision=f2v.BF16) as ctx:
                ctx.train(2)
                want = ctx.embedding().astype(np.float64)
            got = bt.embedding(i)
            err = np.abs(got - want) / np.maximum(np.abs(want), 1e-2)
            assert np.isfinite(got).all()
            assert err.max() <= 2e-2, f"graph {i}: {err.max():.3e}"
            assert np.median(err) <= 1e-5


def test_full_batched_workload_sampled():
    """The batched workload at full size (4,096 SBM graphs, n log-uniform in
    [50, 20000], 2-16 blocks, p_in 0.05, p_out 0.002, d round-robin {2, 16,
    64}, s = 5, b = 128): the first minibatch positions one at a time, the
    bulk of the epoch in one launch, and the last position of the largest
    graphs, each checked on sampled graphs (the largest of each row size and
    random ones) against the oracle."""
    gb = graphs.sbm_batch(4096, seed=1)
    s, b, lr = 5, 128, 0.02
    rng = np.random.default_rng(3)
    pick = []
    for dd in (2, 16, 64):
        idx = np.flatnonzero(gb.d == dd)
        pick.extend(idx[np.argsort(gb.n[idx])[-3:]].tolist())
        pick.extend(rng.choice(idx, 5, replace=False).tolist())
    glist = {int(i): gb.graph(int(i)) for i in pick}
    M = int(max(-(-int(x) // b) for x in gb.n))
    with f2v.Batch.from_graphs(gb, model=f2v.TDIST, s=s, lr=lr, minibatch=b) as bt:
        for k in list(range(3)) + [M - 1]:
            if bt.progress[1] < k:
                bt.run_minibatches(k - bt.progress[1])
            before = {i: bt.embedding(i).astype(np.float64) for i in glist}
            bt.run_minibatches(1)
            check_step(bt, glist, gb.d, gb.seed, f2v.TDIST, s, b, lr, 0, k, before, list(glist))
        assert bt.progress == (1, 0)


def test_batch_create_reports_the_bad_graph():
    """Graphs are checked concurrently; the error names the first bad one."""
    gb = graphs.sbm_batch(8, seed=3, n_range=(50, 400))
    rp = gb.row_ptr.copy()
    ci = gb.col_idx.copy()
    # a self-loop in graph 5: its first entry made to point at its own row
    r0 = int(gb.row_off[5])
    c0 = int(gb.col_off[5])
    u = int(np.flatnonzero(np.diff(rp[r0:r0 + gb.n[5] + 1]) > 0)[0])
    ci[c0 + rp[r0 + u]] = u
    with pytest.raises(f2v.F2VError, match="graph 5: self-loop"):
        f2v.Batch(gb.n, gb.d, gb.seed, rp, ci)
