"""The served form (include/f2v_serve.h): jobs admitted as they arrive under
a device-memory budget, stepped together one epoch at a time.

The property that matters for serving: a job's result is the same whether it
ran alone or in a mix with other jobs.  The server runs a job in the batched
form, whose per-graph arithmetic does not depend on the other graphs of the
batch, so the results are compared bit for bit with a batch holding that
graph alone (whose parity with the FP64 oracle tests/test_batch_gpu.py
checks); one job is also checked against the oracle directly.
"""
import time

import numpy as np
import pytest

import oracle
from paper_2009_10035_gb300 import f2v, graphs

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    torch.cuda.set_device(0)
    f2v.load_library()


def job_mix():
    """(graph, params) of a mixed set of jobs: sizes, row sizes, precisions,
    minibatch sizes and epoch counts differ."""
    gs = [graphs.rmat(11, 8, seed=1), graphs.sbm(1500, 5, 0.05, 0.002, seed=2),
          graphs.erdos_renyi(800, m=4000, seed=3), graphs.rmat(12, 12, seed=4),
          graphs.sbm(300, 2, 0.08, 0.01, seed=5), graphs.rmat(10, 16, seed=6),
          graphs.erdos_renyi(2000, m=9000, seed=7), graphs.sbm(5000, 9, 0.03, 0.001, seed=8)]
    dims = [2, 32, 128, 32, 2, 128, 64, 16]
    prec = [f2v.FP32, f2v.FP32, f2v.BF16, f2v.BF16, f2v.FP32, f2v.FP32, f2v.BF16, f2v.FP32]
    mbs = [256, 256, 1024, 256, 256, 1024, 256, 512]
    eps = [3, 2, 4, 3, 5, 2, 3, 2]
    jobs = []
    for i, g in enumerate(gs):
        jobs.append((g, dict(d=dims[i], precision=prec[i], minibatch=mbs[i], epochs=eps[i],
                             seed=100 + i, model=f2v.TDIST if i % 3 else f2v.SIGMOID,
                             s=5, lr=0.02)))
    return jobs


def run_alone(g, p):
    with f2v.Batch([g.n], [p["d"]], [p["seed"]], g.row_ptr, g.col_idx, model=p["model"],
                   s=p["s"], lr=p["lr"], minibatch=p["minibatch"],
                   precision=p["precision"]) as bt:
        bt.set_schedule(f2v.LR_LINEAR, p["epochs"])
        bt.train(p["epochs"])
        return bt.embedding(0)


def test_results_same_alone_and_in_the_mix():
    jobs = job_mix()
    with f2v.Server(budget_bytes=8 << 30) as srv:
        ids = []
        for i, (g, p) in enumerate(jobs):
            ids.append(srv.submit(g.row_ptr, g.col_idx, g.n, **p))
            if i == 3:
                time.sleep(0.02)       # the rest arrive while the first ones run
        outs = [srv.wait(j) for j in ids]
        infos = [srv.info(j) for j in ids]
        st = srv.stats()
    for (g, p), z, info in zip(jobs, outs, infos):
        assert info.state == f2v.JOB_DONE and info.epochs_done == p["epochs"]
        assert 0 <= info.submit_s <= info.admit_s <= info.finish_s
        want = run_alone(g, p)
        assert np.isfinite(z).all()
        assert np.array_equal(z, want), f"job with n={g.n}, d={p['d']} differs from alone"
    assert st.done == len(jobs) and st.failed == 0
    assert st.pairs_done == sum(i.pairs for i in infos)
    # the jobs shared steps: some ran at the same time
    spans = sorted((i.admit_s, i.finish_s) for i in infos)
    assert any(b[0] < a[1] for a, b in zip(spans, spans[1:]))


def test_served_job_matches_oracle():
    g = graphs.erdos_renyi(1000, m=10000, seed=1)
    with f2v.Server(budget_bytes=1 << 30) as srv:
        jid = srv.submit(g.row_ptr, g.col_idx, g.n, d=32, model=f2v.TDIST, s=5, lr=0.02,
                         minibatch=256, seed=1, epochs=1)
        z = srv.wait(jid)
    want = oracle.train(f2v.TDIST, g.row_ptr, g.col_idx, oracle.init_embedding(g.n, 32, 1), 5,
                        256, 1, 0.02, 1)
    err = np.abs(z - want) / np.maximum(np.abs(want), 1e-3)
    assert err.max() <= 1e-5


def test_budget_bounds_admission_in_arrival_order():
    jobs = [(graphs.rmat(12, 8, seed=s), dict(d=64, epochs=3, seed=s, minibatch=512))
            for s in range(6)]
    with f2v.Server(budget_bytes=1 << 40) as probe:
        g0, p0 = jobs[0]
        need = probe.info(probe.submit(g0.row_ptr, g0.col_idx, g0.n, **p0)).device_bytes
        probe.wait_all()
    budget = int(2.5 * need)          # room for two of these jobs at a time
    with f2v.Server(budget_bytes=budget) as srv:
        ids = [srv.submit(g.row_ptr, g.col_idx, g.n, **p) for g, p in jobs]
        srv.wait_all()
        infos = [srv.info(j) for j in ids]
        st = srv.stats()
    assert all(i.state == f2v.JOB_DONE for i in infos)
    assert st.peak_bytes <= budget
    admits = [i.admit_s for i in infos]
    assert admits == sorted(admits)
    for t in admits:
        live = sum(1 for i in infos if i.admit_s <= t < i.finish_s)
        assert live <= 2


def test_max_active_one_runs_jobs_one_after_another():
    jobs = [(graphs.sbm(400, 2, 0.05, 0.01, seed=s), dict(d=16, epochs=2, seed=s, minibatch=128))
            for s in range(4)]
    with f2v.Server(budget_bytes=1 << 30, max_active=1) as srv:
        ids = [srv.submit(g.row_ptr, g.col_idx, g.n, **p) for g, p in jobs]
        outs = [srv.wait(j) for j in ids]
        infos = [srv.info(j) for j in ids]
    for a, b in zip(infos, infos[1:]):
        assert b.admit_s >= a.finish_s
    for (g, p), z in zip(jobs, outs):
        q = dict(model=f2v.TDIST, s=5, lr=0.02, precision=f2v.FP32, **p)
        assert np.array_equal(z, run_alone(g, q))


def test_invalid_jobs_are_rejected_at_submit():
    g = graphs.erdos_renyi(100, m=300, seed=1)
    with f2v.Server(budget_bytes=1 << 16) as srv:
        with pytest.raises(f2v.F2VError, match="d = 3"):
            srv.submit(g.row_ptr, g.col_idx, g.n, d=3)
        bad = g.col_idx.copy()
        bad[0] = g.n + 5
        with pytest.raises(f2v.F2VError, match="out of range"):
            srv.submit(g.row_ptr, bad, g.n, d=16)
        with pytest.raises(f2v.F2VError, match="budget"):
            srv.submit(g.row_ptr, g.col_idx, g.n, d=128, epochs=1)   # Z alone > 64 KiB
        assert srv.stats().submitted == 0
