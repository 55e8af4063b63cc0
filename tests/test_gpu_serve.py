"""Serving loop: continuous batching with HBM-budget admission (GPU).

Each job's result must be the same alone and in the mix (bit for bit: a job's schedule
depends on its graph only), the running jobs' reservations must never exceed the budget,
and failures are per job and injected on the host (rejection, cancellation, an allocation
that fails by the test hook, invalid input), never by faulting the GPU.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _jobs():
    out = []
    sizes = [(300, 900), (2000, 9000), (800, 6000), (5000, 40000), (150, 300), (3000, 20000),
             (1200, 5000), (700, 2100), (4000, 30000), (250, 1200)]
    for k, (n, E) in enumerate(sizes):
        if k % 3 == 0:
            e = synth.chung_lu_directed(n, E, 2.1, k, max(10.0, E / 20), "uniform")
        else:
            e = synth.chung_lu_undirected(n, E, 2.1, k, max(10.0, E / 20))
        d = [16, 64, 128, 256][k % 4]
        out.append(dict(edges=e, d=d, iters=3 + k % 3, seed=100 + k, storage="bf16" if k % 2 else "f32"))
    return out


@pytest.fixture(scope="module")
def jobs():
    return _jobs()


def _alone(job):
    import paper_2102_02302_gb300 as pkg
    e = job["edges"]
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        n = ctx.info()["n"]
        ctx.init(job["d"], job["seed"], job["storage"])
        out = np.empty((n, job["d"]), np.float32)
        ctx.propagate(job["iters"], out)
        ctx.sync()
    return out


def _submit(srv, job, out):
    e = job["edges"]
    return srv.submit(e.src, e.dst, e.weights, e.directed, job["d"], job["iters"], job["seed"],
                      job["storage"], out)


def test_results_alone_equal_results_in_the_mix(jobs):
    import paper_2102_02302_gb300 as pkg
    alone = [_alone(j) for j in jobs]
    with pkg.Server(0, max_slots=4) as srv:
        outs, ids = [], []
        for j, a in zip(jobs, alone):
            out = np.full(a.shape, np.nan, np.float32)
            outs.append(out)
            ids.append(_submit(srv, j, out))
        results = [srv.poll(i, 60_000) for i in ids]
        assert srv.stats()["completed"] == len(jobs)
    for j, a, o, r in zip(jobs, alone, outs, results):
        assert r is not None and r.status == 0
        assert r.n == a.shape[0]
        assert r.t_submit <= r.t_admit <= r.t_done
        assert np.array_equal(o, a)
    # and the mix still matches the oracle
    for j, o in list(zip(jobs, outs))[:3]:
        g = oracle.build_from(j["edges"])
        T0 = oracle.init(g.ids, j["d"], j["seed"])
        if j["storage"] == "bf16":
            continue
        want = oracle.propagate(g, T0, j["iters"])
        assert np.abs(o.astype(np.float64) - want).max() <= 1e-5
    # work overlapped on the device: some jobs ran at the same time
    spans = sorted((r.t_admit, r.t_done) for r in results)
    assert any(spans[k + 1][0] < spans[k][1] for k in range(len(spans) - 1))


def test_budget_is_never_exceeded_and_oversized_jobs_are_rejected(jobs):
    import paper_2102_02302_gb300 as pkg
    est = []
    with pkg.Server(0, max_slots=4) as probe:
        for j in jobs:
            e = j["edges"]
            est.append(probe.estimate(e.src, e.dst, e.weights, e.directed, j["d"], j["iters"], j["storage"]))
    budget = int(max(est) * 1.5)  # at most ~1-2 jobs at once
    with pkg.Server(0, hbm_budget_bytes=budget, max_slots=4) as srv:
        ids = [_submit(srv, j, None) for j in jobs]
        res = [srv.poll(i, 120_000) for i in ids]
        big = jobs[3]["edges"]
        with pytest.raises(pkg.CleoraError) as ex:
            srv.submit(big.src, big.dst, None, False, 1024, 3, 0, "f32", None)
        assert ex.value.status == pkg.CLEORA_ERR_REJECTED or budget >= srv.estimate(big.src, big.dst, d=1024)
    assert all(r.status == 0 for r in res)
    events = sorted([(r.t_admit, r.bytes_reserved) for r in res] + [(r.t_done, -r.bytes_reserved) for r in res])
    level = 0
    for _, delta in events:
        level += delta
        assert level <= budget


def test_cancel_timeout_injected_failure_and_bad_input(jobs):
    import paper_2102_02302_gb300 as pkg
    # one slot and a slow first job keep the later jobs waiting long enough to cancel one
    blocker = dict(edges=synth.chung_lu_undirected(200_000, 2_000_000, 2.1, 7, 50_000.0), d=1024,
                   iters=5, seed=1, storage="f32")
    with pkg.Server(0, max_slots=1, inject_alloc_failure_every=2) as srv:
        ids = [_submit(srv, j, None) for j in [blocker] + jobs[:5]]
        # poll with a zero timeout on a job that cannot be done yet
        assert srv.poll(ids[-1], 0) is None
        assert srv.cancel(ids[-1]) == 0
        res = [srv.poll(i, 60_000) for i in ids]
        assert res[-1].status == pkg.CLEORA_ERR_CANCELLED
        statuses = [r.status for r in res[:-1]]
        # admitted jobs 2 and 4 had their first device allocation fail (host-side hook)
        assert statuses == [0, pkg.CLEORA_ERR_OOM, 0, pkg.CLEORA_ERR_OOM, 0]
        # the server keeps serving after failures
        jid = _submit(srv, jobs[0], None)
        assert srv.poll(jid, 60_000).status in (0, pkg.CLEORA_ERR_OOM)
        # malformed jobs are refused at submit, bad weights fail the job itself
        e = jobs[1]["edges"]
        with pytest.raises(pkg.CleoraError):
            srv.submit(e.src, e.dst, None, False, 12, 3)
        w = np.zeros(e.num_edges, np.float32)
        jid = srv.submit(e.src, e.dst, w, False, 16, 3)
        r = srv.poll(jid, 60_000)
        assert r.status in (pkg.CLEORA_ERR_INVALID_ARG, pkg.CLEORA_ERR_OOM)


def test_next_returns_every_job_once_in_completion_order(jobs):
    import paper_2102_02302_gb300 as pkg
    with pkg.Server(0, max_slots=3) as srv:
        ids = {_submit(srv, j, None) for j in jobs}
        seen = []
        while len(seen) < len(ids):
            r = srv.next(60_000)
            assert r is not None
            seen.append(r[0])
            assert r[1].status == 0
        assert sorted(seen) == sorted(ids)
        assert srv.next(0) is None  # nothing left
