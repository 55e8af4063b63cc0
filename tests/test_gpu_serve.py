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
        assert r.t_submit <= r.t_admit <= r.t_built <= r.t_inited <= r.t_done
        assert np.array_equal(o, a)
    # and every job of the mix matches the oracle (BF16 jobs from the BF16-rounded T_0)
    for j, o in zip(jobs, outs):
        g = oracle.build_from(j["edges"])
        T0 = oracle.init(g.ids, j["d"], j["seed"])
        if j["storage"] == "bf16":
            b = T0.astype(np.float32).view(np.uint32).astype(np.uint64)
            T0 = ((((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32) << 16).view(np.float32)
            want = oracle.propagate(g, T0.astype(np.float64), j["iters"])
            assert np.abs(o.astype(np.float64) - want).max() <= 2e-2
            cos = (o * want).sum(1) / (np.linalg.norm(o, axis=1) * np.linalg.norm(want, axis=1))
            assert cos.min() >= 0.999
        else:
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
    import time
    with pkg.Server(0, max_slots=1, inject_alloc_failure_every=2) as srv:
        ids = [_submit(srv, blocker, None)]
        t_end = time.time() + 60
        while srv.stats()["running"] == 0 and time.time() < t_end:  # the blocker holds the slot
            time.sleep(0.001)
        ids += [_submit(srv, j, None) for j in jobs[:5]]
        # poll with a zero timeout on a job that cannot be done yet
        assert srv.poll(ids[-1], 0) is None
        assert srv.cancel(ids[-1]) == 0
        res = [srv.poll(i, 60_000) for i in ids]
        assert res[-1].status == pkg.CLEORA_ERR_CANCELLED
        # in admission order, the 2nd and 4th admitted jobs had their first device allocation
        # fail (host-side hook); admission follows the jobs' estimated virtual finish times
        ran = sorted(res[:-1], key=lambda r: r.t_admit)
        assert [r.status for r in ran] == [0, pkg.CLEORA_ERR_OOM, 0, pkg.CLEORA_ERR_OOM, 0]
        assert ran[0].t_done <= ran[1].t_admit  # one slot: the blocker ran first
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


def test_short_jobs_pass_a_long_one_that_arrived_just_before():
    import time
    import paper_2102_02302_gb300 as pkg
    # one slot: a blocker runs; then a long job and, right after it, short ones are queued.
    # The short ones' virtual finish times (arrival + estimated service) come first.
    blocker = synth.chung_lu_undirected(200_000, 2_000_000, 2.1, 7, 50_000.0)
    long_job = synth.chung_lu_undirected(400_000, 4_000_000, 2.1, 8, 80_000.0)
    short = [synth.chung_lu_undirected(300, 900, 2.1, k, 40.0) for k in range(4)]
    with pkg.Server(0, max_slots=1) as srv:
        b = srv.submit(blocker.src, blocker.dst, None, False, 256, 4)
        t_end = time.time() + 60
        while srv.stats()["running"] == 0 and time.time() < t_end:
            time.sleep(0.001)
        lj = srv.submit(long_job.src, long_job.dst, None, False, 256, 4)
        sj = [srv.submit(e.src, e.dst, None, False, 16, 3) for e in short]
        res_long = srv.poll(lj, 120_000)
        res_short = [srv.poll(i, 120_000) for i in sj]
        srv.poll(b, 120_000)
    assert res_long.status == 0 and all(r.status == 0 for r in res_short)
    assert all(r.t_done <= res_long.t_admit for r in res_short)


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


def test_short_slots_run_short_jobs_while_long_ones_hold_every_slot(jobs):
    import time
    import paper_2102_02302_gb300 as pkg
    # two long jobs hold both general slots; short jobs that arrive after them run on the short
    # slot (on a high-priority stream) and finish first, with the same bits as alone
    longs = [synth.chung_lu_undirected(2_000_000, 20_000_000, 2.1, 30 + k, 200_000.0) for k in range(2)]
    short = [jobs[k] for k in (0, 4, 7, 9)]
    alone = [_alone(j) for j in short]
    with pkg.Server(0, max_slots=2, short_slots=1, short_job_seconds=0.02) as srv:
        lid = [srv.submit(e.src, e.dst, None, False, 1024, 5, 0, "f32", None, nodes_hint=2_000_000)
               for e in longs]
        t_end = time.time() + 60
        while srv.stats()["running"] < 2 and time.time() < t_end:
            time.sleep(0.001)
        outs = [np.full(a.shape, np.nan, np.float32) for a in alone]
        sid = [_submit(srv, j, o) for j, o in zip(short, outs)]
        res_short = [srv.poll(i, 120_000) for i in sid]
        res_long = [srv.poll(i, 300_000) for i in lid]
    assert all(r.status == 0 for r in res_long + res_short)
    assert all(r.slot == 2 for r in res_short)  # the short slot (slots 0, 1 are general)
    assert max(r.t_done for r in res_short) < min(r.t_done for r in res_long)
    for o, a in zip(outs, alone):
        assert np.array_equal(o, a)
