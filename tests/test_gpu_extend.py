"""Inductive rows and chunked embedding (Sec. 1 "Inductivity"/"Additivity"; Algorithm 1)
through the C ABI, against the FP64 oracle."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32)
    return (r << 16).view(np.float32).astype(np.float64)


def _new_edges(g, count, per, seed, unknown=True, weighted=True):
    rs = np.random.default_rng(seed)
    new_ids = synth.node_ids(count, 10_000 + seed)
    u = np.repeat(new_ids, per)
    b = g.ids[rs.integers(0, g.n, u.size)]
    if unknown:
        b[::7] = np.uint64(0xDEADBEEF)  # not a node: dropped
    b[1::11] = b[0::11][: b[1::11].size]  # some duplicates
    w = rs.uniform(0.1, 2.0, u.size).astype(np.float32) if weighted else None
    return u, b, w


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("weighted", [False, True])
def test_inductive_rows_match_oracle(storage, weighted):
    import paper_2102_02302_gb300 as pkg
    e = synth.SMALL.generate()
    g = oracle.build_from(e)
    d, iters = 128, 3
    T0 = oracle.init(g.ids, d, 11)
    if storage == "bf16":
        T0 = _bf16_round(T0)
    T = oracle.propagate(g, T0, iters)
    u, b, w = _new_edges(g, 1500, 9, 2, weighted=weighted)
    ids_w, rows_w, dropped_w = oracle.inductive(g, T, u, b, w)
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        ctx.init(d, 11, storage)
        ctx.propagate(iters)
        out = np.empty((len(ids_w), d), np.float32)
        out_ids = np.empty(len(ids_w), np.uint64)
        nn, nd = pkg.cleora_inductive(ctx.handle, u, b, w, out_ids, out)
        # the context is unchanged: its next iteration still works
        ctx.propagate(1)
        ctx.sync()
    assert nn == len(ids_w) and nd == dropped_w
    assert np.array_equal(out_ids, ids_w)
    tol = 1e-5 if storage == "f32" else 2e-2
    assert np.abs(out - rows_w).max() <= tol


def test_inductive_device_buffers_and_errors():
    import torch
    import paper_2102_02302_gb300 as pkg
    e = synth.random_multigraph(500, 3000, 4, True, True)
    g = oracle.build_from(e)
    T = oracle.propagate(g, oracle.init(g.ids, 64, 1), 2)
    u, b, w = _new_edges(g, 200, 4, 5)
    ids_w, rows_w, _ = oracle.inductive(g, T, u, b, w)
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, True)
        with pytest.raises(pkg.CleoraError) as ex:
            pkg.cleora_inductive(ctx.handle, u, b, w)
        assert ex.value.status == pkg.CLEORA_ERR_STATE
        ctx.init(64, 1)
        ctx.propagate(2)
        ctx.sync()
        du = torch.from_numpy(u.view(np.int64)).cuda()
        db = torch.from_numpy(b.view(np.int64)).cuda()
        dw = torch.from_numpy(w).cuda()
        out = torch.empty((len(ids_w), 64), dtype=torch.float32, device="cuda")
        oid = torch.empty(len(ids_w), dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        pkg.cleora_inductive(ctx.handle, du, db, dw, oid, out)
        ctx.sync()
        assert np.array_equal(oid.cpu().numpy().view(np.uint64), ids_w)
        assert np.abs(out.cpu().numpy() - rows_w).max() <= 1e-5
        small = np.empty((1, 64), np.float32)
        with pytest.raises(pkg.CleoraError):
            pkg.cleora_inductive(ctx.handle, u, b, w, None, small)
        bad = w.copy()
        bad[3] = -1.0
        with pytest.raises(pkg.CleoraError):
            pkg.cleora_inductive(ctx.handle, u, b, bad)


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("Q", [1, 3])
def test_chunked_embedding_matches_oracle(storage, Q):
    import paper_2102_02302_gb300 as pkg
    e = synth.SMALL.generate()
    E = e.num_edges
    offs = [E * q // Q for q in range(Q + 1)]
    d, iters = 64, 3
    ids_w, T_w = oracle.chunked_embed(e.src, e.dst, None, offs, False, d, iters, 5)
    if storage == "bf16":  # each chunk starts from the BF16-rounded T_0
        acc = np.zeros_like(T_w)
        ends = np.concatenate([e.src, e.dst])
        occ_all = np.zeros(ids_w.size)
        np.add.at(occ_all, np.searchsorted(ids_w, ends), 1.0)
        for q in range(Q):
            gq = oracle.build_graph(e.src[offs[q]:offs[q + 1]], e.dst[offs[q]:offs[q + 1]], None, False)
            Tq = oracle.propagate(gq, _bf16_round(oracle.init(gq.ids, d, 5)), iters)
            occ = np.zeros(gq.n)
            np.add.at(occ, np.searchsorted(gq.ids, np.concatenate([e.src[offs[q]:offs[q + 1]],
                                                                   e.dst[offs[q]:offs[q + 1]]])), 1.0)
            v = np.searchsorted(ids_w, gq.ids)
            acc[v] += (occ / occ_all[v])[:, None] * Tq
        T_w = acc
    with pkg.Context(0) as ctx:
        out = np.empty((ids_w.size, d), np.float32)
        out_ids = np.empty(ids_w.size, np.uint64)
        n = pkg.cleora_chunked_embed(ctx.handle, e.src, e.dst, None, offs, False, d, iters, 5, storage,
                                     out_ids, out)
    assert n == ids_w.size and np.array_equal(out_ids, ids_w)
    tol = 1e-5 if storage == "f32" else 2e-2
    assert np.abs(out - T_w).max() <= tol


def test_chunked_single_chunk_equals_plain_run_on_gpu():
    import paper_2102_02302_gb300 as pkg
    e = synth.random_multigraph(400, 2000, 9, True, True)
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, True)
        ctx.init(32, 2)
        n = ctx.info()["n"]
        plain = np.empty((n, 32), np.float32)
        ctx.propagate(4, plain)
        out = np.empty((n, 32), np.float32)
        pkg.cleora_chunked_embed(ctx.handle, e.src, e.dst, e.weights, [0, e.num_edges], True, 32, 4, 2,
                                 "f32", None, out)
    assert np.array_equal(out, plain)  # weight 1 for every node


@pytest.fixture(scope="module")
def dense_multigraph():
    # 100k nodes, 20M undirected edges (duplicates kept): the edge list and CSR dominate the
    # footprint, so a chunk of the edges fits where the whole graph does not
    return synth.random_multigraph(100_000, 20_000_000, 21, False, False)


@pytest.mark.parametrize("storage,out_on", [("f32", "host"), ("f32", "device"), ("bf16", "pinned")])
def test_chunked_embedding_out_of_core_under_a_device_cap(dense_multigraph, storage, out_on):
    import torch
    import paper_2102_02302_gb300 as pkg
    e = dense_multigraph
    E, d, iters = e.num_edges, 8, 3
    g_ids = np.unique(np.concatenate([e.src, e.dst]))
    n = g_ids.size
    es = 4 if storage == "f32" else 2
    whole_csr_t = 8 * (n + 1) + 4 * 2 * E + 2 * n * d * es  # CSR (upper bound) + both T buffers
    cap = int(0.9 * whole_csr_t)
    with pkg.Context(0) as ctx:
        ctx.set_option("chunk_bytes", cap)
        if out_on == "device":
            out_t = torch.empty((n, d), dtype=torch.float32, device="cuda")
            ids_t = torch.empty(n, dtype=torch.int64, device="cuda")
            got_n = pkg.cleora_chunked_embed(ctx.handle, e.src, e.dst, None, None, False, d, iters, 4,
                                             storage, ids_t, out_t)
            torch.cuda.synchronize()
            out, out_ids = out_t.cpu().numpy(), ids_t.cpu().numpy().view(np.uint64)
        else:
            if out_on == "pinned":
                out = torch.empty((n, d), dtype=torch.float32, pin_memory=True).numpy()
            else:
                out = np.empty((n, d), np.float32)
            out_ids = np.empty(n, np.uint64)
            got_n = pkg.cleora_chunked_embed(ctx.handle, e.src, e.dst, None, None, False, d, iters, 4,
                                             storage, out_ids, out)
        info = pkg.cleora_chunked_info(ctx.handle)
    Q = info["chunks"]
    assert got_n == n and np.array_equal(out_ids, g_ids)
    assert Q > 1 and whole_csr_t > cap
    assert 0 < info["peak_device_bytes"] <= cap  # the device never held the whole graph
    offs = [E * q // Q for q in range(Q + 1)]
    if storage == "f32":
        _, want = oracle.chunked_embed(e.src, e.dst, None, offs, False, d, iters, 4)
        tol = 1e-5
    else:  # every chunk starts from the BF16-rounded T_0
        occ_all = np.zeros(n)
        np.add.at(occ_all, np.searchsorted(g_ids, np.concatenate([e.src, e.dst])), 1.0)
        want = np.zeros((n, d))
        for q in range(Q):
            s_, t_ = e.src[offs[q]:offs[q + 1]], e.dst[offs[q]:offs[q + 1]]
            gq = oracle.build_graph(s_, t_, None, False)
            Tq = oracle.propagate(gq, _bf16_round(oracle.init(gq.ids, d, 4)), iters)
            occ = np.zeros(gq.n)
            np.add.at(occ, np.searchsorted(gq.ids, np.concatenate([s_, t_])), 1.0)
            v = np.searchsorted(g_ids, gq.ids)
            want[v] += (occ / occ_all[v])[:, None] * Tq
        tol = 2e-2
    assert np.abs(out - want).max() <= tol
