"""Parity at the full workload sizes, in the launch configuration the bench times.

Mid-size weighted directed graph (2M nodes, 40M edges, d = 256): the whole oracle runs, so
CSR, FP32 and BF16 results are compared entry by entry.

Large undirected graph (41M nodes, 1.4B edges, 2.8B CSR entries, d = 128): the oracle cannot
run whole on the host, so the checks are properties that hold at any size (every id present,
CSR invariants, symmetry, unit norms, determinism), the CSR rows of a sample compared bit for
bit with the oracle's own build of the edges that touch them, and the relation that defines an
iteration, T_k[a] = rownorm(sum_b M_ab T_{k-1}[b]), on over a million rows that include every
row the kernel splits across warps: the oracle applies one FP64 step to the library's
previous iterate over the checked CSR.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32)
    return (r << 16).view(np.float32).astype(np.float64)


def test_mid_size_graph_full_oracle_parity():
    import paper_2102_02302_gb300 as pkg
    spec = synth.MID
    e = spec.generate()
    g = oracle.build_from(e)
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        c = ctx.csr()
        assert np.array_equal(ctx.node_ids(), g.ids)
        assert np.array_equal(c["rowptr"], g.rowptr) and np.array_equal(c["col"], g.col)
        assert np.array_equal(c["val"].view(np.uint32), g.val32.view(np.uint32))
        assert np.array_equal(c["deg"].view(np.uint64), g.deg.view(np.uint64))
        del c
        T0 = oracle.init(g.ids, spec.d, 0)
        want = oracle.propagate(g, T0, spec.iters)
        out = np.empty((g.n, spec.d), np.float32)
        ctx.init(spec.d, 0, "f32")
        ctx.propagate(spec.iters, out)
        ctx.sync()
        err = np.abs(out - want).max()
        assert err <= 1e-5, err
        want16 = oracle.propagate(g, _bf16_round(T0), spec.iters)
        ctx.init(spec.d, 0, "bf16")
        ctx.propagate(spec.iters, out)
        ctx.sync()
        err16 = np.abs(out - want16).max()
        assert err16 <= 2e-2, err16
        cos = (out * want16).sum(1) / (np.linalg.norm(out, axis=1) * np.linalg.norm(want16, axis=1))
        assert cos.min() >= 0.999


@pytest.fixture(scope="module")
def large():
    import torch
    import synth.gpu
    spec = synth.LARGE
    src, dst, meta = synth.gpu.chung_lu_undirected(spec.n, spec.edges, spec.gamma, spec.seed,
                                                   spec.max_deg)
    yield spec, src, dst
    del src, dst
    torch.cuda.empty_cache()


SPLIT_LEN = 8192  # the library's default: longer rows run as split chunks


def _id_key(x):
    """uint64 ids held in int64 tensors -> keys whose signed order is the unsigned order."""
    import torch
    return x ^ torch.tensor(-(1 << 63), dtype=torch.int64, device=x.device)


def _segments(rowptr, rows):
    """Entry positions of the given rows, concatenated in the given order."""
    import torch
    beg, end = rowptr[rows], rowptr[rows + 1]
    lens = end - beg
    start = torch.repeat_interleave(beg - torch.cumsum(lens, 0) + lens, lens)
    return start + torch.arange(int(lens.sum()), device=rowptr.device), lens


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_large_graph_properties_and_sampled_step(large, storage):
    import torch
    import paper_2102_02302_gb300 as pkg
    spec, src, dst = large
    dev = torch.device("cuda")
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    with pkg.Context(0, stream.cuda_stream) as ctx:
        ctx.graph_build(src, dst, None, False)
        inf = ctx.info()
        n, nnz = inf["n"], inf["nnz"]
        assert not inf["has_val"] and nnz == 2 * src.numel()  # simple graph: both directions
        ids = torch.empty(n, dtype=torch.int64, device=dev)
        rowptr = torch.empty(n + 1, dtype=torch.int64, device=dev)
        col = torch.empty(nnz, dtype=torch.int32, device=dev)
        deg = torch.empty(n, dtype=torch.float64, device=dev)
        pkg.cleora_node_ids(ctx.handle, ids)
        pkg.cleora_get_csr(ctx.handle, rowptr, col, None, None, deg)
        ctx.sync()
        # ids: strictly ascending as unsigned, and every endpoint is one of them
        flip = _id_key(ids)
        assert bool((flip[1:] > flip[:-1]).all())
        for ends in (src, dst):
            f = _id_key(ends)
            pos = torch.searchsorted(flip, f).clamp_(max=n - 1)
            assert bool((flip[pos] == f).all())
            del f, pos
        # CSR invariants
        lens = rowptr[1:] - rowptr[:-1]
        assert int(rowptr[0]) == 0 and int(rowptr[-1]) == nnz and bool((lens >= 0).all())
        assert bool((deg == lens.to(torch.float64)).all())
        assert int(col.min()) >= 0 and int(col.max()) < n
        assert int(lens.max()) == inf["max_row_len"] and inf["max_row_len"] > 2_000_000
        gen = torch.Generator(device="cpu").manual_seed(7)
        long_rows = torch.nonzero(lens > SPLIT_LEN).flatten().cpu()
        assert long_rows.numel() > 1000
        rnd = torch.randint(0, n, (1_000_000,), generator=gen)
        hubs = torch.topk(lens, 6).indices.cpu()
        rp = rowptr.cpu()
        for r in torch.unique(torch.cat([hubs, rnd[:2000]])).tolist():  # ascending, symmetric
            seg = col[int(rp[r]):int(rp[r + 1])].long()
            assert bool((seg[1:] > seg[:-1]).all())
            if seg.numel() and seg.numel() < 5000:
                back = seg[torch.randint(0, seg.numel(), (1,), generator=gen).item()].item()
                bseg = col[int(rp[back]):int(rp[back + 1])]
                assert bool((bseg == r).any())

        # CSR rows of a sample, bit for bit against the oracle's build of every edge that
        # touches them (that build holds each sampled row whole): neighbour ids and degrees
        sub = torch.unique(torch.cat([hubs, rnd[:100_000],
                                      long_rows[torch.randperm(long_rows.numel(), generator=gen)[:64]]]))
        s_ids = ids[sub.to(dev)]
        s_sorted = torch.sort(_id_key(s_ids)).values

        def member(x):
            f = _id_key(x)
            p = torch.searchsorted(s_sorted, f).clamp_(max=s_sorted.numel() - 1)
            return s_sorted[p] == f

        mask = member(src) | member(dst)
        sg = oracle.build_graph(src[mask].cpu().numpy().view(np.uint64),
                                dst[mask].cpu().numpy().view(np.uint64), None, False)
        del mask
        sg_key = _id_key(torch.from_numpy(sg.ids.view(np.int64)))
        pa = torch.searchsorted(sg_key, _id_key(s_ids.cpu()))  # sampled rows in sg
        assert bool((sg_key[pa] == _id_key(s_ids.cpu())).all())
        lib_pos, lib_len = _segments(rowptr, sub.to(dev))
        lib_nbr = ids[col[lib_pos].long()].cpu().numpy().view(np.uint64)
        sg_pos, sg_len = _segments(torch.from_numpy(sg.rowptr), pa)
        sg_nbr = sg.ids[sg.col[sg_pos.numpy()]]
        assert torch.equal(lib_len.cpu(), sg_len)
        assert np.array_equal(lib_nbr, sg_nbr)
        assert np.array_equal(deg[sub.to(dev)].cpu().numpy(), sg.deg[pa.numpy()])
        del lib_pos, lib_nbr, sg, sg_pos, sg_nbr

        # iterations: deterministic, unit norms
        d = spec.d
        ctx.init(d, 0, storage)
        ctx.propagate(spec.iters - 1)
        T3 = torch.empty((n, d), dtype=torch.float32, device=dev)
        pkg.cleora_get_embeddings(ctx.handle, T3, "f32")
        T4 = torch.empty((n, d), dtype=torch.float32, device=dev)
        ctx.propagate(1, T4)
        ctx.init(d, 0, storage)
        T4b = torch.empty((n, d), dtype=torch.float32, device=dev)
        ctx.propagate(spec.iters, T4b)
        ctx.sync()
        assert torch.equal(T4, T4b)
        del T4b
        norms = torch.linalg.vector_norm(T4, dim=1)
        tol_norm = 1e-5 if storage == "f32" else 1e-2
        assert float((norms - 1).abs().max()) <= tol_norm

        # one step on >= 1M rows including every split row: the oracle's FP64 step over the
        # checked CSR from the library's previous iterate (BF16 values are exact in FP32)
        rows = torch.unique(torch.cat([long_rows, rnd]))
        assert rows.numel() >= 1_000_000
        got = T4[rows.to(dev)].cpu().numpy().astype(np.float64)
        del T4
        T_prev = T3.cpu().numpy()
        del T3
        col_h = col.cpu().numpy()
        want = oracle.step_csr_rows(rp.numpy(), col_h, None, T_prev, rows.numpy())
        del T_prev, col_h
        tol = 1e-5 if storage == "f32" else 2e-2
        assert np.abs(got - want).max() <= tol
        if storage == "bf16":
            cos = (got * want).sum(1) / (np.linalg.norm(got, axis=1) * np.linalg.norm(want, axis=1))
            assert cos.min() >= 0.999
    torch.cuda.set_stream(torch.cuda.default_stream())
