"""Identifier hashing (Sec. 4.3) and hypergraph expansion (Sec. 3.2) on the GPU through the C ABI,
bit for bit against the oracle's independent restatements (XXH64 from the xxHash
specification; clique and star expansion of each hyperedge's distinct members)."""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu


def _strings(count, seed, max_len=200):
    rs = np.random.default_rng(seed)
    lens = rs.integers(0, max_len + 1, count)
    lens[:min(count, max_len + 1)] = np.arange(min(count, max_len + 1))  # every length 0..max_len
    return [rs.integers(0, 256, int(n), dtype=np.uint8).tobytes() for n in lens]


@pytest.mark.parametrize("seed", [0, 20141025, 2**64 - 1])
@pytest.mark.parametrize("on_device", [False, True])
def test_hash_ids_bit_exact(seed, on_device):
    import torch
    import paper_2102_02302_gb300 as pkg
    strs = _strings(3000, 1)
    blob = np.frombuffer(b"".join(strs), dtype=np.uint8).copy()
    offs = np.zeros(len(strs) + 1, np.int64)
    offs[1:] = np.cumsum([len(s) for s in strs])
    want = oracle.hash_strings(strs, seed)
    with pkg.Context(0) as ctx:
        if on_device:
            b, o = torch.from_numpy(blob).cuda(), torch.from_numpy(offs).cuda()
            out = torch.empty(len(strs), dtype=torch.int64, device="cuda")
            pkg.cleora_hash_ids(ctx.handle, b, o, seed, out)
            got = out.cpu().numpy().view(np.uint64)
        else:
            got = pkg.cleora_hash_ids(ctx.handle, blob, offs, seed)
    assert np.array_equal(got, want)
    # the published vectors through the GPU as well
    assert got[0] == oracle.xxh64(b"", seed)


def _hypergraph(H, n, kmax, seed, empty_every=7):
    rs = np.random.default_rng(seed)
    widths = rs.integers(0, kmax + 1, H)
    widths[::empty_every] = 0
    hoff = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
    ids = synth.node_ids(n, seed)
    members = ids[rs.integers(0, n, int(hoff[-1]))]
    return members, hoff


@pytest.mark.parametrize("mode", ["clique", "star"])
@pytest.mark.parametrize("H,n,kmax", [(1, 5, 5), (500, 300, 12), (3000, 20000, 60), (40, 1000, 700)])
def test_expansion_bit_exact(mode, H, n, kmax):
    import paper_2102_02302_gb300 as pkg
    members, hoff = _hypergraph(H, n, kmax, H + kmax)
    star_ids = synth.node_ids(H, 99) if (mode == "star" and H % 2 == 0) else None
    want_s, want_d = oracle.expand(members, hoff, mode, star_ids)
    with pkg.Context(0) as ctx:
        got_s, got_d = pkg.cleora_expand_hypergraph(ctx.handle, members, hoff, mode, star_ids)
    assert np.array_equal(got_s, want_s) and np.array_equal(got_d, want_d)


@pytest.mark.parametrize("mode", ["clique", "star"])
def test_hypergraph_build_equals_building_the_expanded_edges(mode):
    import torch
    import paper_2102_02302_gb300 as pkg
    members, hoff = _hypergraph(2000, 3000, 20, 5)
    src, dst = oracle.expand(members, hoff, mode)
    g = oracle.build_graph(src, dst, None, False)
    with pkg.Context(0) as ctx:
        E = pkg.cleora_hypergraph_build(ctx.handle, torch.from_numpy(members.view(np.int64)).cuda(),
                                        torch.from_numpy(hoff).cuda(), mode)
        assert E == src.size
        assert np.array_equal(ctx.node_ids(), g.ids)
        c = ctx.csr()
        assert np.array_equal(c["rowptr"], g.rowptr) and np.array_equal(c["col"], g.col)
        assert np.array_equal(c["val"].view(np.uint32), (g.val32 if g.has_val else
                                                          np.repeat(g.inv_deg32, np.diff(g.rowptr))).view(np.uint32))
        ctx.init(64, 3)
        out = np.empty((g.n, 64), np.float32)
        ctx.propagate(3, out)
        ctx.sync()
    want = oracle.propagate(g, oracle.init(g.ids, 64, 3), 3)
    assert np.abs(out - want).max() <= 1e-5


def test_expansion_edge_cases():
    import paper_2102_02302_gb300 as pkg
    with pkg.Context(0) as ctx:
        # no hyperedges, only empty ones, one member, repeated members only
        for members, hoff in ((np.zeros(0, np.uint64), np.zeros(1, np.int64)),
                              (np.zeros(0, np.uint64), np.zeros(4, np.int64)),
                              (synth.node_ids(1, 0), np.array([0, 1], np.int64)),
                              (np.repeat(synth.node_ids(1, 0), 5), np.array([0, 5], np.int64))):
            for mode in ("clique", "star"):
                s, d = pkg.cleora_expand_hypergraph(ctx.handle, members, hoff, mode)
                ws, wd = oracle.expand(members, hoff, mode)
                assert np.array_equal(s, ws) and np.array_equal(d, wd)
        with pytest.raises(pkg.CleoraError):  # offsets must start at 0
            pkg.cleora_expand_hypergraph(ctx.handle, synth.node_ids(3, 0), np.array([1, 3], np.int64))
        with pytest.raises(pkg.CleoraError):  # output too small
            m, h = synth.node_ids(4, 0), np.array([0, 4], np.int64)
            pkg.cleora_expand_hypergraph(ctx.handle, m, h, "clique", None, np.empty(2, np.uint64),
                                         np.empty(2, np.uint64))
