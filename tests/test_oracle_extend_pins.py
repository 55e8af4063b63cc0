"""Pins for the oracle's inductive rows and chunked embedding (CPU).

Inductivity (Sec. 1; Sec. 3.2, a new node averages its neighbours) is pinned by a new leaf,
and by the one-step row of the same node in the graph that includes its edges -- an
independent route through the oracle's graph build and propagation.  Additivity
(Algorithm 1, chunks and merge) is pinned by Q = 1, by vertex-disjoint chunks and by a
two-chunk example worked out by hand.
"""
import numpy as np

import oracle
import synth


def _unit(v):
    return v / np.linalg.norm(v)


def test_new_leaf_takes_its_neighbours_row():
    e = synth.random_multigraph(40, 200, 1, False, True)
    g = oracle.build_from(e)
    T = oracle.propagate(g, oracle.init(g.ids, 16, 3), 2)
    new = np.array([12345678901], np.uint64)
    ids, rows, dropped = oracle.inductive(g, T, new, g.ids[[7]])
    assert dropped == 0 and list(ids) == [12345678901]
    np.testing.assert_allclose(rows[0], _unit(T[7]), atol=1e-15)


def test_inductive_row_equals_one_step_in_the_grown_graph():
    # directed base graph; new nodes only point at existing nodes, so adding their edges
    # leaves every old row unchanged and their own row is the one-step row
    base = synth.random_multigraph(60, 300, 2, True, True)
    g = oracle.build_from(base)
    T = oracle.propagate(g, oracle.init(g.ids, 24, 5), 3)
    rs = np.random.default_rng(0)
    new_ids = synth.node_ids(6, 999)
    u = np.repeat(new_ids, 5)
    b = g.ids[rs.integers(0, g.n, u.size)]
    w = rs.uniform(0.1, 2.0, u.size).astype(np.float32)
    ids, rows, dropped = oracle.inductive(g, T, u, b, w)
    grown = oracle.build_graph(np.concatenate([base.src, u]), np.concatenate([base.dst, b]),
                               np.concatenate([base.weights, w]), True)
    # previous iterate of the grown graph: old rows from T, new rows arbitrary
    pos_old = np.searchsorted(grown.ids, g.ids)
    Tg = np.random.default_rng(1).normal(size=(grown.n, 24))
    Tg[pos_old] = T
    want = oracle.step_rows(grown, Tg, np.searchsorted(grown.ids, ids))
    np.testing.assert_allclose(rows, want, atol=1e-14)
    assert dropped == 0


def test_inductive_merges_duplicates_and_drops_unknown_neighbours():
    e = synth.random_multigraph(30, 100, 3, True, False)
    g = oracle.build_from(e)
    T = oracle.init(g.ids, 8, 1)
    u = np.array([1, 1, 1, 2], np.uint64)
    b = np.array([g.ids[0], g.ids[0], g.ids[1], 424242], np.uint64)
    ids, rows, dropped = oracle.inductive(g, T, u, b)
    assert list(ids) == [1] and dropped == 1  # node 2 has no known neighbour
    np.testing.assert_allclose(rows[0], _unit((2 * T[0] + T[1]) / 3), atol=1e-15)


def test_single_chunk_is_the_plain_method():
    e = synth.random_multigraph(80, 400, 4, False, True)
    ids, T = oracle.chunked_embed(e.src, e.dst, e.weights, [0, e.num_edges], False, 16, 3, 7)
    g, T1 = oracle.embed(e, 16, 3, 7)
    assert np.array_equal(ids, g.ids)
    assert np.array_equal(T, T1)


def test_vertex_disjoint_chunks_are_independent_embeddings():
    a = synth.random_multigraph(30, 90, 5, True, False)
    b = synth.from_index_pairs([0, 1, 2], [1, 2, 0], True, seed=77)
    src = np.concatenate([a.src, b.src])
    dst = np.concatenate([a.dst, b.dst])
    ids, T = oracle.chunked_embed(src, dst, None, [0, a.num_edges, src.size], True, 8, 2, 0)
    for part in (a, b):
        g, Tp = oracle.embed(part, 8, 2, 0)
        np.testing.assert_allclose(T[np.searchsorted(ids, g.ids)], Tp, atol=1e-15)


def test_two_chunk_example_by_hand():
    # chunk 1: star h-a, h-b; chunk 2: edge h-c; one iteration (undirected)
    h, a, b, c = (np.uint64(x) for x in (10, 20, 30, 40))
    src = np.array([h, h, h], np.uint64)
    dst = np.array([a, b, c], np.uint64)
    ids, T = oracle.chunked_embed(src, dst, None, [0, 2, 3], False, 8, 1, 3)
    t0 = {int(x): np.array([oracle.init_value(3, int(x), j) for j in range(8)]) for x in (h, a, b, c)}
    # occurrences: h twice in chunk 1, once in chunk 2 -> weights 2/3, 1/3
    want_h = 2 / 3 * _unit((t0[20] + t0[30]) / 2) + 1 / 3 * _unit(t0[40])
    want = {10: want_h, 20: _unit(t0[10]), 30: _unit(t0[10]), 40: _unit(t0[10])}
    for i, x in enumerate(ids):
        np.testing.assert_allclose(T[i], want[int(x)], atol=1e-15)
