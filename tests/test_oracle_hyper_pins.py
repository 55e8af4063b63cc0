"""Pins of the oracle's identifier hash and hypergraph expansion (CPU only).

* XXH64 (Sec. 4.3: identifiers are hashed with xxhash into a small fixed-width format) is pinned
  by published reference outputs that cover the empty input, the one- to three-byte tail, the
  four-byte lane and the 32-byte stripes (tests/golden/xxh64_vectors.txt, cited there).  The
  eight-byte tail lane (inputs whose length mod 32 is 8 or more) has no published output here;
  it is checked only by the GPU kernel's bit-exact agreement with this independent restatement.
* Clique and star expansion (Sec. 3.2 "Hypergraph Expansion") are pinned by a hand example, the
  edge counts the paper states (k(k-1)/2 and k per hyperedge of width k), the star node's degree,
  and the embeddings they produce: one hyperedge expands to K_m (clique) or a star, whose
  embeddings have closed forms independent of the expansion code.
"""
import ast
import itertools
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _vectors():
    rows = []
    with open(os.path.join(GOLDEN, "xxh64_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            seed, digest, data = line.split(" ", 2)
            rows.append((int(seed), int(digest, 16), ast.literal_eval(data)))
    return rows


def test_xxh64_matches_published_outputs():
    vec = _vectors()
    assert len(vec) == 5
    for seed, digest, data in vec:
        assert oracle.xxh64(data, seed) == digest, data
    # the batch form agrees with the single form
    got = oracle.hash_strings([v[2] for v in vec if v[0] == 0], 0)
    assert [int(x) for x in got] == [v[1] for v in vec if v[0] == 0]


def test_xxh64_depends_on_every_byte_and_the_seed():
    base = bytes(range(70))
    h0 = oracle.xxh64(base, 7)
    for i in (0, 31, 32, 39, 40, 63, 69):
        flip = bytearray(base)
        flip[i] ^= 1
        assert oracle.xxh64(bytes(flip), 7) != h0
    assert oracle.xxh64(base, 8) != h0
    assert oracle.xxh64(base[:-1], 7) != h0  # the length is mixed in


def test_expansion_hand_example():
    ids = synth.node_ids(4, 0)
    a, b, c, s = (int(x) for x in np.sort(ids))
    members = np.array([c, a, b, a], np.uint64)  # a repeated member counts once
    hoff = np.array([0, 4], np.int64)
    src, dst = oracle.expand(members, hoff, "clique")
    assert list(zip(src.tolist(), dst.tolist())) == [(a, b), (a, c), (b, c)]
    src, dst = oracle.expand(members, hoff, "star", star_ids=np.array([s], np.uint64))
    assert list(zip(src.tolist(), dst.tolist())) == [(s, a), (s, b), (s, c)]
    src, dst = oracle.expand(members, hoff, "star")
    assert set(src.tolist()) == {oracle.star_node_id(0)}


def _random_hypergraph(H, n, kmax, seed):
    rs = np.random.default_rng(seed)
    widths = rs.integers(0, kmax + 1, H)
    hoff = np.concatenate([[0], np.cumsum(widths)]).astype(np.int64)
    ids = synth.node_ids(n, seed)
    members = ids[rs.integers(0, n, int(hoff[-1]))]
    return members, hoff


@pytest.mark.parametrize("seed", [0, 1])
def test_edge_counts_and_star_degrees(seed):
    members, hoff = _random_hypergraph(300, 200, 12, seed)
    k = np.array([len(set(members[hoff[h]:hoff[h + 1]].tolist())) for h in range(hoff.size - 1)])
    src, dst = oracle.expand(members, hoff, "clique")
    assert src.size == int((k * (k - 1) // 2).sum())  # k(k-1)/2 edges per hyperedge
    assert np.all(src < dst)  # pairs of distinct members, ascending ids
    src, dst = oracle.expand(members, hoff, "star")
    assert src.size == int(k.sum())  # k edges per hyperedge
    g = oracle.build_graph(src, dst, None, False)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    for h in range(hoff.size - 1):  # the star node's degree is the hyperedge's width
        if k[h]:
            assert g.deg[pos[oracle.star_node_id(h)]] == k[h]


def test_pair_multiplicity_counts_shared_hyperedges():
    # e_ab of the clique expansion = number of hyperedges holding both a and b
    members, hoff = _random_hypergraph(200, 30, 8, 3)
    src, dst = oracle.expand(members, hoff, "clique")
    g = oracle.build_graph(src, dst, None, False)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    shared = {}
    for h in range(hoff.size - 1):
        for u, v in itertools.combinations(sorted(set(members[hoff[h]:hoff[h + 1]].tolist())), 2):
            shared[(u, v)] = shared.get((u, v), 0) + 1
    for (u, v), cnt in shared.items():
        a, b = pos[u], pos[v]
        row = g.col[g.rowptr[a]:g.rowptr[a + 1]]
        k = g.rowptr[a] + int(np.searchsorted(row, b))
        assert g.col[k] == b and g.e[k] == cnt


def test_one_hyperedge_embeds_as_a_clique_or_a_star():
    m, d = 9, 16
    ids = synth.node_ids(m, 5)
    hoff = np.array([0, m], np.int64)
    # clique: K_m without self-loops, one step gives (S - T_i) / (m - 1), normalised
    src, dst = oracle.expand(ids, hoff, "clique")
    g = oracle.build_graph(src, dst, None, False)
    T0 = oracle.init(g.ids, d, 1)
    y = (T0.sum(0)[None, :] - T0) / (m - 1)
    want = y / np.linalg.norm(y, axis=1, keepdims=True)
    np.testing.assert_allclose(oracle.propagate(g, T0, 1), want, rtol=0, atol=1e-13)
    # star: leaves copy the star node's row, the star node takes the leaves' mean
    src, dst = oracle.expand(ids, hoff, "star")
    g = oracle.build_graph(src, dst, None, False)
    T0 = oracle.init(g.ids, d, 1)
    hub = int(np.searchsorted(g.ids, np.uint64(oracle.star_node_id(0))))
    T1 = oracle.propagate(g, T0, 1)
    leaves = [i for i in range(g.n) if i != hub]
    h = T0[hub] / np.linalg.norm(T0[hub])
    for i in leaves:
        np.testing.assert_allclose(T1[i], h, rtol=0, atol=1e-13)
    mean = T0[leaves].mean(0)
    np.testing.assert_allclose(T1[hub], mean / np.linalg.norm(mean), rtol=0, atol=1e-13)
