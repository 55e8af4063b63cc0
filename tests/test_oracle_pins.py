"""Pins for the FP64 oracle, against things other than itself (CPU only).

Each check is tied to what Sec. 3.2 / Algorithm 1 of arXiv 2102.02302 fixes:
  * M_ab = e_ab / deg(v_a), e_ab = edge count or weight sum, undirected edges both ways
    (Sec. 3.2 "Embedding", Sec. 4.5) -> brute-force dense D^-1 A product;
  * rows are L2-normalised after every multiplication (Algorithm 1) -> unit norms;
  * M is row-stochastic -> constant columns are fixed points; cliques, stars, K_{m,k},
    regular graphs have closed forms;
  * a leaf takes its neighbour's previous row (Sec. 6.2, homophily discussion);
  * too many iterations collapse all rows to one vector (Sec. 6.1);
  * T0 ~ U(-1, 1) (Sec. 3.2) through splitmix64, pinned by its published outputs.
"""
import os

import numpy as np
import pytest

import oracle
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden_splitmix():
    rows = []
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            parts = line.split()
            rows.append((int(parts[0], 0), [int(x, 0) for x in parts[1:]]))
    return rows


# --------------------------------------------------------------------------------------
# Init hash (Sec. 3.2: T0 ~ U(-1, 1))
# --------------------------------------------------------------------------------------

def test_mix_matches_published_splitmix64_outputs():
    g = 0x9E3779B97F4A7C15
    for seed, outs in _golden_splitmix():
        for k, want in enumerate(outs):
            assert oracle.mix((seed + k * g) % (1 << 64)) == want


def test_init_value_is_the_documented_chain_of_mixes():
    # The chain is checked against the generator module's independent mix (itself pinned
    # to the same published outputs in test_synth.py).
    rs = np.random.default_rng(1)
    for _ in range(200):
        seed = int(rs.integers(0, 2**63)) * 2 + int(rs.integers(0, 2))
        nid = int(rs.integers(0, 2**63)) * 2 + 1
        j = int(rs.integers(0, 4096))
        h = synth.mix_int(synth.mix_int(synth.mix_int(seed) ^ nid) ^ j)
        want = 2.0 * ((h >> 40) * 2.0 ** -24) - 1.0
        assert oracle.init_value(seed, nid, j) == want


def test_init_statistics_are_uniform_minus1_1():
    ids = synth.node_ids(4000, 7)
    T0 = oracle.init(ids, 64, seed=123)
    x = T0.ravel()
    assert x.min() >= -1.0 and x.max() < 1.0
    assert abs(x.mean()) < 0.01
    assert abs(x.var() - 1.0 / 3.0) < 0.005
    # Kolmogorov-Smirnov distance to U(-1, 1): 5-sigma bound for 256k samples
    xs = np.sort(x)
    cdf = (xs + 1.0) / 2.0
    k = np.arange(1, xs.size + 1) / xs.size
    ks = max(np.max(k - cdf), np.max(cdf - (k - 1.0 / xs.size)))
    assert ks < 5.0 / np.sqrt(xs.size)
    # values are exact multiples of 2^-23 in [-1, 1 - 2^-23]
    assert np.all(np.round(x * 2**23) == x * 2**23)


def test_init_depends_on_external_id_not_position():
    ids = synth.node_ids(50, 3)
    a = oracle.init(ids, 16, 9)
    b = oracle.init(ids[::-1].copy(), 16, 9)
    assert np.array_equal(a, b[::-1])


# --------------------------------------------------------------------------------------
# Graph build and M (Sec. 3.2 "Embedding")
# --------------------------------------------------------------------------------------

def _dense_reference(edges):
    """Brute force: adjacency dict -> dense A -> D^-1 A, ids ordered by np.unique."""
    ids = np.unique(np.concatenate([edges.src, edges.dst]))
    pos = {int(x): i for i, x in enumerate(ids)}
    n = ids.size
    A = np.zeros((n, n))
    w = edges.weights if edges.weights is not None else np.ones(edges.num_edges, np.float32)
    for s, t, wk in zip(edges.src, edges.dst, w):
        a, b = pos[int(s)], pos[int(t)]
        A[a, b] += float(wk)
        if not edges.directed and a != b:
            A[b, a] += float(wk)
    deg = A.sum(axis=1)
    M = np.divide(A, deg[:, None], out=np.zeros_like(A), where=deg[:, None] > 0)
    return ids, A, deg, M


def _dense_iterate(M, deg, T, iters):
    for _ in range(iters):
        Y = M @ T
        Y[deg == 0] = T[deg == 0]
        nrm = np.linalg.norm(Y, axis=1, keepdims=True)
        T = np.divide(Y, nrm, out=np.zeros_like(Y), where=nrm > 0)
    return T


TINY_CASES = [
    dict(n=12, E=30, directed=False, weighted=False),
    dict(n=12, E=30, directed=True, weighted=False),
    dict(n=20, E=80, directed=False, weighted=True),
    dict(n=20, E=80, directed=True, weighted=True),
    dict(n=40, E=60, directed=True, weighted=True),   # sparse: many sinks
    dict(n=64, E=400, directed=False, weighted=False),
]


@pytest.mark.parametrize("case", TINY_CASES)
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_oracle_matches_brute_force_dense_product(case, seed):
    e = synth.random_multigraph(case["n"], case["E"], seed, case["directed"], case["weighted"])
    ids, A, deg, M = _dense_reference(e)
    g = oracle.build_from(e)
    assert np.array_equal(g.ids, ids)
    np.testing.assert_allclose(g.dense_m(), M, rtol=0, atol=1e-15)
    np.testing.assert_allclose(g.deg, deg, rtol=1e-15, atol=0)
    # structure: columns strictly ascending within each row
    for a in range(g.n):
        c = g.col[g.rowptr[a]:g.rowptr[a + 1]]
        assert np.all(np.diff(c) > 0)
    T0 = oracle.init(g.ids, 24, seed)
    for iters in (1, 2, 4):
        want = _dense_iterate(M, deg, T0, iters)
        got = oracle.propagate(g, T0, iters)
        np.testing.assert_allclose(got, want, rtol=0, atol=1e-13)


def test_unweighted_has_no_values_unless_duplicates():
    simple = synth.chung_lu_undirected(300, 900, 2.1, 0, 50.0)
    assert not oracle.build_from(simple).has_val
    dup = synth.from_index_pairs([0, 0, 1], [1, 1, 2], True)
    g = oracle.build_from(dup)
    assert g.has_val
    assert sorted(g.e) == [1.0, 2.0]  # rows follow ascending external id


def test_undirected_self_loop_counts_once():
    e = synth.from_index_pairs([0, 0], [0, 1], False)
    g = oracle.build_from(e)
    # node 0: self-loop (1) + edge to 1 (1) -> deg 2; node 1: edge to 0 -> deg 1
    pos = {int(x): i for i, x in enumerate(g.ids)}
    ids = synth.node_ids(2, 0)
    assert g.deg[pos[int(ids[0])]] == 2.0 and g.deg[pos[int(ids[1])]] == 1.0
    assert list(g.e) == [1.0, 1.0, 1.0]


def test_duplicate_edge_equals_one_edge_of_double_weight():
    a = synth.from_index_pairs([0, 0, 1, 2], [1, 1, 2, 0], True, weights=[0.5, 0.5, 1, 1])
    b = synth.from_index_pairs([0, 1, 2], [1, 2, 0], True, weights=[1.0, 1, 1])
    ga, gb = oracle.build_from(a), oracle.build_from(b)
    assert np.array_equal(ga.dense_m(), gb.dense_m())


def _rn32(x):
    """The float32 nearest to the rational x, ties to even: one rounding of the exact
    value (float(x) is within one float32 step of it; the three neighbours are compared
    exactly)."""
    from fractions import Fraction
    c = np.float32(float(x))
    best = None
    for cand in (np.nextafter(c, np.float32(-np.inf)), c, np.nextafter(c, np.float32(np.inf))):
        key = (abs(Fraction(float(cand)) - x), int(np.array(cand).view(np.uint32)) & 1)
        if best is None or key < best[0]:
            best = (key, cand)
    return best[1]


def test_stored_fp32_values_round_the_exact_transition_probabilities_once():
    # The compact store of M (Sec. 3.2: M_ab = e_ab / deg(v_a); the builder keeps FP32
    # values) rounds the exact ratio once, val = fp32(e_ab / deg_a), and keeps
    # inv_deg = 1.0f / fp32(deg_a) (IEEE division, correctly rounded).  Expected values come
    # from exact rationals of a hand-built adjacency, not from the oracle's own arithmetic.
    # The weights make the tempting variants differ: fp32(e)/fp32(deg) for the values and
    # fp32(1/deg) for the inverse degree.
    from fractions import Fraction
    w = [0.7, 0.1, 1.1, 0.1, 0.05, 1.0, 0.3, 2.9, 2.9]
    src = [0, 0, 0, 0, 0, 1, 1, 2, 2]
    dst = [1, 2, 2, 3, 3, 0, 0, 2, 1]
    e = synth.from_index_pairs(src, dst, True, weights=w)
    g = oracle.build_from(e)
    ids = synth.node_ids(4, 0)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    adj = {}
    for s, t, wk in zip(src, dst, np.asarray(w, np.float32)):
        key = (pos[int(ids[s])], pos[int(ids[t])])
        adj[key] = adj.get(key, Fraction(0)) + Fraction(float(wk))
    assert g.has_val
    split_val = split_inv = False
    for a in range(g.n):
        row = {b: x for (r, b), x in adj.items() if r == a}
        deg = sum(row.values(), Fraction(0))
        if deg == 0:
            assert g.inv_deg32[a] == 0.0 and g.rowptr[a] == g.rowptr[a + 1]
            continue
        assert sum((x / deg for x in row.values()), Fraction(0)) == 1  # row-stochastic
        deg32 = np.float32(float(deg))
        want_inv = _rn32(Fraction(1) / Fraction(float(deg32)))
        assert g.inv_deg32[a].view(np.uint32) == want_inv.view(np.uint32)
        split_inv |= want_inv != _rn32(Fraction(1) / deg)
        for k in range(g.rowptr[a], g.rowptr[a + 1]):
            b = int(g.col[k])
            want = _rn32(row[b] / deg)
            assert g.val32[k].view(np.uint32) == want.view(np.uint32), (a, b)
            split_val |= want != np.float32(np.float32(float(row[b])) / deg32)
    assert split_val and split_inv  # the graph tells the rounding rules apart


@pytest.mark.parametrize("c", [4.0, 3.0, 0.125])
def test_scaling_all_weights_leaves_m_unchanged(c):
    e = synth.random_multigraph(30, 120, 5, True, True)
    g1 = oracle.build_from(e)
    e.weights = (e.weights * np.float32(c)).astype(np.float32)
    g2 = oracle.build_from(e)
    # powers of two scale float32 inputs exactly; otherwise each input weight carries one
    # float32 rounding (relative 2^-24), which bounds the change of M
    exact = float(np.log2(c)).is_integer()
    np.testing.assert_allclose(g2.dense_m(), g1.dense_m(), rtol=1e-15 if exact else 2.5e-7,
                               atol=1e-16)


@pytest.mark.parametrize("weighted", [False, True])
def test_edge_order_does_not_change_csr_or_result(weighted):
    e = synth.random_multigraph(50, 300, 11, False, weighted)
    g1 = oracle.build_from(e)
    perm = np.random.default_rng(0).permutation(e.num_edges)
    flip = np.random.default_rng(1).random(e.num_edges) < 0.5
    src = np.where(flip, e.dst, e.src)[perm]
    dst = np.where(flip, e.src, e.dst)[perm]
    w = None if e.weights is None else e.weights[perm]
    g2 = oracle.build_graph(src, dst, w, False)
    for f in ("ids", "rowptr", "col", "e", "deg"):
        assert np.array_equal(getattr(g1, f), getattr(g2, f)), f
    T0 = oracle.init(g1.ids, 16, 0)
    assert np.array_equal(oracle.propagate(g1, T0, 3), oracle.propagate(g2, T0, 3))


def test_invalid_weights_rejected_and_empty_graph():
    e = synth.from_index_pairs([0, 1], [1, 2], True, weights=[1.0, 0.0])
    with pytest.raises(oracle.OracleError):
        oracle.build_from(e)
    for bad in (-1.0, np.nan, np.inf):
        e.weights = np.array([1.0, bad], np.float32)
        with pytest.raises(oracle.OracleError):
            oracle.build_from(e)
    g = oracle.build_graph(np.zeros(0, np.uint64), np.zeros(0, np.uint64))
    assert g.n == 0 and g.nnz == 0


# --------------------------------------------------------------------------------------
# Iteration invariants and closed forms (Algorithm 1)
# --------------------------------------------------------------------------------------

def _unit(v):
    return v / np.linalg.norm(v, axis=-1, keepdims=True)


@pytest.mark.parametrize("directed", [False, True])
def test_rows_have_unit_norm_after_every_iteration(directed):
    e = synth.random_multigraph(200, 900, 4, directed, True)
    g = oracle.build_from(e)
    T = oracle.init(g.ids, 32, 1)
    for _ in range(5):
        T = oracle.propagate(g, T, 1)
        np.testing.assert_allclose(np.linalg.norm(T, axis=1), 1.0, atol=1e-12)


def test_constant_columns_are_a_fixed_point():
    e = synth.random_multigraph(100, 500, 2, False, True)  # undirected: no sinks
    g = oracle.build_from(e)
    v = np.linspace(-1.0, 0.7, 48)
    T0 = np.tile(v, (g.n, 1))
    for iters in (1, 3):
        T = oracle.propagate(g, T0, iters)
        np.testing.assert_allclose(T, np.tile(_unit(v), (g.n, 1)), atol=1e-14)


def test_leaf_takes_its_neighbours_previous_row():
    # path 0-1-2-3 plus a leaf 4 hanging off 2
    e = synth.from_index_pairs([0, 1, 2, 2], [1, 2, 3, 4], False)
    g = oracle.build_from(e)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    leaf, hub = pos[int(e.dst[3])], pos[int(e.src[3])]
    T0 = oracle.init(g.ids, 16, 5)
    prev = T0
    for k in range(1, 5):
        cur = oracle.propagate(g, prev, 1)
        np.testing.assert_allclose(cur[leaf], _unit(prev[hub]), atol=1e-15)
        prev = cur


def test_disjoint_cliques_with_self_loops_reach_their_mean_in_one_step():
    sizes = [3, 5, 8]
    e = synth.disjoint_cliques(sizes, seed=2, self_loops=True)
    g = oracle.build_from(e)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    ids_by_node = synth.node_ids(sum(sizes), 2)
    T0 = oracle.init(g.ids, 32, 8)
    off = 0
    T1 = oracle.propagate(g, T0, 1)
    T4 = oracle.propagate(g, T0, 4)
    for m in sizes:
        rows = [pos[int(ids_by_node[off + i])] for i in range(m)]
        want = _unit(T0[rows].mean(axis=0))
        for r in rows:
            np.testing.assert_allclose(T1[r], want, atol=1e-14)
            np.testing.assert_allclose(T4[r], want, atol=1e-14)
        off += m


def test_clique_without_self_loops_averages_the_others():
    m = 7
    e = synth.disjoint_cliques([m], seed=4, self_loops=False)
    g = oracle.build_from(e)
    T0 = oracle.init(g.ids, 20, 3)
    S = T0.sum(axis=0)
    T1 = oracle.propagate(g, T0, 1)
    for i in range(m):
        np.testing.assert_allclose(T1[i], _unit((S - T0[i]) / (m - 1)), atol=1e-14)


def test_star_leaves_copy_the_hub_and_hub_averages_leaves():
    e = synth.star(9, seed=6)
    g = oracle.build_from(e)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    ids = synth.node_ids(10, 6)
    hub = pos[int(ids[0])]
    leaves = [pos[int(ids[k])] for k in range(1, 10)]
    T0 = oracle.init(g.ids, 16, 2)
    T1 = oracle.propagate(g, T0, 1)
    np.testing.assert_allclose(T1[hub], _unit(T0[leaves].mean(axis=0)), atol=1e-14)
    for r in leaves:
        np.testing.assert_allclose(T1[r], _unit(T0[hub]), atol=1e-15)


def test_complete_bipartite_sides_take_the_other_sides_mean():
    m, k = 4, 6
    e = synth.complete_bipartite(m, k, seed=1)
    g = oracle.build_from(e)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    ids = synth.node_ids(m + k, 1)
    A = [pos[int(ids[i])] for i in range(m)]
    B = [pos[int(ids[m + j])] for j in range(k)]
    T0 = oracle.init(g.ids, 16, 4)
    T1 = oracle.propagate(g, T0, 1)
    for r in A:
        np.testing.assert_allclose(T1[r], _unit(T0[B].mean(axis=0)), atol=1e-14)
    for r in B:
        np.testing.assert_allclose(T1[r], _unit(T0[A].mean(axis=0)), atol=1e-14)


def test_regular_graph_keeps_equal_rows():
    e = synth.circulant_regular(30, 3, seed=0)
    g = oracle.build_from(e)
    assert np.all(g.deg == 6.0)
    v = np.arange(1.0, 17.0)
    T = oracle.propagate(g, np.tile(v, (g.n, 1)), 3)
    np.testing.assert_allclose(T, np.tile(_unit(v), (g.n, 1)), atol=1e-14)


def test_many_iterations_collapse_rows():
    # connected, non-bipartite (odd cycle plus chords): rows converge to one vector
    e = synth.circulant_regular(41, 2, seed=3)
    g = oracle.build_from(e)
    T0 = oracle.init(g.ids, 16, 0)
    T = oracle.propagate(g, T0, 800)
    cos = T @ T[0]
    assert cos.min() > 0.999
    T4 = oracle.propagate(g, T0, 4)
    assert (T4 @ T4[0]).min() < 0.9


def test_sink_keeps_its_row_renormalised_and_step_rows_agrees():
    e = synth.from_index_pairs([0, 1, 2], [1, 2, 3], True)  # node 3 is a sink
    g = oracle.build_from(e)
    pos = {int(x): i for i, x in enumerate(g.ids)}
    sink = pos[int(synth.node_ids(4, 0)[3])]
    T0 = oracle.init(g.ids, 8, 1)
    T1 = oracle.propagate(g, T0, 1)
    np.testing.assert_allclose(T1[sink], _unit(T0[sink]), atol=1e-15)
    rows = np.array([3, 0, 2], np.int64)
    np.testing.assert_array_equal(oracle.step_rows(g, T0, rows), T1[rows])


@pytest.mark.parametrize("weighted,directed", [(False, False), (True, True), (False, True)])
def test_step_over_an_external_csr_equals_the_oracle_step(weighted, directed):
    # The one-step routine for graphs too large to build here takes the CSR from outside;
    # fed the oracle's own CSR (and an FP32-exact previous iterate) it must reproduce the
    # oracle's step bit for bit, sinks and duplicate edges included.
    e = synth.random_multigraph(200, 1500, 4, directed, weighted)
    g = oracle.build_from(e)
    T = oracle.init(g.ids, 24, 3)  # exact in FP32
    rows = np.array([0, g.n - 1, 5, 17, 5, 100], np.int64)
    want = oracle.step_rows(g, T, rows)
    ev = g.e if g.has_val else None
    got = oracle.step_csr_rows(g.rowptr, g.col, ev, T.astype(np.float32), rows)
    assert np.array_equal(got, want)
    with pytest.raises(oracle.OracleError):
        oracle.step_csr_rows(g.rowptr, g.col, ev, T.astype(np.float32), np.array([g.n]))


def test_power_law_small_case_sanity():
    e = synth.SMALL.generate()
    g = oracle.build_from(e)
    assert 45_000 <= e.num_edges <= 60_000
    assert g.nnz == 2 * e.num_edges  # simple undirected graph: both directions, no loops
    assert not g.has_val
    deg = np.diff(g.rowptr)
    assert deg.max() > 300  # heavy tail
    assert np.array_equal(g.deg, deg.astype(np.float64))
