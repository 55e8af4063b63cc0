"""Generator module checks (CPU): published splitmix64 outputs, determinism, shapes."""
import os

import numpy as np

import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_generator_mix_matches_published_outputs():
    g = 0x9E3779B97F4A7C15
    with open(os.path.join(GOLDEN, "splitmix64_vectors.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            seed, *outs = [int(x, 0) for x in line.split()]
            states = (np.uint64(seed) + np.arange(5, dtype=np.uint64) * np.uint64(g))
            assert [int(x) for x in synth.mix(states)] == outs
            assert [synth.mix_int((seed + k * g) % 2**64) for k in range(5)] == outs


def test_node_ids_are_distinct():
    ids = synth.node_ids(200_000, 5)
    assert np.unique(ids).size == ids.size


def test_undirected_power_law_is_simple_and_deterministic():
    a = synth.chung_lu_undirected(5000, 20000, 2.1, 3, 500.0)
    b = synth.chung_lu_undirected(5000, 20000, 2.1, 3, 500.0)
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    assert a.num_edges >= 20000
    assert np.all(a.src != a.dst)
    key = np.minimum(a.src, a.dst).astype(object) * 2**64 + np.maximum(a.src, a.dst).astype(object)
    assert len(set(key.tolist())) == a.num_edges


def test_thresholds_follow_the_weights():
    thr = synth.cdf_thresholds(1000, 2.0, 5.0)
    assert thr[-1] == 2**53 and np.all(np.diff(thr.astype(np.int64)) >= 0)
    draws = synth.rng(0, 1, np.arange(400_000, dtype=np.uint64))
    idx = synth.sample_nodes(thr, draws)
    w = (np.arange(1000) + 5.0) ** -1.0
    p = w / w.sum()
    counts = np.bincount(idx, minlength=1000)
    assert abs(counts[0] / 400_000 - p[0]) < 5 * np.sqrt(p[0] / 400_000)


def test_batch_specs_cover_the_ranges():
    specs = synth.batch_specs(256, seed=0)
    ns = np.array([s.n for s in specs])
    assert ns.min() >= 50 and ns.max() <= 50_000
    assert {s.d for s in specs} == {64, 128, 256}
    assert {s.iters for s in specs} == {3, 4, 5}
    assert 0.3 < np.mean([s.directed for s in specs]) < 0.7
