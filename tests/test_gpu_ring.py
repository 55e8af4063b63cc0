"""Shared-memory ring kernel (option staging = 2: one bulk copy per gathered row; 3: TMA tensor
gathers of 4 rows): gathered rows of T reach the sums through a warp-private ring, with a
per-entry hot bitmap for the L2 policy instead of the hot-first row reorder.  Only the summation order differs from the register kernel, so

  * results stay within the FP32 / BF16 tolerances of the FP64 oracle (Algorithm 1) for every
    shape the ring covers (FP32 d = 64 and 128, BF16 d = 128 and 256), weighted and unit
    graphs, split rows, sinks, 2 to 4 stages, with and without a hot bitmap;
  * results are deterministic and propagate(a) + propagate(b) = propagate(a + b) bit for bit;
  * cleora_get_csr still returns each row in ascending column order;
  * a wait that runs out (test hook) is reported as CLEORA_ERR_DEVICE and leaves the context
    usable.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
BF16_TOL = 2e-2


def _bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32)
    return (r << 16).view(np.float32).astype(np.float64)


GRAPHS = {
    "directed_weighted": lambda: synth.chung_lu_directed(30_000, 300_000, 2.1, 5, 5_000.0, "lognormal"),
    "undirected_unit": lambda: synth.SMALL.generate(),
    "star": lambda: synth.star(20_000, seed=3),
    "sparse_sinks": lambda: synth.random_multigraph(5000, 6000, 9, True, False),
}
_cache = {}


def _graph(name):
    if name not in _cache:
        e = GRAPHS[name]()
        _cache[name] = (e, oracle.build_from(e))
    return _cache[name]


def _run(e, d, storage, opts, iters=4, chunks=(4,), staging=2):
    import paper_2102_02302_gb300 as pkg
    with pkg.Context(0) as ctx:
        ctx.set_option("staging", staging)
        for k, v in opts.items():
            ctx.set_option(k, v)
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        ctx.init(d, 0, storage)
        hot = ctx.hot_entries()
        n = ctx.info()["n"]
        outs = []
        for c in chunks:
            out = np.empty((n, d), np.float32)
            ctx.propagate(c, out)
            ctx.sync()
            outs.append(out)
        csr = ctx.csr()
        return outs, hot, csr


def _check(g, out, d, storage, iters=4):
    T0 = oracle.init(g.ids, d, 0)
    if storage == "f32":
        want = oracle.propagate(g, T0, iters)
        err = np.abs(out - want).max()
        assert err <= F32_TOL, err
    else:
        want = oracle.propagate(g, _bf16_round(T0), iters)
        err = np.abs(out - want).max()
        assert err <= BF16_TOL, err
        cos = (out * want).sum(1) / (np.linalg.norm(out, axis=1) * np.linalg.norm(want, axis=1))
        assert cos.min() >= 0.999


SHAPES = [(64, "f32"), (128, "f32"), (128, "bf16"), (256, "bf16")]


@pytest.mark.parametrize("staging", [2, 3])
@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("d,storage", SHAPES)
def test_ring_matches_oracle(name, d, storage, staging):
    e, g = _graph(name)
    opts = {"split_len": 256} if name in ("star", "undirected_unit") else {}
    (out,), hot, csr = _run(e, d, storage, opts, staging=staging)
    assert hot == 0  # T fits in L2: no hot bitmap
    assert np.array_equal(csr["rowptr"], g.rowptr) and np.array_equal(csr["col"], g.col)
    _check(g, out, d, storage)


@pytest.mark.parametrize("staging", [2, 3])
@pytest.mark.parametrize("stages", [2, 3, 4])
@pytest.mark.parametrize("d,storage", [(128, "f32"), (128, "bf16")])
def test_ring_stages_and_hot_bitmap(stages, d, storage, staging):
    e, g = _graph("directed_weighted")
    opts = {"ring_stages": stages, "hot_bytes": 256 << 10, "split_len": 512}
    (out,), hot, csr = _run(e, d, storage, opts, staging=staging)
    assert 0 < hot < g.nnz  # bitmap marks the entries of the hottest rows
    assert np.array_equal(csr["col"], g.col)  # rows keep ascending column order
    assert np.array_equal(csr["val"].view(np.uint32), g.val32.view(np.uint32))
    _check(g, out, d, storage)


def test_hot_set_is_the_exact_top_rows():
    # The hot rows are the highest in-degrees that fit in the budget of R rows: every row whose
    # in-degree is above the R-th largest is hot, and the marked entries never exceed those of
    # the R most-referenced rows (rows tied at the boundary count may be left out).
    e, g = _graph("directed_weighted")
    d, budget = 128, 256 << 10
    (_,), hot, _ = _run(e, d, "f32", {"hot_bytes": budget})
    indeg = np.bincount(g.col, minlength=g.n)
    rows = budget // (d * 4)
    order = np.sort(indeg)[::-1]
    best = int(order[:rows].sum())
    above = int(indeg[indeg > order[rows - 1]].sum())
    assert above <= hot <= best


@pytest.mark.parametrize("staging", [2, 3])
def test_ring_deterministic_and_resumable(staging):
    e, g = _graph("undirected_unit")
    opts = {"hot_bytes": 64 << 10, "split_len": 256}
    outs, _, _ = _run(e, 128, "bf16", opts, chunks=(2, 2), staging=staging)
    outs4, _, _ = _run(e, 128, "bf16", opts, chunks=(4,), staging=staging)
    again, _, _ = _run(e, 128, "bf16", opts, chunks=(4,), staging=staging)
    assert np.array_equal(outs[1].view(np.uint32), outs4[0].view(np.uint32))
    assert np.array_equal(again[0].view(np.uint32), outs4[0].view(np.uint32))
    if staging == 3:  # both issue modes fill the same slots: the same bits
        bulk, _, _ = _run(e, 128, "bf16", opts, chunks=(4,), staging=2)
        assert np.array_equal(bulk[0].view(np.uint32), outs4[0].view(np.uint32))


def test_ring_and_register_kernels_agree():
    import paper_2102_02302_gb300 as pkg
    e, g = _graph("directed_weighted")
    res = {}
    for staging in (1, 2):
        with pkg.Context(0) as ctx:
            ctx.set_option("staging", staging)
            ctx.graph_build(e.src, e.dst, e.weights, e.directed)
            ctx.init(128, 0, "f32")
            out = np.empty((g.n, 128), np.float32)
            ctx.propagate(3, out)
            ctx.sync()
            res[staging] = out
    assert np.abs(res[1] - res[2]).max() <= 2e-6


@pytest.mark.parametrize("staging", [2, 3])
def test_ring_wait_that_runs_out_is_reported_and_context_stays_usable(staging):
    import paper_2102_02302_gb300 as pkg
    e, g = _graph("undirected_unit")
    with pkg.Context(0) as ctx:
        ctx.set_option("staging", staging)
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        ctx.init(128, 0, "f32")
        ctx.set_option("test_ring_wait", 1)
        ctx.propagate(1)
        with pytest.raises(pkg.CleoraError) as ex:
            ctx.sync()
        assert ex.value.status == pkg.CLEORA_ERR_DEVICE
        ctx.set_option("test_ring_wait", 0)
        ctx.init(128, 0, "f32")
        out = np.empty((g.n, 128), np.float32)
        ctx.propagate(4, out)
        ctx.sync()
    _check(g, out, 128, "f32")
