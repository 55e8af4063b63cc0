"""The allocation-free propagation step against the regular entry point (GPU).

cleora_propagate_noalloc exists for callers that may not let the library allocate device
memory (a framework allocator that owns all of HBM, a latency-critical loop that cannot pay
for cudaMalloc/cudaFree, a job that must not fail with out-of-memory halfway).  Here the
test owns every buffer: it reads the CSR and T_0 from a regular context, then runs two
allocation-free steps in a row and compares each with cleora_propagate's own iterations,
within the parity tolerances.  This file is collected last on purpose.
"""
import numpy as np
import pytest

import synth

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
BF16_TOL = 2e-2


def _bf16_to_f32(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32)


CASES = [
    # (graph, d, storage, split_len): split_len 256 forces rows into split chunks, which
    # use the shared scratch array's partial sums
    ("power_law", 128, "f32", 256),
    ("power_law", 64, "bf16", 0),
    ("weighted_directed", 96, "f32", 0),
    ("star", 32, "f32", 256),
    ("star", 256, "bf16", 300),
]


def _graph(name):
    if name == "power_law":
        return synth.SMALL.generate()
    if name == "weighted_directed":
        return synth.random_multigraph(3000, 20000, 8, True, True)
    return synth.star(20000, seed=3)


@pytest.mark.parametrize("name,d,storage,split_len", CASES)
def test_noalloc_two_steps_match_propagate(name, d, storage, split_len):
    import torch
    import paper_2102_02302_gb300 as pkg

    e = _graph(name)
    tdtype = torch.float32 if storage == "f32" else torch.int16
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        info = ctx.info()
        n, nnz = info["n"], info["nnz"]
        rowptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(max(nnz, 1), dtype=torch.int32, device="cuda")
        val = torch.empty(max(nnz, 1), dtype=torch.float32, device="cuda") if info["has_val"] else None
        torch.cuda.synchronize()
        pkg.cleora_get_csr(ctx.handle, rowptr, col, val)
        ctx.init(d, 5, storage)
        T0 = torch.empty((n, d), dtype=tdtype, device="cuda")
        pkg.cleora_get_embeddings(ctx.handle, T0, storage)
        ctx.sync()
        want = []
        for _ in range(2):
            ctx.propagate(1)
            want.append(ctx.embeddings(storage))
    torch.cuda.synchronize()

    T1 = torch.empty_like(T0)
    T2 = torch.empty_like(T0)
    pkg.cleora_propagate_noalloc(rowptr, col, val, n, nnz, T0, T1, d, storage, split_len)
    pkg.cleora_propagate_noalloc(rowptr, col, val, n, nnz, T1, T2, d, storage, split_len)
    torch.cuda.synchronize()
    for got_t, ref in zip((T1, T2), want):
        got = got_t.cpu().numpy()
        if storage == "f32":
            err = np.abs(got.astype(np.float64) - ref.astype(np.float64)).max()
            assert err <= F32_TOL, err
        else:
            g = _bf16_to_f32(got.view(np.uint16)).astype(np.float64)
            r = _bf16_to_f32(ref).astype(np.float64)
            assert np.abs(g - r).max() <= BF16_TOL
        assert np.isfinite(got.astype(np.float64)).all()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    import torch
    import paper_2102_02302_gb300 as pkg

    lim = pkg.cleora_noalloc_limits(1024)
    assert lim["scratch_bytes"] == 8_618_240 and lim["max_split_chunks"] == 2048
    dummy = torch.empty(8, dtype=torch.int64, device="cuda")
    t = torch.empty((4, 1024), dtype=torch.float32, device="cuda")
    nnz = 10_000_000  # needs split_len >= ceil(2 * nnz / 2048)
    with pytest.raises(pkg.CleoraError) as ex:
        pkg.cleora_propagate_noalloc(dummy, dummy, None, 4, nnz, t, t, 1024, "f32", 256)
    assert ex.value.status == pkg.CLEORA_ERR_INVALID_ARG
    with pytest.raises(pkg.CleoraError):
        pkg.cleora_propagate_noalloc(dummy, dummy, None, 4, 10, t, t, 2048, "f32", 0)
