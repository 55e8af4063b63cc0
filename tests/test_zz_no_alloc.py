"""The allocation-free propagation step against the regular entry point and the oracle (GPU).

cleora_propagate_noalloc exists for callers that may not let the library allocate device
memory (a framework allocator that owns all of HBM, a latency-critical loop that cannot pay
for cudaMalloc/cudaFree, a job that must not fail with out-of-memory halfway).  Here the
test owns every buffer: it reads the CSR and T_0 from a regular context, then runs two
allocation-free steps in a row and compares each with cleora_propagate's own iterations and
with the FP64 oracle, within the parity tolerances.  It also checks that the calls take no
device memory and that misaligned or overlapping buffers are refused before any launch.
This file is collected last on purpose.
"""
import numpy as np
import pytest

import oracle
import synth

pytestmark = pytest.mark.gpu

F32_TOL = 1e-5
BF16_TOL = 2e-2


def _bf16_to_f32(bits):
    return (bits.astype(np.uint32) << 16).view(np.float32)


def _bf16_round(x):
    b = np.ascontiguousarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    r = (((b + 0x7FFF + ((b >> 16) & 1)) >> 16) & 0xFFFF).astype(np.uint32)
    return (r << 16).view(np.float32).astype(np.float64)


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

    g = oracle.build_from(e)
    T0o = oracle.init(g.ids, d, 5)
    if storage == "bf16":
        T0o = _bf16_round(T0o)
    oracle_want = [oracle.propagate(g, T0o, k) for k in (1, 2)]

    T1 = torch.empty_like(T0)
    T2 = torch.empty_like(T0)
    pkg.cleora_propagate_noalloc(rowptr, col, val, n, nnz, T0, T1, d, storage, split_len)
    pkg.cleora_propagate_noalloc(rowptr, col, val, n, nnz, T1, T2, d, storage, split_len)
    torch.cuda.synchronize()
    for got_t, ref, ow in zip((T1, T2), want, oracle_want):
        got = got_t.cpu().numpy()
        if storage == "f32":
            gf = got.astype(np.float64)
            assert np.abs(gf - ref.astype(np.float64)).max() <= F32_TOL
            assert np.abs(gf - ow).max() <= F32_TOL
        else:
            gf = _bf16_to_f32(got.view(np.uint16)).astype(np.float64)
            r = _bf16_to_f32(ref).astype(np.float64)
            assert np.abs(gf - r).max() <= BF16_TOL
            assert np.abs(gf - ow).max() <= BF16_TOL
            cos = (gf * ow).sum(1) / (np.linalg.norm(gf, axis=1) * np.linalg.norm(ow, axis=1))
            assert cos.min() >= 0.999
        assert np.isfinite(gf).all()


def test_noalloc_takes_no_device_memory_and_refuses_bad_views():
    import torch
    import paper_2102_02302_gb300 as pkg

    e = synth.star(20000, seed=3)
    d = 64
    with pkg.Context(0) as ctx:
        ctx.graph_build(e.src, e.dst, e.weights, e.directed)
        info = ctx.info()
        n, nnz = info["n"], info["nnz"]
        rowptr = torch.empty(n + 1, dtype=torch.int64, device="cuda")
        col = torch.empty(nnz, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        pkg.cleora_get_csr(ctx.handle, rowptr, col)
        ctx.init(d, 1, "bf16")
        T0 = torch.empty((n, d), dtype=torch.int16, device="cuda")
        pkg.cleora_get_embeddings(ctx.handle, T0, "bf16")
        ctx.sync()
    torch.cuda.synchronize()
    T1 = torch.empty_like(T0)
    # the first call on the device looks up the scratch array and loads the kernels
    pkg.cleora_propagate_noalloc(rowptr, col, None, n, nnz, T0, T1, d, "bf16", 256)
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    alloc0, reserved0 = torch.cuda.memory_allocated(), torch.cuda.memory_reserved()
    for _ in range(3):
        pkg.cleora_propagate_noalloc(rowptr, col, None, n, nnz, T0, T1, d, "bf16", 256)
        pkg.cleora_propagate_noalloc(rowptr, col, None, n, nnz, T1, T0, d, "bf16", 256)
    torch.cuda.synchronize()
    assert torch.cuda.mem_get_info()[0] == free0
    assert torch.cuda.memory_allocated() == alloc0 and torch.cuda.memory_reserved() == reserved0
    # a view 8 bytes into T (BF16, 4 elements) is not 16-byte aligned; overlapping input and
    # output buffers are refused as well; nothing is launched for either
    flat = T0.view(-1)
    shifted = flat[4:4 + (n - 1) * d].view(n - 1, d)
    out = torch.empty((n - 1, d), dtype=torch.int16, device="cuda")
    with pytest.raises(pkg.CleoraError) as ex:
        pkg.cleora_propagate_noalloc(rowptr, col, None, n - 1, nnz, shifted, out, d, "bf16", 256)
    assert ex.value.status == pkg.CLEORA_ERR_INVALID_ARG
    with pytest.raises(pkg.CleoraError) as ex:
        pkg.cleora_propagate_noalloc(rowptr, col, None, n, nnz, T0, T0, d, "bf16", 256)
    assert ex.value.status == pkg.CLEORA_ERR_INVALID_ARG
    torch.cuda.synchronize()


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
