"""Thin ctypes binding of ``libcleora.so`` (include/cleora.h), same names as the C ABI.

Only argument marshalling lives here: every step of the method runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host) or torch tensors (host or CUDA); 64-bit ids may
be passed as uint64 or int64 (same bits).  There is no CPU fallback: if the library cannot be
built or loaded, importing this module's functions raises.
"""
from __future__ import annotations

import ctypes
import os
import threading

import numpy as np

from . import build_native

_P = ctypes.c_void_p
_I64 = ctypes.c_int64
_lib = None
_lock = threading.Lock()

CLEORA_OK = 0
CLEORA_ERR_INVALID_ARG = -1
CLEORA_ERR_OOM = -2
CLEORA_ERR_CUDA = -3
CLEORA_ERR_STATE = -4
CLEORA_ERR_TIMEOUT = -5
CLEORA_ERR_REJECTED = -6
CLEORA_ERR_DEVICE = -7
CLEORA_ERR_CANCELLED = -8

CLEORA_F32 = 0
CLEORA_BF16 = 1
DTYPES = {"f32": CLEORA_F32, "float32": CLEORA_F32, "bf16": CLEORA_BF16, "bfloat16": CLEORA_BF16}

OPTIONS = {"vec_bytes": 0, "row_mode": 1, "split_len": 2, "task_nnz": 3, "blocks_per_sm": 4,
           "hot_bytes": 5, "id_slots": 6, "staging": 7, "ring_stages": 8,
           "test_ring_wait": 9, "chunk_bytes": 10}

# Every symbol include/cleora.h declares: name -> (restype, argtypes)
SIGNATURES = {
    "cleora_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P]),
    "cleora_destroy": (None, [_P]),
    "cleora_last_error": (ctypes.c_char_p, [_P]),
    "cleora_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "cleora_sync": (ctypes.c_int, [_P]),
    "cleora_graph_build": (ctypes.c_int, [_P, _P, _P, _P, _I64, ctypes.c_int, ctypes.c_int]),
    "cleora_num_nodes": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "cleora_num_entries": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "cleora_graph_info": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                         ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64)]),
    "cleora_node_ids": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "cleora_get_csr": (ctypes.c_int, [_P, _P, _P, _P, _P, _P, ctypes.c_int]),
    "cleora_init": (ctypes.c_int, [_P, ctypes.c_int, ctypes.c_uint64, ctypes.c_int]),
    "cleora_propagate": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "cleora_iteration": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int)]),
    "cleora_get_embeddings": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int]),
    "cleora_set_embeddings": (ctypes.c_int, [_P, _P, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
    "cleora_set_option": (ctypes.c_int, [_P, ctypes.c_int, _I64]),
    "cleora_get_option": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64)]),
    "cleora_launch_count": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "cleora_hot_entries": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "cleora_inductive": (ctypes.c_int, [_P, _P, _P, _P, _I64, ctypes.c_int, _P, _P, _I64,
                                        ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.c_int]),
    "cleora_chunked_embed": (ctypes.c_int, [_P, _P, _P, _P, _P, ctypes.c_int, ctypes.c_int,
                                            ctypes.c_int, ctypes.c_int, ctypes.c_uint64, ctypes.c_int,
                                            ctypes.c_int, _P, _P, _I64, ctypes.POINTER(_I64),
                                            ctypes.c_int]),
    "cleora_hash_ids": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_uint64, _P, ctypes.c_int, ctypes.c_int]),
    "cleora_expand_hypergraph": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, _P, ctypes.c_int, _P, _P, _I64,
                                                ctypes.POINTER(_I64), ctypes.c_int]),
    "cleora_hypergraph_build": (ctypes.c_int, [_P, _P, _P, _I64, ctypes.c_int, _P, ctypes.c_int,
                                               ctypes.POINTER(_I64)]),
    "cleora_chunked_info": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(_I64)]),
    "cleora_batch_create": (ctypes.c_int, [ctypes.POINTER(_P), ctypes.c_int, _P, _P, ctypes.c_int,
                                           ctypes.c_int, ctypes.c_int]),
    "cleora_batch_destroy": (None, [_P]),
    "cleora_batch_last_error": (ctypes.c_char_p, [_P]),
    "cleora_batch_totals": (ctypes.c_int, [_P, ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                           ctypes.POINTER(_I64), ctypes.POINTER(ctypes.c_int)]),
    "cleora_batch_graph_info": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64),
                                               ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "cleora_batch_schedule": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(_I64),
                                             ctypes.POINTER(_I64), ctypes.POINTER(_I64),
                                             ctypes.POINTER(_I64)]),
    "cleora_batch_node_ids": (ctypes.c_int, [_P, ctypes.c_int, _P, ctypes.c_int]),
    "cleora_batch_run": (ctypes.c_int, [_P, _P, ctypes.c_int]),
    "cleora_batch_launches": (ctypes.c_int, [_P, ctypes.POINTER(_I64)]),
    "cleora_serve_create": (ctypes.c_int, [ctypes.POINTER(_P), _P]),
    "cleora_serve_submit": (ctypes.c_int, [_P, _P, ctypes.POINTER(ctypes.c_uint64)]),
    "cleora_serve_poll": (ctypes.c_int, [_P, ctypes.c_uint64, ctypes.c_int, _P]),
    "cleora_serve_cancel": (ctypes.c_int, [_P, ctypes.c_uint64]),
    "cleora_serve_next": (ctypes.c_int, [_P, ctypes.c_int, ctypes.POINTER(ctypes.c_uint64), _P]),
    "cleora_serve_estimate": (_I64, [_P]),
    "cleora_serve_now": (ctypes.c_double, [_P]),
    "cleora_serve_stats": (ctypes.c_int, [_P, ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int),
                                          ctypes.POINTER(_I64), ctypes.POINTER(_I64), ctypes.POINTER(_I64)]),
    "cleora_serve_destroy": (None, [_P]),
    "cleora_propagate_noalloc": (ctypes.c_int, [_P, _P, _P, _I64, _I64, _P, _P, ctypes.c_int,
                                                ctypes.c_int, _I64, _P]),
    "cleora_noalloc_limits": (ctypes.c_int, [ctypes.c_int, ctypes.POINTER(_I64),
                                             ctypes.POINTER(_I64)]),
}


class CleoraError(RuntimeError):
    def __init__(self, status: int, message: str):
        super().__init__(f"{message} (status {status})")
        self.status = status


def library_path() -> str:
    return build_native.LIB


def load(build: bool = True):
    """Load (building first if needed) libcleora.so; raises if that is impossible."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = build_native.build() if build else build_native.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"{path} is missing: run build() first (no CPU fallback exists)")
        lib = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


# ---- pointer marshalling ----------------------------------------------------------------

def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(address, on_device) of a numpy array or torch tensor (contiguous), or (None, 0)."""
    if x is None:
        return None, 0
    if _is_torch(x):
        if not x.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return x.data_ptr(), 1 if x.is_cuda else 0
    if isinstance(x, np.ndarray):
        if not x.flags["C_CONTIGUOUS"]:
            raise ValueError("array must be C-contiguous")
        return x.ctypes.data, 0
    raise TypeError(f"unsupported array type {type(x)}")


def _check(ctx, status: int):
    if status != CLEORA_OK:
        lib = load()
        msg = lib.cleora_last_error(ctx).decode() if ctx else lib.cleora_status_string(status).decode()
        raise CleoraError(status, msg or lib.cleora_status_string(status).decode())


# ---- the C functions, one Python function each --------------------------------------------

def cleora_create(device: int = 0, stream: int | None = None):
    lib = load()
    h = _P()
    st = lib.cleora_create(ctypes.byref(h), device, stream)
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_create failed: " + lib.cleora_status_string(st).decode())
    return h


def cleora_destroy(ctx) -> None:
    load().cleora_destroy(ctx)


def cleora_last_error(ctx) -> str:
    return load().cleora_last_error(ctx).decode()


def cleora_sync(ctx) -> None:
    _check(ctx, load().cleora_sync(ctx))


def cleora_graph_build(ctx, src, dst, weights=None, directed: bool = False) -> None:
    ps, ds = _ptr(src)
    pd, dd = _ptr(dst)
    pw, dw = _ptr(weights)
    n_edges = int(src.shape[0])
    if int(dst.shape[0]) != n_edges or (weights is not None and int(weights.shape[0]) != n_edges):
        raise ValueError("src, dst and weights must have the same length")
    on_dev = ds
    if dd != on_dev or (weights is not None and dw != on_dev):
        raise ValueError("src, dst and weights must all be on the host or all on the device")
    _check(ctx, load().cleora_graph_build(ctx, ps, pd, pw, n_edges, int(bool(directed)), on_dev))


def cleora_num_nodes(ctx) -> int:
    v = _I64()
    _check(ctx, load().cleora_num_nodes(ctx, ctypes.byref(v)))
    return v.value


def cleora_num_entries(ctx) -> int:
    v = _I64()
    _check(ctx, load().cleora_num_entries(ctx, ctypes.byref(v)))
    return v.value


def cleora_graph_info(ctx) -> dict:
    n, nnz, mx = _I64(), _I64(), _I64()
    hv = ctypes.c_int()
    _check(ctx, load().cleora_graph_info(ctx, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(hv),
                                         ctypes.byref(mx)))
    return {"n": n.value, "nnz": nnz.value, "has_val": bool(hv.value), "max_row_len": mx.value}


def cleora_node_ids(ctx, out) -> None:
    p, dev = _ptr(out)
    _check(ctx, load().cleora_node_ids(ctx, p, dev))


def cleora_get_csr(ctx, rowptr=None, col=None, val=None, inv_deg=None, deg=None) -> None:
    ptrs = [_ptr(x) for x in (rowptr, col, val, inv_deg, deg)]
    devs = {d for (p, d) in ptrs if p is not None}
    if len(devs) > 1:
        raise ValueError("outputs must all be on the host or all on the device")
    dev = devs.pop() if devs else 0
    _check(ctx, load().cleora_get_csr(ctx, *[p for p, _ in ptrs], dev))


def cleora_init(ctx, d: int, seed: int = 0, storage: str | int = "f32") -> None:
    dt = DTYPES[storage] if isinstance(storage, str) else int(storage)
    _check(ctx, load().cleora_init(ctx, int(d), int(seed) & (2**64 - 1), dt))


def cleora_propagate(ctx, iters: int, out=None) -> None:
    p, dev = _ptr(out)
    _check(ctx, load().cleora_propagate(ctx, int(iters), p, dev))


def cleora_iteration(ctx) -> int:
    v = ctypes.c_int()
    _check(ctx, load().cleora_iteration(ctx, ctypes.byref(v)))
    return v.value


def cleora_get_embeddings(ctx, out, dtype: str | int = "f32") -> None:
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    p, dev = _ptr(out)
    _check(ctx, load().cleora_get_embeddings(ctx, p, dt, dev))


def cleora_set_embeddings(ctx, inp, dtype: str | int = "f32", iteration: int = 0) -> None:
    dt = DTYPES[dtype] if isinstance(dtype, str) else int(dtype)
    p, dev = _ptr(inp)
    _check(ctx, load().cleora_set_embeddings(ctx, p, dt, dev, int(iteration)))


def cleora_set_option(ctx, name: str, value: int) -> None:
    _check(ctx, load().cleora_set_option(ctx, OPTIONS[name], int(value)))


def cleora_get_option(ctx, name: str) -> int:
    v = _I64()
    _check(ctx, load().cleora_get_option(ctx, OPTIONS[name], ctypes.byref(v)))
    return v.value


def cleora_launch_count(ctx) -> int:
    v = _I64()
    _check(ctx, load().cleora_launch_count(ctx, ctypes.byref(v)))
    return v.value


def cleora_hot_entries(ctx) -> int:
    v = _I64()
    _check(ctx, load().cleora_hot_entries(ctx, ctypes.byref(v)))
    return v.value


def cleora_propagate_noalloc(rowptr, col, val, n: int, nnz: int, T_in, T_out, d: int,
                             storage: str | int = "f32", split_len: int = 0,
                             stream: int | None = None) -> None:
    """One allocation-free step on device tensors (see include/cleora.h)."""
    dt = DTYPES[storage] if isinstance(storage, str) else int(storage)
    ptrs = [_ptr(x) for x in (rowptr, col, val, T_in, T_out)]
    if any(p is not None and dev != 1 for p, dev in ptrs):
        raise ValueError("all arrays must be device tensors")
    st = load().cleora_propagate_noalloc(ptrs[0][0], ptrs[1][0], ptrs[2][0], int(n), int(nnz),
                                         ptrs[3][0], ptrs[4][0], int(d), dt, int(split_len), stream)
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_propagate_noalloc: " + load().cleora_status_string(st).decode())


def cleora_noalloc_limits(d: int) -> dict:
    sb, mc = _I64(), _I64()
    st = load().cleora_noalloc_limits(int(d), ctypes.byref(sb), ctypes.byref(mc))
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_noalloc_limits: invalid d")
    return {"scratch_bytes": sb.value, "max_split_chunks": mc.value}


# ---- inductivity and additivity ----------------------------------------------------------

def cleora_inductive(ctx, new_ids, nbr_ids, weights=None, out_ids=None, out=None):
    """Rows of new nodes from the current embeddings; returns (num_new, num_dropped)."""
    pn, dn = _ptr(new_ids)
    pb, _ = _ptr(nbr_ids)
    pw, _ = _ptr(weights)
    po, do = _ptr(out)
    pi, di = _ptr(out_ids)
    nn, nd = _I64(), _I64()
    rows = 0 if out is None else int(out.shape[0])
    _check(ctx, load().cleora_inductive(ctx, pn, pb, pw, int(new_ids.shape[0]), dn, pi, po, rows,
                                        ctypes.byref(nn), ctypes.byref(nd), do or di))
    return nn.value, nd.value


def cleora_chunked_embed(ctx, src, dst, weights, chunk_offsets, directed, d, iters, seed=0,
                         storage="f32", out_ids=None, out=None) -> int:
    """Algorithm 1 with edge chunks; returns the number of nodes.  chunk_offsets None: the
    library picks the chunks (see cleora_chunked_info)."""
    auto = chunk_offsets is None
    offs = np.ascontiguousarray([int(src.shape[0])] if auto else chunk_offsets, dtype=np.int64)
    ps, ds = _ptr(src)
    pd, _ = _ptr(dst)
    pw, _ = _ptr(weights)
    po, do = _ptr(out)
    pi, di = _ptr(out_ids)
    nn = _I64()
    st = DTYPES[storage] if isinstance(storage, str) else int(storage)
    rows = 0 if out is None else int(out.shape[0])
    _check(ctx, load().cleora_chunked_embed(ctx, ps, pd, pw, offs.ctypes.data, 0 if auto else len(offs) - 1,
                                            int(bool(directed)), int(d), int(iters),
                                            int(seed) & (2**64 - 1), st, ds, pi, po, rows,
                                            ctypes.byref(nn), do or di))
    return nn.value


def cleora_chunked_info(ctx) -> dict:
    q = ctx_int = ctypes.c_int()
    peak = _I64()
    _check(ctx, load().cleora_chunked_info(ctx, ctypes.byref(ctx_int), ctypes.byref(peak)))
    return {"chunks": q.value, "peak_device_bytes": peak.value}


# ---- identifiers and hypergraphs ----------------------------------------------------------

CLEORA_EXPAND_CLIQUE = 0
CLEORA_EXPAND_STAR = 1
EXPANSIONS = {"clique": CLEORA_EXPAND_CLIQUE, "star": CLEORA_EXPAND_STAR}


def _same_place(*arrays):
    devs = {_ptr(a)[1] for a in arrays if a is not None}
    if len(devs) > 1:
        raise ValueError("arrays must all be on the host or all on the device")
    return devs.pop() if devs else 0


def cleora_hash_ids(ctx, bytes_, offsets, seed=0, out=None):
    """XXH64 of strings bytes_[offsets[i]:offsets[i+1]] (uint8 and int64 arrays) -> uint64 ids."""
    count = int(offsets.shape[0]) - 1
    if out is None:
        out = np.empty(max(count, 0), np.uint64)
    on_dev = _same_place(bytes_, offsets)
    pb, _ = _ptr(bytes_)
    po, _ = _ptr(offsets)
    pout, dout = _ptr(out)
    _check(ctx, load().cleora_hash_ids(ctx, pb, po, count, int(seed) & (2**64 - 1), pout, on_dev, dout))
    return out


def cleora_expand_hypergraph(ctx, members, hoff, mode="clique", star_ids=None, src_out=None, dst_out=None):
    """Edges of the clique or star expansion; with no outputs given, host arrays sized by a
    counting call are returned."""
    H = int(hoff.shape[0]) - 1
    on_dev = _same_place(members, hoff, star_ids)
    m = EXPANSIONS[mode] if isinstance(mode, str) else int(mode)
    pm, _ = _ptr(members)
    ph, _ = _ptr(hoff)
    ps, _ = _ptr(star_ids)
    ne = _I64()
    if src_out is None:
        _check(ctx, load().cleora_expand_hypergraph(ctx, pm, ph, H, m, ps, on_dev, None, None, 0,
                                                    ctypes.byref(ne), 0))
        src_out = np.empty(ne.value, np.uint64)
        dst_out = np.empty(ne.value, np.uint64)
    psrc, dsrc = _ptr(src_out)
    pdst, _ = _ptr(dst_out)
    _check(ctx, load().cleora_expand_hypergraph(ctx, pm, ph, H, m, ps, on_dev, psrc, pdst,
                                                int(src_out.shape[0]), ctypes.byref(ne), dsrc))
    return src_out[:ne.value], dst_out[:ne.value]


def cleora_hypergraph_build(ctx, members, hoff, mode="clique", star_ids=None) -> int:
    H = int(hoff.shape[0]) - 1
    on_dev = _same_place(members, hoff, star_ids)
    m = EXPANSIONS[mode] if isinstance(mode, str) else int(mode)
    pm, _ = _ptr(members)
    ph, _ = _ptr(hoff)
    ps, _ = _ptr(star_ids)
    ne = _I64()
    _check(ctx, load().cleora_hypergraph_build(ctx, pm, ph, H, m, ps, on_dev, ctypes.byref(ne)))
    return ne.value


# ---- batched small graphs -------------------------------------------------------------

class cleora_graph_desc(ctypes.Structure):
    _fields_ = [("src", _P), ("dst", _P), ("weights", _P), ("num_edges", _I64),
                ("directed", ctypes.c_int), ("d", ctypes.c_int), ("iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("storage", ctypes.c_int)]


def _bcheck(b, status: int):
    if status != CLEORA_OK:
        lib = load()
        msg = lib.cleora_batch_last_error(b).decode() if b else ""
        raise CleoraError(status, msg or lib.cleora_status_string(status).decode())


def cleora_batch_create(graphs, device: int = 0, stream: int | None = None, autotune: bool = True):
    """graphs: sequence of dicts with src, dst, weights (or None), directed, d, iters, seed,
    storage; all arrays on the host (numpy) or all on the device (torch CUDA)."""
    lib = load()
    descs = (cleora_graph_desc * max(len(graphs), 1))()
    on_dev = None
    for i, g in enumerate(graphs):
        ps, ds = _ptr(g["src"])
        pd, dd = _ptr(g["dst"])
        pw, dw = _ptr(g.get("weights"))
        devs = {ds, dd} | ({dw} if g.get("weights") is not None else set())
        if len(g["src"]) == 0:
            devs = set()
        if len(devs) > 1 or (on_dev is not None and devs and devs != {on_dev}):
            raise ValueError("all edge arrays must be on the host or all on the device")
        if devs:
            on_dev = devs.pop()
        st = g.get("storage", "f32")
        descs[i] = cleora_graph_desc(ps, pd, pw, int(len(g["src"])), int(bool(g["directed"])),
                                     int(g["d"]), int(g["iters"]), int(g.get("seed", 0)) & (2**64 - 1),
                                     DTYPES[st] if isinstance(st, str) else int(st))
    h = _P()
    st = lib.cleora_batch_create(ctypes.byref(h), device, stream, descs, len(graphs), on_dev or 0,
                                 int(bool(autotune)))
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_batch_create failed: " + lib.cleora_status_string(st).decode())
    return h


def cleora_batch_destroy(b) -> None:
    load().cleora_batch_destroy(b)


def cleora_batch_last_error(b) -> str:
    return load().cleora_batch_last_error(b).decode()


def cleora_batch_totals(b) -> dict:
    n, nnz, oe = _I64(), _I64(), _I64()
    mi = ctypes.c_int()
    _bcheck(b, load().cleora_batch_totals(b, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(oe),
                                          ctypes.byref(mi)))
    return {"nodes": n.value, "nnz": nnz.value, "out_elems": oe.value, "max_iters": mi.value}


def cleora_batch_graph_info(b, g: int) -> dict:
    n, nnz, off = _I64(), _I64(), _I64()
    _bcheck(b, load().cleora_batch_graph_info(b, g, ctypes.byref(n), ctypes.byref(nnz), ctypes.byref(off)))
    return {"n": n.value, "nnz": nnz.value, "out_offset": off.value}


def cleora_batch_schedule(b, g: int) -> dict:
    v, m, s, t = _I64(), _I64(), _I64(), _I64()
    _bcheck(b, load().cleora_batch_schedule(b, g, ctypes.byref(v), ctypes.byref(m), ctypes.byref(s),
                                            ctypes.byref(t)))
    return {"vec_bytes": v.value, "row_mode": m.value, "split_len": s.value, "task_nnz": t.value}


def cleora_batch_node_ids(b, g: int, out) -> None:
    p, dev = _ptr(out)
    _bcheck(b, load().cleora_batch_node_ids(b, g, p, dev))


def cleora_batch_run(b, out=None) -> None:
    p, dev = _ptr(out)
    _bcheck(b, load().cleora_batch_run(b, p, dev))


def cleora_batch_launches(b) -> int:
    v = _I64()
    _bcheck(b, load().cleora_batch_launches(b, ctypes.byref(v)))
    return v.value


class Batch:
    """Many graphs embedded together (wraps a ``cleora_batch``)."""

    def __init__(self, graphs, device: int = 0, stream: int | None = None, autotune: bool = True):
        self._keep = graphs  # the inputs must stay alive during create
        self.handle = cleora_batch_create(graphs, device, stream, autotune)
        self._keep = None
        self.count = len(graphs)
        self.totals = cleora_batch_totals(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            cleora_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def run(self, out=None):
        """Replays the batch; copies the packed FP32 results to `out` when given."""
        cleora_batch_run(self.handle, out)
        return out

    def run_host(self) -> np.ndarray:
        out = np.empty(self.totals["out_elems"], np.float32)
        cleora_batch_run(self.handle, out)
        return out

    def graph(self, out, g: int, d: int):
        inf = cleora_batch_graph_info(self.handle, g)
        return out[inf["out_offset"]: inf["out_offset"] + inf["n"] * d].reshape(inf["n"], d)

    def info(self, g: int) -> dict:
        return cleora_batch_graph_info(self.handle, g)

    def schedule(self, g: int) -> dict:
        return cleora_batch_schedule(self.handle, g)

    def node_ids(self, g: int) -> np.ndarray:
        out = np.empty(cleora_batch_graph_info(self.handle, g)["n"], np.uint64)
        cleora_batch_node_ids(self.handle, g, out)
        return out

    def launches(self) -> int:
        return cleora_batch_launches(self.handle)


# ---- serving ---------------------------------------------------------------------------

class cleora_server_config(ctypes.Structure):
    _fields_ = [("device", ctypes.c_int), ("hbm_budget_bytes", _I64), ("max_slots", ctypes.c_int),
                ("queue_capacity", ctypes.c_int), ("inject_alloc_failure_every", ctypes.c_int),
                ("short_slots", ctypes.c_int), ("short_job_seconds", ctypes.c_double)]


class cleora_job(ctypes.Structure):
    _fields_ = [("src", _P), ("dst", _P), ("weights", _P), ("num_edges", _I64),
                ("directed", ctypes.c_int), ("d", ctypes.c_int), ("iters", ctypes.c_int),
                ("seed", ctypes.c_uint64), ("storage", ctypes.c_int), ("out", _P),
                ("out_rows", _I64), ("nodes_hint", _I64)]


class cleora_result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("slot", ctypes.c_int), ("n", _I64), ("nnz", _I64),
                ("bytes_reserved", _I64), ("t_submit", ctypes.c_double),
                ("t_admit", ctypes.c_double), ("t_done", ctypes.c_double),
                ("t_built", ctypes.c_double), ("t_inited", ctypes.c_double)]


def _job_struct(src, dst, weights, directed, d, iters, seed, storage, out, nodes_hint):
    for x in (src, dst, weights, out):
        if x is not None and _ptr(x)[1]:
            raise ValueError("serving jobs take host arrays")
    st = DTYPES[storage] if isinstance(storage, str) else int(storage)
    out_rows = 0 if out is None else int(out.shape[0])
    return cleora_job(_ptr(src)[0], _ptr(dst)[0], _ptr(weights)[0], int(len(src)), int(bool(directed)),
                      int(d), int(iters), int(seed) & (2**64 - 1), st, _ptr(out)[0], out_rows,
                      int(nodes_hint))


def cleora_serve_create(device: int = 0, hbm_budget_bytes: int = 0, max_slots: int = 0,
                        queue_capacity: int = 0, inject_alloc_failure_every: int = 0,
                        short_slots: int = 0, short_job_seconds: float = 0.0):
    lib = load()
    cfg = cleora_server_config(device, hbm_budget_bytes, max_slots, queue_capacity,
                               inject_alloc_failure_every, short_slots, float(short_job_seconds))
    h = _P()
    st = lib.cleora_serve_create(ctypes.byref(h), ctypes.byref(cfg))
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_serve_create failed: " + lib.cleora_status_string(st).decode())
    return h


def cleora_serve_submit(server, job: cleora_job) -> int:
    jid = ctypes.c_uint64()
    st = load().cleora_serve_submit(server, ctypes.byref(job), ctypes.byref(jid))
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_serve_submit: " + load().cleora_status_string(st).decode())
    return jid.value


def cleora_serve_poll(server, job_id: int, timeout_ms: int = -1):
    """Returns a cleora_result, or None when the job is not done within timeout_ms."""
    res = cleora_result()
    st = load().cleora_serve_poll(server, job_id, int(timeout_ms), ctypes.byref(res))
    if st == CLEORA_ERR_TIMEOUT:
        return None
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_serve_poll: " + load().cleora_status_string(st).decode())
    return res


def cleora_serve_next(server, timeout_ms: int = -1):
    """(job_id, cleora_result) of the next finished job, or None after timeout_ms."""
    jid = ctypes.c_uint64()
    res = cleora_result()
    st = load().cleora_serve_next(server, int(timeout_ms), ctypes.byref(jid), ctypes.byref(res))
    if st == CLEORA_ERR_TIMEOUT:
        return None
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_serve_next: " + load().cleora_status_string(st).decode())
    return jid.value, res


def cleora_serve_cancel(server, job_id: int) -> int:
    return load().cleora_serve_cancel(server, job_id)


def cleora_serve_estimate(job: cleora_job) -> int:
    return load().cleora_serve_estimate(ctypes.byref(job))


def cleora_serve_now(server) -> float:
    return load().cleora_serve_now(server)


def cleora_serve_stats(server) -> dict:
    q, r = ctypes.c_int(), ctypes.c_int()
    b, c, bud = _I64(), _I64(), _I64()
    st = load().cleora_serve_stats(server, ctypes.byref(q), ctypes.byref(r), ctypes.byref(b),
                                   ctypes.byref(c), ctypes.byref(bud))
    if st != CLEORA_OK:
        raise CleoraError(st, "cleora_serve_stats")
    return {"queued": q.value, "running": r.value, "bytes_reserved": b.value,
            "completed": c.value, "budget": bud.value}


def cleora_serve_destroy(server) -> None:
    load().cleora_serve_destroy(server)


class Server:
    """Continuous-batching embedding server (wraps a ``cleora_server``)."""

    def __init__(self, device: int = 0, hbm_budget_bytes: int = 0, max_slots: int = 0,
                 queue_capacity: int = 0, inject_alloc_failure_every: int = 0,
                 short_slots: int = 0, short_job_seconds: float = 0.0):
        self.handle = cleora_serve_create(device, hbm_budget_bytes, max_slots, queue_capacity,
                                          inject_alloc_failure_every, short_slots,
                                          short_job_seconds)
        self._held = {}  # job id -> arrays the job reads or writes (kept alive until collected)

    def submit(self, src, dst, weights=None, directed=False, d=128, iters=4, seed=0,
               storage="f32", out=None, nodes_hint=0) -> int:
        job = _job_struct(src, dst, weights, directed, d, iters, seed, storage, out, nodes_hint)
        jid = cleora_serve_submit(self.handle, job)
        self._held[jid] = (src, dst, weights, out)
        return jid

    def estimate(self, src, dst, weights=None, directed=False, d=128, iters=4, storage="f32",
                 nodes_hint=0) -> int:
        return cleora_serve_estimate(_job_struct(src, dst, weights, directed, d, iters, 0, storage,
                                                 None, nodes_hint))

    def poll(self, job_id: int, timeout_ms: int = -1):
        res = cleora_serve_poll(self.handle, job_id, timeout_ms)
        if res is not None:
            self._held.pop(job_id, None)
        return res

    def next(self, timeout_ms: int = -1):
        r = cleora_serve_next(self.handle, timeout_ms)
        if r is not None:
            self._held.pop(r[0], None)
        return r

    def cancel(self, job_id: int) -> int:
        return cleora_serve_cancel(self.handle, job_id)

    def now(self) -> float:
        return cleora_serve_now(self.handle)

    def stats(self) -> dict:
        return cleora_serve_stats(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            cleora_serve_destroy(self.handle)
            self.handle = None
            self._held.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


# ---- convenience object (same calls, owns the handle) ------------------------------------

class Context:
    """One graph and its embeddings on one GPU; wraps a ``cleora_ctx``."""

    def __init__(self, device: int = 0, stream: int | None = None):
        self.handle = cleora_create(device, stream)
        self.device = device

    def close(self):
        if getattr(self, "handle", None):
            cleora_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def graph_build(self, src, dst, weights=None, directed=False):
        cleora_graph_build(self.handle, src, dst, weights, directed)
        return self

    def info(self) -> dict:
        return cleora_graph_info(self.handle)

    def node_ids(self) -> np.ndarray:
        out = np.empty(cleora_num_nodes(self.handle), np.uint64)
        cleora_node_ids(self.handle, out)
        return out

    def csr(self) -> dict:
        inf = self.info()
        n, nnz = inf["n"], inf["nnz"]
        r = {"rowptr": np.empty(n + 1, np.int64), "col": np.empty(nnz, np.int32),
             "val": np.empty(nnz, np.float32), "inv_deg": np.empty(n, np.float32),
             "deg": np.empty(n, np.float64)}
        cleora_get_csr(self.handle, r["rowptr"], r["col"], r["val"], r["inv_deg"], r["deg"])
        r.update(inf)
        return r

    def init(self, d, seed=0, storage="f32"):
        cleora_init(self.handle, d, seed, storage)
        self.d = d
        self.storage = storage
        return self

    def propagate(self, iters, out=None):
        cleora_propagate(self.handle, iters, out)
        return out

    def embeddings(self, dtype="f32"):
        n = cleora_num_nodes(self.handle)
        if dtype == "f32":
            out = np.empty((n, self.d), np.float32)
        else:
            out = np.empty((n, self.d), np.uint16)  # raw bf16 bits
        cleora_get_embeddings(self.handle, out, dtype)
        return out

    def set_embeddings(self, arr, dtype="f32", iteration=0):
        cleora_set_embeddings(self.handle, arr, dtype, iteration)

    def set_option(self, name, value):
        cleora_set_option(self.handle, name, value)

    def sync(self):
        cleora_sync(self.handle)

    def launches(self) -> int:
        return cleora_launch_count(self.handle)

    def hot_entries(self) -> int:
        return cleora_hot_entries(self.handle)
