"""Cleora FP64 CPU oracle -- TEST INFRASTRUCTURE ONLY.

Python access to ``cleora_oracle.c`` (plain C, FP64, pthreads over blocks of rows), written
from arXiv 2102.02302 Sec. 3.2 and Algorithm 1.  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import this package; the CUDA library never
does, and the two share no code.

Pins (``tests/test_oracle_pins.py``): the splitmix64 reference outputs, brute-force dense
D^-1 A products on tiny graphs, unit row norms, fixed points of constant columns, leaf
rows, disjoint cliques, stars, complete bipartite and regular graphs, weight scaling,
duplicate edges and edge-order invariance.  Nothing here is "parity unpinned".
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cleora_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

_P = ctypes.c_void_p
_I64 = ctypes.c_int64


def build(force: bool = False) -> str:
    """Compile liboracle.so with gcc (FP contraction off so both host CPUs agree)."""
    stale = (not os.path.exists(_LIB_PATH)
             or os.path.getmtime(_LIB_PATH) < max(os.path.getmtime(_SRC),
                                                  os.path.getmtime(_SRC[:-2] + ".h")))
    if force or stale:
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        cmd = ["gcc", "-O2", "-std=c11", "-D_POSIX_C_SOURCE=200809L", "-fPIC", "-shared",
               "-ffp-contract=off", "-fno-fast-math", "-pthread", "-o", tmp, _SRC, "-lm"]
        subprocess.run(cmd, check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        try:
            lib = ctypes.CDLL(_LIB_PATH)
        except OSError:  # a library built for another CPU: rebuild here
            build(force=True)
            lib = ctypes.CDLL(_LIB_PATH)
        lib.oracle_build.argtypes = [_P, _P, _P, _I64, ctypes.c_int, ctypes.POINTER(_P)]
        lib.oracle_build.restype = ctypes.c_int
        lib.oracle_graph_free.argtypes = [_P]
        lib.oracle_graph_free.restype = None
        lib.oracle_graph_n.argtypes = [_P]
        lib.oracle_graph_n.restype = _I64
        lib.oracle_graph_nnz.argtypes = [_P]
        lib.oracle_graph_nnz.restype = _I64
        lib.oracle_graph_has_val.argtypes = [_P]
        lib.oracle_graph_has_val.restype = ctypes.c_int
        lib.oracle_graph_copy.argtypes = [_P, _P, _P, _P, _P, _P]
        lib.oracle_graph_copy.restype = None
        lib.oracle_stored_values.argtypes = [_P, _P, _P]
        lib.oracle_stored_values.restype = None
        lib.oracle_mix.argtypes = [ctypes.c_uint64]
        lib.oracle_mix.restype = ctypes.c_uint64
        lib.oracle_init_value.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_uint32]
        lib.oracle_init_value.restype = ctypes.c_double
        lib.oracle_init.argtypes = [_P, _I64, ctypes.c_int, ctypes.c_uint64, _P]
        lib.oracle_init.restype = None
        lib.oracle_propagate.argtypes = [_P, ctypes.c_int, _P, ctypes.c_int, _P, ctypes.c_int]
        lib.oracle_propagate.restype = ctypes.c_int
        lib.oracle_step_rows.argtypes = [_P, ctypes.c_int, _P, _P, _I64, _P, ctypes.c_int]
        lib.oracle_step_rows.restype = ctypes.c_int
        lib.oracle_step_csr_rows.argtypes = [_P, _P, _P, _I64, ctypes.c_int, _P, _P, _I64, _P,
                                             ctypes.c_int]
        lib.oracle_step_csr_rows.restype = ctypes.c_int
        lib.oracle_xxh64.argtypes = [_P, _I64, ctypes.c_uint64]
        lib.oracle_xxh64.restype = ctypes.c_uint64
        lib.oracle_hash_strings.argtypes = [_P, _P, _I64, ctypes.c_uint64, _P]
        lib.oracle_hash_strings.restype = None
        _lib = lib
        return lib


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_P)


class OracleError(RuntimeError):
    pass


@dataclass
class Graph:
    """The oracle's graph: ids, CSR of M's pattern, e_ab, deg_a and the compact FP32 store."""
    handle: int
    n: int
    nnz: int
    has_val: bool
    ids: np.ndarray
    rowptr: np.ndarray
    col: np.ndarray
    e: np.ndarray
    deg: np.ndarray
    val32: np.ndarray      # fp32(e_ab / deg_a), nnz
    inv_deg32: np.ndarray  # 1.0f / fp32(deg_a), n

    def __del__(self):
        if self.handle and _lib is not None:
            _lib.oracle_graph_free(ctypes.c_void_p(self.handle))
            self.handle = 0

    def dense_m(self) -> np.ndarray:
        """Dense M (tiny graphs only)."""
        m = np.zeros((self.n, self.n))
        for a in range(self.n):
            for k in range(self.rowptr[a], self.rowptr[a + 1]):
                m[a, self.col[k]] = self.e[k] / self.deg[a]
        return m


def build_graph(src, dst, weights=None, directed: bool = False) -> Graph:
    lib = _load()
    src = np.ascontiguousarray(src, dtype=np.uint64)
    dst = np.ascontiguousarray(dst, dtype=np.uint64)
    w = None if weights is None else np.ascontiguousarray(weights, dtype=np.float32)
    h = _P()
    rc = lib.oracle_build(_ptr(src), _ptr(dst), _ptr(w), src.shape[0], int(directed),
                          ctypes.byref(h))
    if rc != 0:
        raise OracleError(f"oracle_build failed ({rc})")
    n = lib.oracle_graph_n(h)
    nnz = lib.oracle_graph_nnz(h)
    ids = np.empty(n, np.uint64)
    rowptr = np.empty(n + 1, np.int64)
    col = np.empty(nnz, np.int32)
    e = np.empty(nnz, np.float64)
    deg = np.empty(n, np.float64)
    lib.oracle_graph_copy(h, _ptr(ids), _ptr(rowptr), _ptr(col), _ptr(e), _ptr(deg))
    val32 = np.empty(nnz, np.float32)
    inv32 = np.empty(n, np.float32)
    lib.oracle_stored_values(h, _ptr(val32), _ptr(inv32))
    return Graph(h.value, n, nnz, bool(lib.oracle_graph_has_val(h)), ids, rowptr, col, e, deg,
                 val32, inv32)


def build_from(edges) -> Graph:
    """Build from a ``synth.EdgeList``."""
    return build_graph(edges.src, edges.dst, edges.weights, edges.directed)


def mix(z: int) -> int:
    return _load().oracle_mix(z)


def init_value(seed: int, node_id: int, j: int) -> float:
    return _load().oracle_init_value(seed, node_id, j)


def init(ids, d: int, seed: int) -> np.ndarray:
    ids = np.ascontiguousarray(ids, dtype=np.uint64)
    out = np.empty((ids.shape[0], d), np.float64)
    _load().oracle_init(_ptr(ids), ids.shape[0], d, seed, _ptr(out))
    return out


def propagate(g: Graph, T, iters: int, nthreads: int = 0) -> np.ndarray:
    T = np.ascontiguousarray(T, dtype=np.float64)
    if T.shape[0] != g.n:
        raise ValueError("T must have one row per node")
    out = np.empty_like(T)
    rc = _load().oracle_propagate(ctypes.c_void_p(g.handle), T.shape[1], _ptr(T), iters,
                                  _ptr(out), nthreads)
    if rc != 0:
        raise OracleError(f"oracle_propagate failed ({rc})")
    return out


def step_rows(g: Graph, T_prev, rows, nthreads: int = 0) -> np.ndarray:
    T_prev = np.ascontiguousarray(T_prev, dtype=np.float64)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    out = np.empty((rows.shape[0], T_prev.shape[1]), np.float64)
    rc = _load().oracle_step_rows(ctypes.c_void_p(g.handle), T_prev.shape[1], _ptr(T_prev),
                                  _ptr(rows), rows.shape[0], _ptr(out), nthreads)
    if rc != 0:
        raise OracleError(f"oracle_step_rows failed ({rc})")
    return out


def step_csr_rows(rowptr, col, e, T_prev_f32, rows, nthreads: int = 0) -> np.ndarray:
    """One iteration on the listed rows of a graph given as a CSR (e = None: unit e_ab), from
    an FP32 previous iterate: rownorm(sum_b (e_ab / deg_a) T_prev[b]) in FP64.  For graphs
    too large for the oracle's own build; the CSR must come from a checked source."""
    rowptr = np.ascontiguousarray(rowptr, dtype=np.int64)
    col = np.ascontiguousarray(col, dtype=np.int32)
    e = None if e is None else np.ascontiguousarray(e, dtype=np.float64)
    T = np.ascontiguousarray(T_prev_f32, dtype=np.float32)
    rows = np.ascontiguousarray(rows, dtype=np.int64)
    n = rowptr.shape[0] - 1
    if T.shape[0] != n:
        raise ValueError("T_prev must have one row per node")
    out = np.empty((rows.shape[0], T.shape[1]), np.float64)
    rc = _load().oracle_step_csr_rows(_ptr(rowptr), _ptr(col), _ptr(e), n, T.shape[1], _ptr(T),
                                      _ptr(rows), rows.shape[0], _ptr(out), nthreads)
    if rc != 0:
        raise OracleError(f"oracle_step_csr_rows failed ({rc})")
    return out


def embed(edges, d: int, iters: int, seed: int = 0, nthreads: int = 0):
    """Whole method on one graph: returns (graph, T_I) with T_I in ascending-id row order."""
    g = build_from(edges)
    T0 = init(g.ids, d, seed)
    return g, propagate(g, T0, iters, nthreads)


def inductive(g: Graph, T, new_ids, nbr_ids, weights=None):
    """Rows for nodes added after the embedding (Sec. 1, "Inductivity"; Sec. 3.2: a new node
    is the weighted average of its neighbours' representations).  For every new id u with at
    least one edge to a node of g: e_ub = weight sum of its edges to b (FP64, edge order),
    deg_u = sum_b e_ub (ascending b), y = sum_b (e_ub / deg_u) T[b], row = y / ||y||.  Edges to
    ids that are not nodes of g are dropped.  Returns (ids ascending, rows, dropped)."""
    T = np.asarray(T, dtype=np.float64)
    new_ids = np.asarray(new_ids, dtype=np.uint64)
    nbr_ids = np.asarray(nbr_ids, dtype=np.uint64)
    w = np.ones(new_ids.size) if weights is None else np.asarray(weights, dtype=np.float32).astype(np.float64)
    pos = np.searchsorted(g.ids, nbr_ids)
    known = (pos < g.n) & (g.ids[np.minimum(pos, max(g.n - 1, 0))] == nbr_ids) if g.n else np.zeros(new_ids.size, bool)
    rows = {}
    for k in range(new_ids.size):
        if not known[k]:
            continue
        e = rows.setdefault(int(new_ids[k]), {})
        b = int(pos[k])
        e[b] = e.get(b, 0.0) + float(w[k])
    ids = np.array(sorted(rows), dtype=np.uint64)
    out = np.zeros((ids.size, T.shape[1]))
    for i, u in enumerate(ids):
        e = rows[int(u)]
        deg = 0.0
        for b in sorted(e):
            deg += e[b]
        y = np.zeros(T.shape[1])
        for b in sorted(e):
            y += (e[b] / deg) * T[b]
        nrm = np.sqrt(np.sum(y * y))
        out[i] = y / nrm if nrm > 0 else 0.0
    return ids, out, int((~known).sum())


def chunked_embed(src, dst, weights, chunk_offsets, directed, d, iters, seed=0):
    """Algorithm 1 with Q edge chunks: chunk q (edges chunk_offsets[q]..chunk_offsets[q+1]-1)
    is embedded alone (its own M_q, T_0 from the same id hash, I iterations), then
    T_v = sum_q w_qv T^q_v with w_qv = occ_q(v) / sum_k occ_k(v), occ_q(v) the number of
    endpoints of chunk q's edges equal to v (the node weight of Algorithm 1 read as an
    occurrence share).  Returns (ids ascending, T)."""
    src = np.asarray(src, dtype=np.uint64)
    dst = np.asarray(dst, dtype=np.uint64)
    ids = np.unique(np.concatenate([src, dst]))
    ends = np.concatenate([src, dst])
    occ_all = np.zeros(ids.size)
    np.add.at(occ_all, np.searchsorted(ids, ends), 1.0)
    acc = np.zeros((ids.size, d))
    for q in range(len(chunk_offsets) - 1):
        b, t = int(chunk_offsets[q]), int(chunk_offsets[q + 1])
        if t == b:
            continue
        wq = None if weights is None else np.asarray(weights)[b:t]
        gq = build_graph(src[b:t], dst[b:t], wq, directed)
        Tq = propagate(gq, init(gq.ids, d, seed), iters)
        occ_q = np.zeros(gq.n)
        np.add.at(occ_q, np.searchsorted(gq.ids, np.concatenate([src[b:t], dst[b:t]])), 1.0)
        v = np.searchsorted(ids, gq.ids)
        acc[v] += (occ_q / occ_all[v])[:, None] * Tq
    return ids, acc


# ---- identifiers and hypergraphs (Sec. 4.3; Sec. 3.2 "Hypergraph Expansion") ------------------

def xxh64(data: bytes, seed: int = 0) -> int:
    """XXH64 of a byte string (xxHash specification), the paper's identifier hash (Sec. 4.3)."""
    buf = np.frombuffer(bytes(data), dtype=np.uint8) if len(data) else np.zeros(1, np.uint8)
    return _load().oracle_xxh64(_ptr(buf), len(data), seed & (2**64 - 1))


def hash_strings(strings, seed: int = 0) -> np.ndarray:
    """XXH64 of every string (bytes or str, UTF-8) -> uint64 ids."""
    enc = [s.encode() if isinstance(s, str) else bytes(s) for s in strings]
    offsets = np.zeros(len(enc) + 1, np.int64)
    offsets[1:] = np.cumsum([len(b) for b in enc])
    blob = np.frombuffer(b"".join(enc) or b"\0", dtype=np.uint8)
    out = np.empty(len(enc), np.uint64)
    _load().oracle_hash_strings(_ptr(blob), _ptr(offsets), len(enc), seed & (2**64 - 1), _ptr(out))
    return out


STAR_KEY = 0x5354415253544152  # "STARSTAR": star-node ids when the caller gives none


def star_node_id(h: int) -> int:
    """Id of hyperedge h's star node when none is given: the splitmix64 output function of
    h ^ STAR_KEY."""
    return mix(h ^ STAR_KEY)


def expand(members, hoff, mode: str, star_ids=None):
    """Hypergraph expansion (Sec. 3.2): hyperedge h holds members[hoff[h]:hoff[h+1]]; its
    distinct members in ascending id order u_0 < ... < u_{k-1} give
      clique: the edges (u_i, u_j) for i < j, in lexicographic (i, j) order, k(k-1)/2 of them;
      star:   the edges (s_h, u_i) for every i, s_h the star node (star_ids[h] or
              star_node_id(h)), k of them.
    Hyperedges follow their order.  Returns (src, dst) uint64 arrays (undirected edges)."""
    members = np.asarray(members, dtype=np.uint64)
    hoff = np.asarray(hoff, dtype=np.int64)
    src, dst = [], []
    for h in range(hoff.size - 1):
        u = sorted(set(int(x) for x in members[hoff[h]:hoff[h + 1]]))
        if mode == "clique":
            for i in range(len(u)):
                for j in range(i + 1, len(u)):
                    src.append(u[i])
                    dst.append(u[j])
        elif mode == "star":
            s = int(star_ids[h]) if star_ids is not None else star_node_id(h)
            for x in u:
                src.append(s)
                dst.append(x)
        else:
            raise ValueError(mode)
    return np.array(src, dtype=np.uint64), np.array(dst, dtype=np.uint64)
