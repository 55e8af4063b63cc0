"""Seeded synthetic graph generators shared by the tests, the bench and the oracle checks.

This module holds no arithmetic of the embedding method itself: it only draws edge lists
(and edge weights) from counter-based splitmix64 streams, so the same call gives the same
graph whatever the thread count or the machine.  The GPU generator in ``synth/gen_gpu.cu``
implements the same definitions for the large power-law graph and is checked against this
file bit for bit.

Counter-based stream.  ``mix`` is splitmix64's output function (Steele, Lea & Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014; Vigna's public-domain
``splitmix64.c``): add the golden-ratio increment, then two xor-shift/multiply rounds.
A draw is ``rng(seed, stream, counter) = mix(mix(mix(seed) ^ stream) ^ counter)``.

Chung-Lu power law.  Node ``i`` (0 <= i < n) has weight ``w_i = (i + i0)^(-alpha)`` with
``alpha = 1/(gamma - 1)``.  ``i0`` is solved by bisection so that node 0's expected number
of edge endpoints equals a requested maximum degree.  An endpoint is drawn by inverse CDF
over the cumulative weights, held as integers ``thr[i] = round(cum_i * 2^53)`` so that both
this file and the CUDA generator decide every draw by the same integer comparison.

External ids.  Node ``i`` is published under ``id(i) = mix(i ^ mix(seed ^ ID_KEY))``; mix is
a bijection of 64-bit words, so ids are distinct, and their order is unrelated to degree.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

U64 = np.uint64
GOLDEN = 0x9E3779B97F4A7C15
ID_KEY = 0xC1E0A5EED0000001
STREAM_SRC = 1
STREAM_DST = 2
STREAM_W1 = 3
STREAM_W2 = 4
TWO53 = 1 << 53


def mix(z):
    """splitmix64 output function on a numpy uint64 array (wrapping arithmetic)."""
    z = np.asarray(z, dtype=U64)
    with np.errstate(over="ignore"):
        z = z + U64(GOLDEN)
        z = (z ^ (z >> U64(30))) * U64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> U64(27))) * U64(0x94D049BB133111EB)
        return z ^ (z >> U64(31))


def mix_int(z: int) -> int:
    """splitmix64 output function on a Python int (used for scalar keys)."""
    m = (1 << 64) - 1
    z = (z + GOLDEN) & m
    z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & m
    z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & m
    return z ^ (z >> 31)


def rng(seed: int, stream: int, counter) -> np.ndarray:
    """Counter-based draw: mix(mix(mix(seed) ^ stream) ^ counter), vectorised over counter."""
    key = mix_int(mix_int(seed & ((1 << 64) - 1)) ^ stream)
    return mix(U64(key) ^ np.asarray(counter, dtype=U64))


def node_ids(n: int, seed: int, start: int = 0) -> np.ndarray:
    """External uint64 ids of nodes start..start+n-1 (distinct: mix is a bijection)."""
    key = mix_int((seed ^ ID_KEY) & ((1 << 64) - 1))
    return mix(np.arange(start, start + n, dtype=U64) ^ U64(key))


# ---------------------------------------------------------------------------------------
# Chung-Lu power-law sampling
# ---------------------------------------------------------------------------------------

def _weights(n: int, gamma: float, i0: float) -> np.ndarray:
    alpha = 1.0 / (gamma - 1.0)
    return (np.arange(n, dtype=np.float64) + i0) ** (-alpha)


def solve_i0(n: int, gamma: float, endpoints: int, max_deg: float) -> float:
    """Offset i0 such that node 0 expects ``max_deg`` of the ``endpoints`` endpoint draws."""
    lo, hi = 1e-6, float(n)
    alpha = 1.0 / (gamma - 1.0)
    head = min(n, 100_000)

    def total(i0):
        # exact head sum plus the midpoint-rule integral of the smooth tail
        s = _weights(head, gamma, i0).sum()
        if n > head:
            a, b = head - 0.5 + i0, n - 0.5 + i0
            if abs(alpha - 1.0) < 1e-12:
                s += math.log(b / a)
            else:
                s += (b ** (1.0 - alpha) - a ** (1.0 - alpha)) / (1.0 - alpha)
        return s

    def share0(i0):
        return endpoints * i0 ** (-alpha) / total(i0)

    for _ in range(60):  # share0 decreases in i0
        mid = math.sqrt(lo * hi)
        if share0(mid) > max_deg:
            lo = mid
        else:
            hi = mid
    return math.sqrt(lo * hi)


def cdf_thresholds(n: int, gamma: float, i0: float) -> np.ndarray:
    """Integer inverse-CDF table: endpoint = first i with r < thr[i], r uniform in [0, 2^53)."""
    w = _weights(n, gamma, i0)
    cum = np.cumsum(w)
    thr = np.rint(cum / cum[-1] * float(TWO53)).astype(np.uint64)
    thr[-1] = U64(TWO53)
    return thr


def sample_nodes(thr: np.ndarray, draws: np.ndarray) -> np.ndarray:
    """Map 64-bit draws to node indices through the threshold table (top 53 bits)."""
    r = draws >> U64(11)
    return np.searchsorted(thr, r, side="right").astype(np.int64)


@dataclass
class EdgeList:
    """A synthetic edge list: external ids, optional float32 weights, directed flag."""
    src: np.ndarray          # uint64 [E]
    dst: np.ndarray          # uint64 [E]
    weights: np.ndarray | None  # float32 [E] or None (unit weights)
    directed: bool
    n_nodes: int = 0         # node-index range the generator drew from
    meta: dict = field(default_factory=dict)

    @property
    def num_edges(self) -> int:
        return int(self.src.shape[0])


def undirected_rounds(E: int):
    """Candidate-batch sizes of the dedup loop: need + need/8 + 1024 while short of E."""
    return lambda need: need + need // 8 + 1024


def _sorted_unique(x: np.ndarray) -> np.ndarray:
    x = np.sort(x)
    if x.size == 0:
        return x
    keep = np.empty(x.size, dtype=bool)
    keep[0] = True
    np.not_equal(x[1:], x[:-1], out=keep[1:])
    return x[keep]


def chung_lu_undirected_idx(n: int, E: int, gamma: float, seed: int, max_deg: float,
                            max_rounds: int = 64):
    """Undirected simple power-law graph as sorted unique (u < v) index pairs.

    Rounds of candidates (counter range [c, c + m)) are drawn, self-loops dropped, each pair
    keyed as (min << 32) | max, and the union deduplicated until at least E distinct edges
    exist (the last round may overshoot; the actual count is returned).
    """
    if E > n * (n - 1) // 4:
        raise ValueError("too many edges requested for a simple graph on n nodes")
    i0 = solve_i0(n, gamma, 2 * E, max_deg)
    thr = cdf_thresholds(n, gamma, i0)
    keys = np.empty(0, dtype=U64)
    c = 0
    for _ in range(max_rounds):
        need = E - keys.shape[0]
        if need <= 0:
            break
        m = need + need // 8 + 1024
        cnt = np.arange(c, c + m, dtype=U64)
        c += m
        u = sample_nodes(thr, rng(seed, STREAM_SRC, cnt))
        v = sample_nodes(thr, rng(seed, STREAM_DST, cnt))
        keep = u != v
        a = np.minimum(u, v)[keep].astype(U64)
        b = np.maximum(u, v)[keep].astype(U64)
        keys = _sorted_unique(np.concatenate([keys, (a << U64(32)) | b]))
    u = (keys >> U64(32)).astype(np.int64)
    v = (keys & U64(0xFFFFFFFF)).astype(np.int64)
    return u, v, {"i0": i0, "rounds_counter_end": c}


def chung_lu_undirected(n: int, E: int, gamma: float, seed: int, max_deg: float) -> EdgeList:
    u, v, meta = chung_lu_undirected_idx(n, E, gamma, seed, max_deg)
    ids = node_ids(n, seed)
    return EdgeList(ids[u], ids[v], None, False, n, meta)


def lognormal_weights(seed: int, counter: np.ndarray) -> np.ndarray:
    """exp(N(0,1)) by Box-Muller on two 53-bit uniforms, rounded to float32."""
    u1 = ((rng(seed, STREAM_W1, counter) >> U64(11)).astype(np.float64) + 1.0) * 2.0 ** -53
    u2 = (rng(seed, STREAM_W2, counter) >> U64(11)).astype(np.float64) * 2.0 ** -53
    z = np.sqrt(-2.0 * np.log(u1)) * np.cos(2.0 * np.pi * u2)
    return np.exp(z).astype(np.float32)


def uniform_weights(seed: int, counter: np.ndarray, lo: float = 0.1, hi: float = 1.0) -> np.ndarray:
    """Uniform(lo, hi) weights from the top 53 bits, rounded to float32."""
    u = (rng(seed, STREAM_W1, counter) >> U64(11)).astype(np.float64) * 2.0 ** -53
    return (lo + (hi - lo) * u).astype(np.float32)


def chung_lu_directed(n: int, E: int, gamma: float, seed: int, max_deg: float,
                      weights: str | None = None) -> EdgeList:
    """Directed power-law multigraph: src and dst drawn independently; duplicates and
    self-loops are kept (the builder merges duplicates into edge multiplicities)."""
    i0 = solve_i0(n, gamma, E, max_deg)
    thr = cdf_thresholds(n, gamma, i0)
    cnt = np.arange(E, dtype=U64)
    u = sample_nodes(thr, rng(seed, STREAM_SRC, cnt))
    v = sample_nodes(thr, rng(seed, STREAM_DST, cnt))
    ids = node_ids(n, seed)
    w = None
    if weights == "lognormal":
        w = lognormal_weights(seed, cnt)
    elif weights == "uniform":
        w = uniform_weights(seed, cnt)
    elif weights is not None:
        raise ValueError(weights)
    return EdgeList(ids[u], ids[v], w, True, n, {"i0": i0})


# ---------------------------------------------------------------------------------------
# Small structured graphs (closed-form cases) and random multigraphs
# ---------------------------------------------------------------------------------------

def from_index_pairs(u, v, directed: bool, seed: int = 0, weights=None, n: int | None = None) -> EdgeList:
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    if n is None:
        n = int(max(u.max(initial=-1), v.max(initial=-1)) + 1)
    ids = node_ids(max(n, 1), seed)
    w = None if weights is None else np.asarray(weights, dtype=np.float32)
    return EdgeList(ids[u], ids[v], w, directed, n)


def random_multigraph(n: int, E: int, seed: int, directed: bool, weighted: bool,
                      self_loops: bool = True) -> EdgeList:
    """Uniform random endpoints with duplicates and (optionally) self-loops."""
    cnt = np.arange(E, dtype=U64)
    u = (rng(seed, STREAM_SRC, cnt) % U64(n)).astype(np.int64)
    v = (rng(seed, STREAM_DST, cnt) % U64(n)).astype(np.int64)
    if not self_loops:
        v = np.where(u == v, (v + 1) % n, v)
    w = uniform_weights(seed, cnt) if weighted else None
    return from_index_pairs(u, v, directed, seed, w, n)


def clique_edges(m: int, offset: int = 0, self_loops: bool = False):
    u, v = [], []
    for a in range(m):
        for b in range(a if self_loops else a + 1, m):
            u.append(offset + a)
            v.append(offset + b)
    return u, v


def disjoint_cliques(sizes, seed: int = 0, self_loops: bool = True) -> EdgeList:
    """Undirected disjoint union of cliques (optionally with a self-loop on every node)."""
    us, vs, off = [], [], 0
    for m in sizes:
        u, v = clique_edges(m, off, self_loops)
        us += u
        vs += v
        off += m
    return from_index_pairs(us, vs, False, seed, None, off)


def star(leaves: int, seed: int = 0) -> EdgeList:
    """Undirected star: node 0 is the hub."""
    return from_index_pairs([0] * leaves, list(range(1, leaves + 1)), False, seed, None, leaves + 1)


def complete_bipartite(m: int, k: int, seed: int = 0) -> EdgeList:
    """Undirected K_{m,k}: nodes 0..m-1 on one side, m..m+k-1 on the other."""
    u = [a for a in range(m) for _ in range(k)]
    v = [m + b for _ in range(m) for b in range(k)]
    return from_index_pairs(u, v, False, seed, None, m + k)


def circulant_regular(n: int, k: int, seed: int = 0) -> EdgeList:
    """Undirected 2k-regular circulant graph: i ~ i+1, ..., i+k (mod n), n > 2k."""
    u = [i for i in range(n) for s in range(1, k + 1)]
    v = [(i + s) % n for i in range(n) for s in range(1, k + 1)]
    return from_index_pairs(u, v, False, seed, None, n)


# ---------------------------------------------------------------------------------------
# Workload presets
# ---------------------------------------------------------------------------------------

@dataclass(frozen=True)
class PowerLawSpec:
    """A power-law graph workload (shape of the paper's social graphs, synthetic)."""
    name: str
    n: int
    edges: int
    gamma: float
    max_deg: float
    directed: bool
    weights: str | None
    d: int
    iters: int
    seed: int = 0

    def generate(self) -> EdgeList:
        if self.directed:
            return chung_lu_directed(self.n, self.edges, self.gamma, self.seed, self.max_deg,
                                     self.weights)
        if self.weights is not None:
            raise ValueError("undirected power-law preset is unit-weight")
        return chung_lu_undirected(self.n, self.edges, self.gamma, self.seed, self.max_deg)


# Small undirected case the oracle finishes in seconds (about 100k CSR entries).
SMALL = PowerLawSpec("chung_lu_10k_undirected_d128", 10_000, 50_000, 2.1, 1_000.0,
                     False, None, 128, 4)
# Mid-size weighted directed case (2M nodes, 40M edges, log-normal weights, d = 256).
MID = PowerLawSpec("chung_lu_2M_40M_directed_lognormal_d256", 2_000_000, 40_000_000, 2.1,
                   100_000.0, True, "lognormal", 256, 4)
# Large social-graph shape (41M nodes, 1.4B undirected edges, d = 128).  The degree target
# counts raw endpoint draws; 8.5M of them leave node 0 with ~3.0M distinct neighbours after
# deduplication (expected value sum_j 1 - exp(-lambda_0j)).
LARGE = PowerLawSpec("chung_lu_41M_1p4B_undirected_d128", 41_000_000, 1_400_000_000, 2.0,
                     8_500_000.0, False, None, 128, 4)


@dataclass(frozen=True)
class BatchGraphSpec:
    """One member of the batched workload: a small Chung-Lu graph with its own d and I."""
    n: int
    edges: int
    directed: bool
    d: int
    iters: int
    seed: int

    def generate(self) -> EdgeList:
        max_deg = max(4.0, 0.05 * 2 * self.edges)
        if self.directed:
            return chung_lu_directed(self.n, self.edges, 2.1, self.seed, max_deg, "uniform")
        u, v, meta = chung_lu_undirected_idx(self.n, self.edges, 2.1, self.seed, max_deg)
        cnt = np.arange(u.shape[0], dtype=U64)
        ids = node_ids(self.n, self.seed)
        return EdgeList(ids[u], ids[v], uniform_weights(self.seed, cnt), False, self.n, meta)


def batch_specs(count: int = 4096, seed: int = 0, n_lo: int = 50, n_hi: int = 50_000,
                dims=(64, 128, 256), iters=(3, 4, 5)):
    """Mixed small graphs: n log-uniform in [n_lo, n_hi], average degree U[4, 30],
    directed with probability 1/2, d and I drawn uniformly from the given sets."""
    cnt = np.arange(count, dtype=U64)
    r = [(rng(seed, 100 + k, cnt) >> U64(11)).astype(np.float64) * 2.0 ** -53 for k in range(5)]
    out = []
    for g in range(count):
        n = int(round(math.exp(math.log(n_lo) + r[0][g] * (math.log(n_hi) - math.log(n_lo)))))
        avg_deg = 4.0 + 26.0 * r[1][g]
        directed = bool(r[2][g] < 0.5)
        e = max(1, int(n * avg_deg / (1 if directed else 2)))
        e = min(e, n * (n - 1) // 4) if not directed else e
        d = dims[min(int(r[3][g] * len(dims)), len(dims) - 1)]
        it = iters[min(int(r[4][g] * len(iters)), len(iters) - 1)]
        out.append(BatchGraphSpec(n, e, directed, d, it, seed * 1_000_003 + g + 1))
    return out
