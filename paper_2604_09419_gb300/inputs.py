"""Seeded synthetic graph generators (inputs only).

This module produces the graphs that both the CUDA path and the FP64 oracle
consume.  It holds none of the method's arithmetic: no alias tables, no
sampling of training pairs, no embedding updates.  Its random numbers come
from SplitMix64 (Steele, Lea and Flood, OOPSLA 2014), used as a counter-based
hash so that every generated graph is a pure function of its parameters and
seed, identical on x86 and Arm and across NumPy versions.

Graphs are returned in canonical form, the form the library's
``line_build_alias`` expects:

* directed arcs ``(src[e], dst[e], w[e])``, ``w > 0``;
* an undirected edge is stored as two arcs;
* self-loops are dropped and duplicate arcs merged by summing their weights;
* arcs sorted by ``(src, dst)``, so ``src`` is non-decreasing (CSR order, the
  binary CSR layout of the paper's Section V-A).

Workload shapes follow the synthetic stand-ins for the paper's datasets
(Table II spans 7.5K-111M vertices and 89K-6.4B edges):

* ``chung_lu_undirected`` - tiny power-law graph (1,000 nodes, exponent 2.1);
* ``rmat`` - R-MAT with (a,b,c,d) = (.57,.19,.19,.05), edge factor 16,
  symmetrised, duplicates merged into integer weights;
* ``chung_lu_directed`` - weighted directed graph, power-law out-weights
  (exponent 2.2), uniform in-endpoints, lognormal(0,1) arc weights.
"""
from __future__ import annotations

import dataclasses
import os

import numpy as np

__all__ = [
    "Graph",
    "splitmix64",
    "uniform01",
    "canonicalize",
    "chung_lu_undirected",
    "rmat",
    "chung_lu_directed",
    "tiny_chung_lu",
    "rmat20",
    "split_edges",
    "non_edges",
    "hold_out_nodes",
]

_GOLDEN = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)

# stream identifiers keep the draws of different generators independent
STREAM_CHUNG_LU = 5
STREAM_RMAT = 6
STREAM_DIRECTED = 7
STREAM_SPLIT = 8
STREAM_NON_EDGE = 9
STREAM_NODE_SPLIT = 10


@dataclasses.dataclass
class Graph:
    """A canonical arc list (see the module docstring)."""

    n_nodes: int
    src: np.ndarray  # int32, non-decreasing
    dst: np.ndarray  # int32
    w: np.ndarray  # float32, > 0
    directed: bool
    name: str = ""

    @property
    def n_arcs(self) -> int:
        return int(self.src.shape[0])

    def row_ptr(self) -> np.ndarray:
        """CSR row pointer (int64, n_nodes + 1) derived from the sorted src."""
        return np.searchsorted(self.src, np.arange(self.n_nodes + 1, dtype=np.int64),
                               side="left").astype(np.int64)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 output function applied element-wise to uint64 state values."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + _GOLDEN
        z = (z ^ (z >> np.uint64(30))) * _M1
        z = (z ^ (z >> np.uint64(27))) * _M2
        return z ^ (z >> np.uint64(31))


def _hash(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """64 random bits for each counter value of one (seed, stream) pair."""
    base = splitmix64(np.array([(seed * 0x10001 + stream) & 0xFFFFFFFFFFFFFFFF], dtype=np.uint64))[0]
    with np.errstate(over="ignore"):
        return splitmix64(np.asarray(counter, dtype=np.uint64) * _GOLDEN + base)


def uniform01(seed: int, stream: int, counter: np.ndarray) -> np.ndarray:
    """Uniform doubles in [0, 1) with 53 random bits, one per counter value."""
    h = _hash(seed, stream, counter)
    return (h >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def canonicalize(n_nodes: int, src: np.ndarray, dst: np.ndarray, w: np.ndarray | None,
                 symmetrize: bool, name: str = "") -> Graph:
    """Drop self-loops, optionally add reverse arcs, merge duplicates, sort by (src, dst)."""
    src = np.asarray(src, dtype=np.int64)
    dst = np.asarray(dst, dtype=np.int64)
    keep = src != dst
    src, dst = src[keep], dst[keep]
    if w is not None:
        w = np.asarray(w, dtype=np.float64)[keep]
    if symmetrize:
        src, dst = np.concatenate([src, dst]), np.concatenate([dst, src])
        if w is not None:
            w = np.concatenate([w, w])
    key = src * np.int64(n_nodes) + dst
    if w is None:
        uk, counts = np.unique(key, return_counts=True)
        wm = counts.astype(np.float64)
    else:
        order = np.argsort(key, kind="stable")
        key = key[order]
        w = w[order]
        starts = np.flatnonzero(np.concatenate([[True], key[1:] != key[:-1]])) if key.size else np.zeros(0, np.int64)
        uk = key[starts]
        wm = np.add.reduceat(w, starts) if key.size else np.zeros(0)
    s = (uk // n_nodes).astype(np.int32)
    d = (uk % n_nodes).astype(np.int32)
    return Graph(int(n_nodes), s, d, wm.astype(np.float32), directed=not symmetrize, name=name)


def chung_lu_undirected(n: int = 1000, gamma: float = 2.1, n_edges: float = 10000.0,
                        seed: int = 0) -> Graph:
    """Undirected Chung-Lu graph with unit weights.

    Expected degree weights ``w_i ∝ (i+1)^(-1/(gamma-1))``; every pair
    ``i<j`` is an edge independently with probability
    ``min(1, w_i w_j / sum(w))`` (exact O(n^2) Bernoulli draws).  The weights
    are scaled (by bisection) so that the expected edge count, clipping
    included, equals ``n_edges``.
    """
    i = np.arange(n, dtype=np.float64)
    base = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    a, b = np.triu_indices(n, k=1)

    def probs(scale):
        wt = base * scale
        return np.minimum(1.0, wt[a] * wt[b] / wt.sum())

    lo, hi = 0.0, 4.0 * n_edges / base.sum()
    while probs(hi).sum() < n_edges:
        hi *= 2.0
    for _ in range(60):
        mid = 0.5 * (lo + hi)
        if probs(mid).sum() < n_edges:
            lo = mid
        else:
            hi = mid
    p = probs(hi)
    u = uniform01(seed, STREAM_CHUNG_LU, a.astype(np.uint64) * np.uint64(n) + b.astype(np.uint64))
    hit = u < p
    return canonicalize(n, a[hit], b[hit], None, symmetrize=True,
                        name=f"chung_lu_n{n}_g{gamma}_m{int(n_edges)}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, abcd=(0.57, 0.19, 0.19, 0.05), seed: int = 0,
         symmetrize: bool = True) -> Graph:
    """R-MAT graph: ``edge_factor * 2^scale`` draws of ``scale`` recursive quadrant picks.

    Each level uses 16 random bits compared against the cumulative quadrant
    probabilities (quantised to 1/65536).  Quadrant ``a`` keeps both bits 0,
    ``b`` sets the destination bit, ``c`` the source bit, ``d`` both.  The
    draws are symmetrised, self-loops dropped and duplicates merged into
    integer weights.  Vertex labels are not permuted.
    """
    n = 1 << scale
    m = edge_factor * n
    a, b, c, _ = abcd
    ta = np.uint64(int(round(a * 65536)))
    tb = np.uint64(int(round((a + b) * 65536)))
    tc = np.uint64(int(round((a + b + c) * 65536)))
    src = np.zeros(m, dtype=np.int64)
    dst = np.zeros(m, dtype=np.int64)
    draw = np.arange(m, dtype=np.uint64)
    words = (scale + 3) // 4
    level = 0
    for wi in range(words):
        h = _hash(seed, STREAM_RMAT, draw * np.uint64(words) + np.uint64(wi))
        for q in range(4):
            if level >= scale:
                break
            u = (h >> np.uint64(16 * q)) & np.uint64(0xFFFF)
            bit = np.int64(1) << np.int64(scale - 1 - level)
            sbit = u >= tb  # quadrants c and d
            dbit = ((u >= ta) & (u < tb)) | (u >= tc)  # quadrants b and d
            src |= np.where(sbit, bit, 0)
            dst |= np.where(dbit, bit, 0)
            level += 1
    return canonicalize(n, src, dst, None, symmetrize=symmetrize,
                        name=f"rmat{scale}_ef{edge_factor}_s{seed}")


def chung_lu_directed(n: int = 1 << 22, m: int = 1 << 26, gamma: float = 2.2,
                      seed: int = 0) -> Graph:
    """Weighted directed Chung-Lu graph.

    ``m`` arc draws; the source of each is drawn with probability proportional
    to ``(i+1)^(-1/(gamma-1))`` (power-law out-weights), the destination
    uniformly.  Each draw carries a lognormal(0,1) weight (Box-Muller); self
    loops are dropped and duplicates merged by summing weights.
    """
    i = np.arange(n, dtype=np.float64)
    wt = (i + 1.0) ** (-1.0 / (gamma - 1.0))
    cdf = np.cumsum(wt)
    cdf /= cdf[-1]
    draw = np.arange(m, dtype=np.uint64)
    u0 = uniform01(seed, STREAM_DIRECTED, draw * np.uint64(4))
    src = np.minimum(np.searchsorted(cdf, u0, side="right"), n - 1)
    del u0
    h = _hash(seed, STREAM_DIRECTED, draw * np.uint64(4) + np.uint64(1))
    dst = ((h >> np.uint64(32)) * np.uint64(n)) >> np.uint64(32)
    del h
    u1 = uniform01(seed, STREAM_DIRECTED, draw * np.uint64(4) + np.uint64(2))
    u2 = uniform01(seed, STREAM_DIRECTED, draw * np.uint64(4) + np.uint64(3))
    z = np.sqrt(-2.0 * np.log1p(-u1)) * np.cos(2.0 * np.pi * u2)
    del u1, u2
    w = np.exp(z)
    return canonicalize(n, src, dst.astype(np.int64), w, symmetrize=False,
                        name=f"dchung_lu_n{n}_m{m}_g{gamma}_s{seed}")


def _cached(name: str, fn):
    cache = os.environ.get("LINE_GRAPH_CACHE", "")
    if not cache:
        return fn()
    os.makedirs(cache, exist_ok=True)
    path = os.path.join(cache, name + ".npz")
    if os.path.exists(path):
        z = np.load(path)
        return Graph(int(z["n"]), z["src"], z["dst"], z["w"], bool(z["directed"]), name)
    g = fn()
    np.savez(path, n=g.n_nodes, src=g.src, dst=g.dst, w=g.w, directed=g.directed)
    return g


def tiny_chung_lu(seed: int = 0) -> Graph:
    """1,000-node undirected Chung-Lu graph, exponent 2.1, ~10,000 edges."""
    return chung_lu_undirected(1000, 2.1, 10000.0, seed)


def rmat20(seed: int = 0) -> Graph:
    """R-MAT scale 20, edge factor 16, symmetrised, integer weights."""
    return _cached(f"rmat20_s{seed}", lambda: rmat(20, 16, seed=seed))


def split_edges(g: Graph, frac: float = 0.1, seed: int = 0):
    """Hold out ``frac`` of the undirected edges (both arcs) of a symmetric graph.

    Returns ``(train_graph, held_src, held_dst)`` where the held-out pairs are
    listed once with ``src < dst``.
    """
    lo = np.minimum(g.src, g.dst).astype(np.uint64)
    hi = np.maximum(g.src, g.dst).astype(np.uint64)
    u = uniform01(seed, STREAM_SPLIT, lo * np.uint64(g.n_nodes) + hi)
    held = u < frac
    keep = ~held
    train = Graph(g.n_nodes, g.src[keep], g.dst[keep], g.w[keep], g.directed, g.name + "_train")
    once = held & (g.src < g.dst)
    return train, g.src[once].copy(), g.dst[once].copy()


def non_edges(g: Graph, count: int, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """``count`` uniform node pairs ``u != v`` that are not arcs of ``g``.

    Pairs are drawn in counter order from one SplitMix64 stream and rejected
    when ``u == v`` or ``(u, v)`` is an arc of ``g`` (for a symmetric graph that
    also excludes ``(v, u)``); the first ``count`` accepted pairs are returned,
    so the result is a pure function of ``(g, count, seed)``.  These are the
    negative pairs of a link-prediction AUC.
    """
    n = np.uint64(g.n_nodes)
    arcs = np.sort(g.src.astype(np.uint64) * n + g.dst.astype(np.uint64))
    out_u, out_v = [], []
    have, ctr = 0, 0
    while have < count:
        m = max(2 * (count - have), 1024)
        c = np.arange(ctr, ctr + m, dtype=np.uint64)
        ctr += m
        u = (_hash(seed, STREAM_NON_EDGE, 2 * c) % n).astype(np.int64)
        v = (_hash(seed, STREAM_NON_EDGE, 2 * c + np.uint64(1)) % n).astype(np.int64)
        key = u.astype(np.uint64) * n + v.astype(np.uint64)
        pos = np.searchsorted(arcs, key)
        hit = (pos < arcs.size) & (arcs[np.minimum(pos, max(arcs.size - 1, 0))] == key) if arcs.size else np.zeros(m, bool)
        ok = (u != v) & ~hit
        take = min(count - have, int(ok.sum()))
        out_u.append(u[ok][:take])
        out_v.append(v[ok][:take])
        have += take
    return (np.concatenate(out_u).astype(np.int32) if out_u else np.zeros(0, np.int32),
            np.concatenate(out_v).astype(np.int32) if out_v else np.zeros(0, np.int32))


def hold_out_nodes(g: Graph, frac: float = 0.1, seed: int = 0) -> tuple[np.ndarray, Graph]:
    """Hold out ``frac`` of the nodes: returns ``(held, graph)``, ``held`` a
    boolean mask over nodes and ``graph`` the arcs of ``g`` with neither
    endpoint held (same node count, so the held nodes are isolated)."""
    held = uniform01(seed, STREAM_NODE_SPLIT, np.arange(g.n_nodes, dtype=np.uint64)) < frac
    keep = ~held[g.src] & ~held[g.dst]
    return held, Graph(g.n_nodes, g.src[keep], g.dst[keep], g.w[keep], g.directed, g.name + "_kept")
