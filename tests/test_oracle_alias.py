"""Pins of the oracle's random streams and alias tables (no GPU).

Philox is pinned by the published known-answer vectors; the alias tables by
hand-derived cases, exact integer invariants (the implied probability of every
item equals its integer mass), brute-force enumeration of the draw on tiny
tables, and chi-square tests of sampled frequencies against Eq. 1 and the
weight-proportional edge pick of Algorithm 3.
"""
import math
import os

import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
Q = 1 << 32


def _read_cases(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append(line)
    return rows


def test_philox_known_answers():
    for line in _read_cases("philox4x32_10_kat.txt"):
        words = [int(x, 16) for x in line.split()]
        ctr, key, want = words[0:4], words[4:6], words[6:10]
        assert list(O.philox(ctr, key)) == want


def test_alias_hand_cases():
    for line in _read_cases("alias_cases.txt"):
        name, xs, ms, thrs, als = [p.strip() for p in line.split("|")]
        x = np.array([float(v) for v in xs.split()])
        m, thr, alias = O.alias_build(x)
        assert list(m) == [int(v) for v in ms.split()], name
        assert list(thr) == [int(v) for v in thrs.split()], name
        assert list(alias) == [int(v) for v in als.split()], name


def test_fixed_sum_order():
    # blocks of 1024 reduced by halving strides: [1e16, 1, -1e16, 1] pairs
    # (1e16 + -1e16) and (1 + 1) first, giving 2; a left-to-right sum gives 1.
    assert O.fixed_sum(np.array([1e16, 1.0, -1e16, 1.0])) == 2.0
    rng = np.random.default_rng(1)
    for n in [1, 2, 1023, 1024, 1025, 5000, 1 << 20]:
        x = rng.random(n)
        assert abs(O.fixed_sum(x) - math.fsum(x)) <= 1e-13 * math.fsum(x)


def implied_masses(thr, alias):
    """Mass each item receives from the table: thr from its own bucket plus
    (2^32 - thr) from every bucket that aliases it."""
    n = thr.size
    got = np.zeros(n, np.uint64)
    np.add.at(got, np.arange(n), thr.astype(np.uint64))
    np.add.at(got, alias.astype(np.int64), np.uint64(Q) - thr.astype(np.uint64))
    return got


def _weights(kind, n, rng):
    if kind == "uniform":
        return np.ones(n)
    if kind == "random":
        return rng.random(n)
    if kind == "zeros":
        x = rng.random(n)
        x[rng.random(n) < 0.4] = 0.0
        if not x.any():
            x[0] = 1.0
        return x
    if kind == "powerlaw":
        return (np.arange(n) + 1.0) ** -1.2
    if kind == "range":
        return 10.0 ** rng.uniform(-12, 12, n)
    if kind == "integer":
        return rng.integers(1, 50, n).astype(np.float64)
    raise ValueError(kind)


@pytest.mark.parametrize("kind", ["uniform", "random", "zeros", "powerlaw", "range", "integer"])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 1023, 1024, 1025, 4097, 50000])
def test_alias_invariants(kind, n):
    rng = np.random.default_rng(n * 31 + len(kind))
    x = _weights(kind, n, rng)
    m, thr, alias = O.alias_build(x)
    # masses sum to exactly n * 2^32 and are realised exactly by the table
    assert int(m.sum(dtype=np.uint64)) == n * Q
    assert np.array_equal(implied_masses(thr, alias), m)
    # masses approximate x / W: floor + remainder + FP error of S and W
    W = math.fsum(x)
    exact = x / W * (n * float(Q))
    slack = 2.0 + 1e-13 * exact + (int(n * Q - int(np.floor(x * (n * Q / W)).sum())) // max(1, int((x > 0).sum())))
    assert np.all(np.abs(m.astype(np.float64) - exact) <= slack)
    # zero-weight items get no mass, are never an alias target
    zero = x == 0
    assert np.all(m[zero] == 0)
    assert not np.isin(np.flatnonzero(zero), alias[~zero]).any()
    assert np.all(thr[zero] == 0)
    # alias targets are heavy items (m > 2^32) or self
    heavy = m > np.uint64(Q)
    tgt = alias[alias != np.arange(n)]
    assert np.all(heavy[tgt])


def test_alias_draw_enumeration():
    """Brute force: every bucket i, and both sides of its coin threshold."""
    rng = np.random.default_rng(5)
    for n in [1, 2, 3, 5, 6]:
        x = rng.integers(0, 4, n).astype(np.float64)
        if not x.any():
            x[-1] = 1
        m, thr, alias = O.alias_build(x)
        got = np.zeros(n, dtype=object)
        for i in range(n):
            # smallest 64-bit r with floor(r * n / 2^64) == i
            r = -((-i << 64) // n)
            w0, w1 = r & 0xFFFFFFFF, r >> 32
            assert ((r * n) >> 64) == i
            if thr[i] > 0:
                assert O.alias_draw(thr, alias, w0, w1, int(thr[i]) - 1) == i
            if thr[i] < 0xFFFFFFFF:
                assert O.alias_draw(thr, alias, w0, w1, int(thr[i])) == alias[i]
            assert O.alias_draw(thr, alias, w0, w1, 0xFFFFFFFF) == alias[i]
            got[i] += int(thr[i])
            got[alias[i]] += Q - int(thr[i])
        assert list(got) == [int(v) for v in m]
        # probabilities equal x / W to within 2 / (n 2^32)
        p = np.array([int(v) for v in got], dtype=np.float64) / (n * Q)
        assert np.all(np.abs(p - x / x.sum()) <= 2.0 / (n * Q) + 1e-15)


def _chi2_pvalue(obs, exp):
    from scipy import stats
    keep = exp > 0
    assert obs[~keep].sum() == 0
    chi = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    return stats.chi2.sf(chi, keep.sum() - 1)


def test_sample_frequencies_match_eq1_and_edge_weights():
    g = I.chung_lu_undirected(200, 2.1, 1500.0, seed=3)
    T = O.Tables(g)
    K = 5
    cnt = 200_000
    rec = O.sample(T, seed=11, t0=0, count=cnt, K=K)
    # negatives ~ q(v) = d(v)^0.75 / sum (Eq. 1), d = out-degree (unit weights)
    deg = np.bincount(g.src, minlength=g.n_nodes).astype(np.float64)
    q = deg ** 0.75 / (deg ** 0.75).sum()
    neg = np.bincount(rec[:, 2:].ravel(), minlength=g.n_nodes)
    assert _chi2_pvalue(neg.astype(np.float64), q * neg.sum()) > 1e-3
    # positives: arcs drawn in proportion to weight -> (u, v) pair counts
    key = rec[:, 0].astype(np.int64) * g.n_nodes + rec[:, 1]
    arc_key = g.src.astype(np.int64) * g.n_nodes + g.dst
    assert np.isin(key, arc_key).all()
    pos = np.bincount(np.searchsorted(arc_key, key), minlength=g.n_arcs).astype(np.float64)
    assert _chi2_pvalue(pos, g.w / g.w.sum() * cnt) > 1e-3


def test_weighted_degree_and_pow():
    g = I.chung_lu_directed(n=3000, m=40000, seed=2)
    x = O.neg_weights(g)
    d = np.bincount(g.src, weights=g.w.astype(np.float64), minlength=g.n_nodes)
    ref = np.power(d, 0.75)
    assert np.all(np.abs(x - ref) <= 4 * np.spacing(np.maximum(ref, 1e-300)))
    assert np.all(x[d == 0] == 0)


def test_sample_draw_layout():
    """call 0 picks the arc, calls 1..K the negatives, counters (t_lo, t_hi, call, domain)."""
    g = I.chung_lu_undirected(100, 2.1, 600.0, seed=1)
    T = O.Tables(g)
    seed, t0 = 0x1234_5678_9ABC_DEF0, (5 << 32) + 17
    rec = O.sample(T, seed=seed, t0=t0, count=3, K=2, domain=4)
    key = [seed & 0xFFFFFFFF, seed >> 32]
    for i in range(3):
        t = t0 + i
        w = O.philox([t & 0xFFFFFFFF, t >> 32, 0, 4], key)
        e = O.alias_draw(T.thr_e, T.alias_e, int(w[0]), int(w[1]), int(w[2]))
        assert rec[i, 0] == g.src[e] and rec[i, 1] == g.dst[e]
        for j in (1, 2):
            w = O.philox([t & 0xFFFFFFFF, t >> 32, j, 4], key)
            assert rec[i, 1 + j] == O.alias_draw(T.thr_n, T.alias_n, int(w[0]), int(w[1]), int(w[2]))
