"""Pins of the oracle's walk sampler (the local walk of Algorithms 2-3):
cumulative weights against numpy, the pair enumeration by brute force, every
step an arc, weight-proportional transitions and roots (chi-square), dead
ends, and the window-1 pairs against the Philox words computed one by one."""
import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I


def chi2_ok(counts, probs, n):
    from scipy.stats import chisquare
    exp = np.asarray(probs) * n
    return chisquare(counts, exp).pvalue > 1e-3


def test_cumulative_weights_per_node():
    g = I.chung_lu_directed(n=300, m=3000, seed=2)
    cw = O.walk_cumw(g)
    for v in range(g.n_nodes):
        lo, hi = np.searchsorted(g.src, v), np.searchsorted(g.src, v, side="right")
        np.testing.assert_array_equal(cw[lo:hi], np.cumsum(g.w[lo:hi].astype(np.float64)))


@pytest.mark.parametrize("L,W", [(1, 1), (5, 1), (5, 2), (7, 3), (100, 2), (4, 4)])
def test_pair_count_and_order(L, W):
    pairs = [(i, i + k) for i in range(L) for k in range(1, W + 1) if i + k <= L]
    assert O.walk_pairs_per_walk(L, W) == len(pairs)


def _walk_nodes_from_records(rec, L, W):
    """Rebuild a walk's nodes from its records (pairs in (i, k) order)."""
    nodes = {}
    p = 0
    for i in range(L):
        for k in range(1, W + 1):
            if i + k > L:
                continue
            nodes.setdefault(i, rec[p, 0])
            assert nodes[i] == rec[p, 0]
            nodes.setdefault(i + k, rec[p, 1])
            assert nodes[i + k] == rec[p, 1]
            p += 1
    return [nodes[i] for i in range(L + 1)]


def test_walk_steps_are_arcs_and_pairs_are_consistent():
    g = I.tiny_chung_lu()
    T, cw = O.Tables(g), O.walk_cumw(g)
    arcs = set(zip(g.src.tolist(), g.dst.tolist()))
    L, W = 30, 2
    P = O.walk_pairs_per_walk(L, W)
    rec = O.sample_walk(T, cw, 5, 0, 4 * P, 3, L, W)
    for wk in range(4):
        nodes = _walk_nodes_from_records(rec[wk * P:(wk + 1) * P], L, W)
        for a, b in zip(nodes[:-1], nodes[1:]):
            assert (a, b) in arcs
    # the chunking of the sample range does not matter
    part = np.concatenate([O.sample_walk(T, cw, 5, t, 37, 3, L, W) for t in range(0, 4 * P - 36, 37)])
    np.testing.assert_array_equal(part, rec[:len(part)])


def test_window_one_walk_of_length_one_is_the_weighted_root_arc():
    g = I.chung_lu_directed(n=200, m=2000, seed=3)
    T, cw = O.Tables(g), O.walk_cumw(g)
    rec = O.sample_walk(T, cw, 77, 1000, 50, 2, 1, 1)
    for t in range(50):
        wd = O.philox([(1000 + t) & 0xFFFFFFFF, (1000 + t) >> 32, 0, 8], [77, 0])
        e = O.alias_draw(T.thr_e, T.alias_e, int(wd[0]), int(wd[1]), int(wd[2]))
        assert (rec[t, 0], rec[t, 1]) == (g.src[e], g.dst[e])


def test_transitions_and_roots_follow_the_weights():
    # a star-like weighted graph: node 0 -> 1, 2, 3 with weights 1, 2, 5 (and back)
    src = np.array([0, 0, 0, 1, 2, 3])
    dst = np.array([1, 2, 3, 0, 0, 0])
    w = np.array([1.0, 2.0, 5.0, 1.0, 2.0, 5.0])
    g = I.canonicalize(4, src, dst, w, symmetrize=False)
    T, cw = O.Tables(g), O.walk_cumw(g)
    L, W = 2, 1
    n = 40_000
    rec = O.sample_walk(T, cw, 9, 0, 2 * n, 0, L, W)
    # pair 1 of each walk is (nodes[1], nodes[2]); whenever nodes[1] == 0 the
    # step from node 0 picks 1, 2, 3 with probability 1/8, 2/8, 5/8
    second = rec[1::2]
    from0 = second[second[:, 0] == 0, 1]
    counts = np.bincount(from0, minlength=4)[1:]
    assert len(from0) > 10_000 and chi2_ok(counts, [1 / 8, 2 / 8, 5 / 8], len(from0))
    # roots: arcs by weight (total 16)
    first = rec[0::2]
    keys = first[:, 0] * 4 + first[:, 1]
    arcs = g.src.astype(np.int64) * 4 + g.dst
    counts = np.array([(keys == a).sum() for a in arcs])
    assert chi2_ok(counts, g.w / g.w.sum(), n)


def test_dead_end_steps_back():
    # 0 -> 1 -> 2, node 2 has no out-arcs
    g = I.canonicalize(3, np.array([0, 1]), np.array([1, 2]), None, symmetrize=False)
    T, cw = O.Tables(g), O.walk_cumw(g)
    L, W = 6, 1
    rec = O.sample_walk(T, cw, 1, 0, 3 * L, 0, L, W)
    for wk in range(3):
        nodes = _walk_nodes_from_records(rec[wk * L:(wk + 1) * L], L, W)
        for a, b, c in zip(nodes[:-2], nodes[1:-1], nodes[2:]):
            if b == 2:
                assert c == a  # back to where it came from
            else:
                assert (b, c) in {(0, 1), (1, 2)}


def test_walk_training_differs_from_edge_training_and_is_deterministic():
    g = I.tiny_chung_lu()
    T, cw = O.Tables(g), O.walk_cumw(g)
    runs = []
    for _ in range(2):
        U = O.init_uniform(g.n_nodes, 8, 1)
        C = np.zeros_like(U)
        O.train(T, U, C, order=2, K=3, n_samples=5000, seed=4, batch=128, walk=(cw, 20, 2))
        runs.append((U, C))
    np.testing.assert_array_equal(runs[0][0], runs[1][0])
    U = O.init_uniform(g.n_nodes, 8, 1)
    C = np.zeros_like(U)
    O.train(T, U, C, order=2, K=3, n_samples=5000, seed=4, batch=128)
    assert not np.array_equal(U, runs[0][0])


def test_reuse_replays_each_walk_and_keeps_the_negatives():
    """With reuse r, the r passes over a walk repeat the positive pairs of
    that walk (as drawn without reuse at the walk's own index), and the
    negatives stay the edge sampler's at each sample's counter."""
    g = I.tiny_chung_lu()
    T, cw = O.Tables(g), O.walk_cumw(g)
    L, W, r, K = 12, 3, 3, 4
    P = O.walk_pairs_per_walk(L, W)
    n_walks = 5
    one = O.sample_walk(T, cw, 21, 0, n_walks * P, K, L, W)
    rec = O.sample_walk(T, cw, 21, 0, n_walks * r * P, K, L, W, reuse=r)
    for wk in range(n_walks):
        for q in range(r):
            blk = rec[(wk * r + q) * P:(wk * r + q + 1) * P]
            np.testing.assert_array_equal(blk[:, :2], one[wk * P:(wk + 1) * P, :2])
    negs = O.sample(T, 21, 0, n_walks * r * P, K)
    np.testing.assert_array_equal(rec[:, 2:], negs[:, 2:])
    # reuse 1 is the plain walk sampler; a window starting mid-pass agrees
    np.testing.assert_array_equal(O.sample_walk(T, cw, 21, 0, 50, K, L, W, reuse=1), one[:50])
    np.testing.assert_array_equal(O.sample_walk(T, cw, 21, 2 * P + 5, 40, K, L, W, reuse=r),
                                  rec[2 * P + 5:2 * P + 45])
