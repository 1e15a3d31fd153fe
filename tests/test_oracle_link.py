"""Pins of the link-prediction oracle (cosine scores, Mann-Whitney AUC) and of
the non-edge generator, none of which reuse the oracle's own formulas."""
import numpy as np
import pytest

from oracle import link as OL
from paper_2604_09419_gb300 import inputs as I


def brute_auc(pos, neg):
    s = 0.0
    for p in pos:
        for q in neg:
            s += 1.0 if p > q else (0.5 if p == q else 0.0)
    return s / (len(pos) * len(neg))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_mann_whitney_equals_brute_force_with_ties(seed):
    rng = np.random.default_rng(seed)
    pos = rng.integers(0, 6, 37).astype(np.float32)  # many ties
    neg = rng.integers(0, 6, 23).astype(np.float32)
    assert OL.mann_whitney(pos, neg) == pytest.approx(brute_auc(pos, neg), abs=1e-15)
    less, eq = OL.mann_whitney_counts(pos, neg)
    assert less == sum(int(q < p) for p in pos for q in neg)
    assert eq == sum(int(q == p) for p in pos for q in neg)


def test_mann_whitney_matches_scipy_u_statistic():
    stats = pytest.importorskip("scipy.stats")
    rng = np.random.default_rng(7)
    pos = np.round(rng.normal(0.3, 1, 400), 1)
    neg = np.round(rng.normal(0.0, 1, 300), 1)
    u = stats.mannwhitneyu(pos, neg, alternative="two-sided", method="asymptotic").statistic
    assert OL.mann_whitney(pos, neg) == pytest.approx(u / (400 * 300), abs=1e-12)


def test_mann_whitney_closed_forms():
    assert OL.mann_whitney([2.0, 3.0], [0.0, 1.0]) == 1.0
    assert OL.mann_whitney([0.0, 1.0], [2.0, 3.0]) == 0.0
    assert OL.mann_whitney([1.0] * 5, [1.0] * 7) == 0.5
    rng = np.random.default_rng(3)
    a, b = rng.normal(size=50), rng.normal(size=60)
    assert OL.mann_whitney(a, b) + OL.mann_whitney(b, a) == pytest.approx(1.0, abs=1e-14)


def test_pair_scores_single_order_plain_dot_and_cosine():
    rng = np.random.default_rng(0)
    U = rng.normal(size=(20, 8))
    s, d = np.arange(10), np.arange(10, 20)
    want = [float(U[i] @ U[j] / (np.linalg.norm(U[i]) * np.linalg.norm(U[j]))) for i, j in zip(s, d)]
    np.testing.assert_allclose(OL.pair_scores([U], s, d, "cosine"), want, rtol=0, atol=1e-14)
    want = [sum(U[i, k] * U[j, k] for k in range(8)) for i, j in zip(s, d)]
    np.testing.assert_allclose(OL.pair_scores([U], s, d), want, rtol=0, atol=1e-13)
    # concatenation: the dot of two orders is the sum of the dots
    V = rng.normal(size=(20, 3))
    np.testing.assert_allclose(OL.pair_scores([U, V], s, d), OL.pair_scores([U], s, d) + OL.pair_scores([V], s, d),
                               rtol=0, atol=1e-13)


def test_pair_scores_cosine_concatenation_cases():
    # node 0 and 1: equal order-1 rows, opposite order-2 rows -> 1/2 (1 + -1) = 0
    U1 = np.array([[1.0, 0.0], [3.0, 0.0], [0.0, 0.0]])
    U2 = np.array([[0.0, 2.0, 0.0], [0.0, -5.0, 0.0], [1.0, 0.0, 0.0]])
    assert OL.pair_scores([U1, U2], [0], [1], "cosine")[0] == pytest.approx(0.0, abs=1e-15)
    # node 2 has a zero order-1 row: its vector is (0, 0 | 1, 0, 0), norm 1;
    # node 0 is (1, 0 | 0, 1, 0), norm sqrt(2); dot = 0
    assert OL.pair_scores([U1, U2], [0], [2], "cosine")[0] == pytest.approx(0.0, abs=1e-15)
    # equal order-2 directions, orthogonal order-1 directions: 1/2
    V1 = np.array([[1.0, 0.0], [0.0, 4.0]])
    V2 = np.array([[1.0, 1.0, 0.0], [2.0, 2.0, 0.0]])
    assert OL.pair_scores([V1, V2], [0], [1], "cosine")[0] == pytest.approx(0.5, abs=1e-15)
    # an all-zero node scores 0 with anything
    Z = np.zeros((2, 4))
    Z[1] = 1.0
    assert OL.pair_scores([Z], [0], [1], "cosine")[0] == 0.0
    # scale invariance per order
    rng = np.random.default_rng(1)
    A, B = rng.normal(size=(6, 4)), rng.normal(size=(6, 5))
    s1 = OL.pair_scores([A, B], [0, 1, 2], [3, 4, 5], "cosine")
    s2 = OL.pair_scores([A * 7.0, B * 0.1], [0, 1, 2], [3, 4, 5], "cosine")
    np.testing.assert_allclose(s1, s2, rtol=0, atol=1e-14)


def test_non_edges_are_non_edges_and_deterministic():
    g = I.tiny_chung_lu()
    u, v = I.non_edges(g, 5000, seed=3)
    assert len(u) == 5000 and (u != v).all()
    arcs = set(zip(g.src.tolist(), g.dst.tolist()))
    assert not any((a, b) in arcs for a, b in zip(u.tolist(), v.tolist()))
    u2, v2 = I.non_edges(g, 5000, seed=3)
    assert (u == u2).all() and (v == v2).all()
    # a prefix of a longer draw
    u3, v3 = I.non_edges(g, 100, seed=3)
    assert (u3 == u[:100]).all() and (v3 == v[:100]).all()


def test_trained_embeddings_separate_held_out_edges():
    """The oracle's own training, on the tiny graph with 10% of edges held
    out, ranks held-out edges above random non-edges (a sanity check of the
    evaluation as a whole, not a pin of one formula)."""
    from oracle import Tables, init_uniform, train
    g = I.tiny_chung_lu()
    tr, hs, hd = I.split_edges(g, 0.1, seed=0)
    ns, nd = I.non_edges(g, len(hs), seed=0)
    T = Tables(tr)
    U = init_uniform(g.n_nodes, 16, 1)
    C = np.zeros_like(U)
    train(T, U, C, order=2, K=5, n_samples=200_000, seed=1, batch=256)
    a = OL.auc([U], hs, hd, ns, nd)
    U0 = init_uniform(g.n_nodes, 16, 1)
    a0 = OL.auc([U0], hs, hd, ns, nd)
    # inner products of trained second-order rows rank held-out edges above
    # non-edges (0.65 measured); untrained rows are at chance
    assert a > 0.6 and abs(a0 - 0.5) < 0.05, (a, a0)
