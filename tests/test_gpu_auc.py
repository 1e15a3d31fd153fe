"""Link-prediction AUC through the C ABI against the FP64 oracle.

* FP32 scores (inner product or cosine) against the oracle's FP64 scores of
  the same tables, within bounds derived from FP32 dot products of d terms;
* the AUC counts (#(neg < pos), #(neg == pos)) equal to the oracle's
  Mann-Whitney counts over the GPU's own scores, exactly (the comparison
  decisions are taken in the kernel's precision on both sides);
* ties, several radix tiles with a ragged tail, BF16 tables, both orders,
  error cases.
"""
import numpy as np
import pytest

from oracle import link as OL
from paper_2604_09419_gb300 import inputs as I
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def score_tol(dims, tabs, src, dst, score):
    if score == "cosine":
        # |fl(cos) - cos|: about d unit roundoffs in the dot and the norms, a
        # few more in the sqrt/div/combination
        return (2 * max(dims) + 16) * 2.0 ** -24
    # FP32 FMA dot of d terms: |error| <= d u sum |a_k b_k| (plus the sum of orders)
    absdot = OL.pair_scores([np.abs(t) for t in tabs], src, dst, "dot")
    return (max(dims) + 4) * 2.0 ** -24 * absdot + 1e-30


@pytest.fixture(scope="module")
def ctx():
    c = G.context()
    yield c
    c.close()


def split_pairs(g, seed=0, frac=0.1):
    tr, hs, hd = I.split_edges(g, frac, seed=seed)
    ns, nd = I.non_edges(g, len(hs), seed=seed)
    return tr, hs, hd, ns, nd


def check(ctx, orders, tabs, hs, hd, ns, nd, dims, score="dot"):
    from paper_2604_09419_gb300 import line as L
    n = len(hs) + len(ns)
    scores = np.empty(n, np.float32)
    code = L.SCORE_DOT if score == "dot" else L.SCORE_COSINE
    auc, (less, eq) = ctx.eval_auc(orders, hs, hd, ns, nd, scores, score=code)
    src, dst = np.concatenate([hs, ns]), np.concatenate([hd, nd])
    want = OL.pair_scores(tabs, src, dst, score)
    err = np.abs(scores.astype(np.float64) - want)
    assert (err <= score_tol(dims, tabs, src, dst, score)).all(), err.max()
    # exact counts over the GPU's scores
    l2, e2 = OL.mann_whitney_counts(scores[:len(hs)], scores[len(hs):])
    assert (less, eq) == (l2, e2)
    assert auc == (2 * l2 + e2) / (2.0 * len(hs) * len(ns))
    return auc, OL.mann_whitney(want[:len(hs)], want[len(hs):])


def oracle_trained(g, order, dim, n, seed):
    from oracle import Tables, init_uniform, train
    U = init_uniform(g.n_nodes, dim, seed)
    C = np.zeros_like(U) if order == 2 else None
    train(Tables(g), U, C, order=order, K=5, n_samples=n, seed=seed, batch=256)
    return U, C


def test_auc_tiny_both_orders(ctx):
    """Oracle-trained tables of the tiny graph with 10% of edges held out."""
    g = G.graph("tiny")
    tr, hs, hd, ns, nd = split_pairs(g)
    G.upload(ctx, tr)
    U1, _ = oracle_trained(tr, 1, 16, 100_000, 3)
    U2, C2 = oracle_trained(tr, 2, 16, 100_000, 4)
    U1 = G.upload_tables(ctx, 1, U1)
    U2, _ = G.upload_tables(ctx, 2, U2, C2)
    res = []
    for score in ("dot", "cosine"):
        res.append(check(ctx, 1, [U1], hs, hd, ns, nd, [16], score))
        res.append(check(ctx, 2, [U2], hs, hd, ns, nd, [16], score))
        res.append(check(ctx, 3, [U1, U2], hs, hd, ns, nd, [16, 16], score))
    # FP32 against FP64 scores: the AUCs agree to a few flipped near-ties
    for a, w in res:
        assert abs(a - w) < 1e-3


def test_auc_ties_many_tiles_and_bf16(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    tr, hs, hd, ns, nd = split_pairs(g, seed=1, frac=0.3)
    # more negatives than positives, not a multiple of the sort tile
    ns, nd = I.non_edges(g, 3 * len(hs) + 123, seed=2)
    assert len(ns) > 4 * 4096
    G.upload(ctx, tr)
    U, C = oracle_trained(tr, 2, 128, 100_000, 5)
    # zero a third of the rows: pairs touching them score exactly 0 (ties)
    U[::3] = 0.0
    U2, _ = G.upload_tables(ctx, 2, U, C, dtype=L.DTYPE_BF16)
    auc, want = check(ctx, 2, [U2], hs, hd, ns, nd, [128])
    check(ctx, 2, [U2], hs, hd, ns, nd, [128], "cosine")
    scores = np.empty(len(hs) + len(ns), np.float32)
    ctx.eval_auc(2, hs, hd, ns, nd, scores)
    assert (scores == 0).sum() > len(scores) // 4
    assert abs(auc - want) < 1e-3


def test_auc_errors(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(1, 16, L.DTYPE_F32, seed=1)
    hs = np.array([0, 1], np.int32)
    hd = np.array([2, 3], np.int32)
    with pytest.raises(L.LineError) as ei:  # order 2 has no tables
        ctx.eval_auc(2, hs, hd, hs, hd)
    assert ei.value.status == L.LINE_ERR_STATE
    with pytest.raises(L.LineError) as ei:
        ctx.eval_auc(4, hs, hd, hs, hd)
    assert ei.value.status == L.LINE_ERR_ARG
    with pytest.raises(L.LineError) as ei:
        ctx.eval_auc(1, hs, hd, hs, hd, score=2)
    assert ei.value.status == L.LINE_ERR_ARG
    bad = np.array([0, g.n_nodes], np.int32)
    with pytest.raises(L.LineError) as ei:
        ctx.eval_auc(1, hs, hd, hs, bad)
    assert ei.value.status == L.LINE_ERR_ARG
    # the context is still usable; identical positive and negative sets give 1/2
    auc, (less, eq) = ctx.eval_auc(1, hs, hd, hs, hd)
    assert auc == 0.5 and less == 1 and eq == 2
