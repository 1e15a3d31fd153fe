"""FP64 oracle of the link-prediction evaluation (reporting, not training).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

Embeddings are judged here by how well they separate held-out edges from
vertex pairs that are not edges (link prediction; the paper's own measure,
node classification by Micro/Macro-F1 in §V-C, needs node labels).  The
score and the statistic are the plain textbook definitions, written out:

* ``pair_scores`` - the inner product of the endpoints' concatenated U
  rows of the requested orders (``score="dot"``), or their cosine similarity
  after scaling each order's row to unit L2 norm (``score="cosine"``; an
  all-zero row stays zero, and a pair with a zero concatenated vector scores
  0);
* ``mann_whitney`` - the area under the ROC curve as the Mann-Whitney
  statistic: the fraction of (positive, negative) pairs in which the positive
  scores higher, ties counted one half.

Pinned by ``tests/test_oracle_link.py`` against brute-force double loops,
``scipy.stats.mannwhitneyu`` and closed-form cases.
"""
from __future__ import annotations

import numpy as np


def normalised_rows(tables, nodes) -> np.ndarray:
    """Concatenation over ``tables`` of the rows ``nodes``, each scaled to unit norm (FP64)."""
    parts = []
    for U in tables:
        R = np.asarray(U, np.float64)[np.asarray(nodes, np.int64)]
        nrm = np.sqrt((R * R).sum(axis=1))
        scale = np.where(nrm > 0, 1.0 / np.where(nrm > 0, nrm, 1.0), 0.0)
        parts.append(R * scale[:, None])
    return np.concatenate(parts, axis=1)


def pair_scores(tables, src, dst, score: str = "dot") -> np.ndarray:
    """Inner product (or cosine of the per-order normalised rows) of the
    concatenated U rows of each pair (FP64)."""
    if score == "dot":
        out = np.zeros(len(src))
        for U in tables:
            U = np.asarray(U, np.float64)
            out += (U[np.asarray(src, np.int64)] * U[np.asarray(dst, np.int64)]).sum(axis=1)
        return out
    assert score == "cosine", score
    a = normalised_rows(tables, src)
    b = normalised_rows(tables, dst)
    na = np.sqrt((a * a).sum(axis=1))
    nb = np.sqrt((b * b).sum(axis=1))
    dot = (a * b).sum(axis=1)
    den = na * nb
    return np.where(den > 0, dot / np.where(den > 0, den, 1.0), 0.0)


def mann_whitney_counts(pos, neg) -> tuple[int, int]:
    """(pairs with neg < pos, pairs with neg == pos) over all (pos, neg) pairs.

    Counted per positive by binary search in the sorted negatives (a library
    sort and search as the steps of the double sum).
    """
    pos = np.asarray(pos)
    neg = np.sort(np.asarray(neg))
    lo = np.searchsorted(neg, pos, side="left")
    hi = np.searchsorted(neg, pos, side="right")
    return int(lo.astype(np.int64).sum()), int((hi - lo).astype(np.int64).sum())


def mann_whitney(pos, neg) -> float:
    """AUC = (#(neg < pos) + #(neg == pos) / 2) / (|pos| |neg|)."""
    less, equal = mann_whitney_counts(pos, neg)
    return (2 * less + equal) / (2.0 * len(pos) * len(neg))


def auc(tables, pos_src, pos_dst, neg_src, neg_dst, score: str = "dot") -> float:
    """Link-prediction AUC of FP64 scores."""
    return mann_whitney(pair_scores(tables, pos_src, pos_dst, score), pair_scores(tables, neg_src, neg_dst, score))
