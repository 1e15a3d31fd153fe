"""Pins of the oracle's LINE update (no GPU).

* Finite differences: one minibatch changes every table entry by exactly
  -eta_b times the gradient, at the batch-start state, of the batch's
  negative-sampling loss (Algorithm 1's g scalars come from that loss, the
  l2 term from the weight decay of Eq. 2-3, the batch-start reads and the
  summation from Eq. 4).
* A closed-form two-node recurrence.
* Invariants: lr 0, untouched rows, the zero context table, a split at a
  batch boundary, the linear schedule.
* The loss at symmetric states, in closed form.
"""
import math

import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I


def _small_graph():
    return I.chung_lu_undirected(40, 2.1, 120.0, seed=7)


def _batch_loss(pairs, U, C, order, alpha, lam):
    """Negative-sampling LINE loss of a list of (x, y, label) pairs plus the
    l2 penalty once per pair occurrence."""
    Ctx = U if order == 1 else C
    L = 0.0
    for x, y, label in pairs:
        s = float(U[x] @ Ctx[y])
        if label:
            L += math.log1p(math.exp(-s))
        else:
            L += alpha * math.log1p(math.exp(s))
        L += 0.5 * lam * (float(U[x] @ U[x]) + float(Ctx[y] @ Ctx[y]))
    return L


@pytest.mark.parametrize("order", [1, 2])
def test_update_is_minus_eta_gradient(order):
    g = _small_graph()
    T = O.Tables(g)
    dim, K, B, seed = 6, 3, 5, 99
    eta, lam, alpha = 0.05, 1e-2, 0.7
    rng = np.random.default_rng(order)
    U = rng.normal(0, 0.5, (g.n_nodes, dim))
    C = rng.normal(0, 0.5, (g.n_nodes, dim)) if order == 2 else None
    U1, C1 = U.copy(), (C.copy() if C is not None else None)
    O.train(T, U1, C1, order=order, K=K, lr0=eta, schedule=0, n_samples=B, seed=seed, batch=B,
            lam=lam, alpha_neg=alpha)
    rec = O.sample(T, seed=seed, t0=0, count=B, K=K)
    pairs = [(int(r[0]), int(r[1 + j]), j == 0) for r in rec for j in range(K + 1)]
    h = 1e-6
    tables = [("U", U, U1)] + ([("C", C, C1)] if order == 2 else [])
    touched = sorted({p[0] for p in pairs} | {p[1] for p in pairs})
    for name, X, X1 in tables:
        for r in touched:
            for k in range(dim):
                old = X[r, k]
                X[r, k] = old + h
                lp = _batch_loss(pairs, U, C, order, alpha, lam)
                X[r, k] = old - h
                lm = _batch_loss(pairs, U, C, order, alpha, lam)
                X[r, k] = old
                want = -eta * (lp - lm) / (2 * h)
                got = X1[r, k] - X[r, k]
                assert abs(got - want) <= 1e-6 * max(1e-3, abs(want)), (name, r, k, got, want)
        untouched = np.setdiff1d(np.arange(g.n_nodes), touched)
        assert np.array_equal(X1[untouched], X[untouched])


def test_two_node_closed_form():
    """Two nodes, one undirected edge, K = 0, second order, C = 0.

    Every sample is the arc (u, v) = (0, 1) or (1, 0) and g = eta (1 - sigma(s)).
    Batch 1: s = 0, so dU = 0 and dC[v] = eta/2 U[u].  Afterwards each
    single-sample batch maps (U[u], C[v]) -> (U[u] + g C[v], C[v] + g U[u])
    with s = U[u].C[v] read before the update.
    """
    g = I.canonicalize(2, np.array([0]), np.array([1]), None, symmetrize=True)
    T = O.Tables(g)
    dim, eta, n = 4, 0.1, 9
    U = O.init_uniform(2, dim, seed=3)
    C = np.zeros_like(U)
    U1, C1 = U.copy(), C.copy()
    O.train(T, U1, C1, order=2, K=0, lr0=eta, schedule=0, n_samples=n, seed=5, batch=1)
    rec = O.sample(T, seed=5, t0=0, count=n, K=0)
    u0, v0 = rec[0, 0], rec[0, 1]
    Uh, Ch = U.copy(), C.copy()
    # batch 1 by hand
    Ch[v0] = 0.5 * eta * Uh[u0]
    for t in range(1, n):
        u, v = rec[t, 0], rec[t, 1]
        s = Uh[u] @ Ch[v]
        gg = eta / (1.0 + math.exp(s))  # eta (1 - sigma(s))
        Uh[u], Ch[v] = Uh[u] + gg * Ch[v], Ch[v] + gg * Uh[u]
    np.testing.assert_allclose(U1, Uh, rtol=0, atol=1e-15)
    np.testing.assert_allclose(C1, Ch, rtol=0, atol=1e-15)


def test_invariants():
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    dim = 8
    U0 = O.init_uniform(g.n_nodes, dim, seed=1)
    # lr 0: no change
    U, C = U0.copy(), np.zeros_like(U0)
    O.train(T, U, C, order=2, K=5, lr0=0.0, n_samples=2000, seed=1, batch=64)
    assert np.array_equal(U, U0) and not C.any()
    # second order, first batch: C = 0 makes dU = g * 0, so U is unchanged
    U, C = U0.copy(), np.zeros_like(U0)
    O.train(T, U, C, order=2, K=5, n_samples=64, seed=1, batch=64)
    assert np.array_equal(U, U0) and C.any()
    # split at a batch boundary equals one run (same schedule total)
    Ua, Ca = U0.copy(), np.zeros_like(U0)
    O.train(T, Ua, Ca, order=2, K=5, n_samples=1000, seed=4, batch=100, lam=1e-4, lr_total=1000)
    Ub, Cb = U0.copy(), np.zeros_like(U0)
    O.train(T, Ub, Cb, order=2, K=5, n_samples=300, seed=4, batch=100, lam=1e-4, lr_total=1000)
    O.train(T, Ub, Cb, order=2, K=5, n_samples=700, seed=4, batch=100, lam=1e-4, lr_total=1000,
            sample_offset=300)
    assert np.array_equal(Ua, Ub) and np.array_equal(Ca, Cb)
    # a ragged last batch: 1000 samples in batches of 300 -> 300,300,300,100;
    # differs from batches of 250 (batch semantics matter)
    Uc, Cc = U0.copy(), np.zeros_like(U0)
    O.train(T, Uc, Cc, order=2, K=5, n_samples=1000, seed=4, batch=300, lam=1e-4, lr_total=1000)
    assert not np.array_equal(Uc, Ua)
    # nodes never drawn keep their initial U row and a zero C row
    rec = O.sample(T, seed=4, t0=0, count=1000, K=5)
    used = np.unique(rec)
    unused = np.setdiff1d(np.arange(g.n_nodes), used)
    assert np.array_equal(Ua[unused], U0[unused]) and not Ca[unused].any()


def test_linear_schedule():
    assert O.batch_lr(0.025, 0, 1e-4, 1000, 500) == 0.025
    assert O.batch_lr(0.025, 1, 1e-4, 1000, 0) == 0.025
    assert O.batch_lr(0.025, 1, 1e-4, 1000, 250) == 0.025 * 0.75
    assert O.batch_lr(0.025, 1, 1e-4, 1000, 1000) == 0.025 * 1e-4


@pytest.mark.parametrize("order", [1, 2])
def test_loss_closed_forms(order):
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    n, dim, K, M = g.n_nodes, 8, 5, 3000
    # all scores zero: every term is log 2
    U = O.init_uniform(n, dim, seed=2)
    Z = np.zeros_like(U)
    if order == 2:
        assert O.eval_loss(T, U, Z, order=2, K=K, seed=0, m=M) == pytest.approx(M * (K + 1) * math.log(2), rel=1e-12)
    # every score equal to a*b: L = M (softplus(-ab) + K softplus(ab))
    a, b = 0.8, -1.3
    U = np.zeros((n, dim)); U[:, 0] = a
    C = np.zeros((n, dim)); C[:, 0] = b
    s = a * b if order == 2 else a * a
    want = M * (math.log1p(math.exp(-s)) + K * math.log1p(math.exp(s)))
    got = O.eval_loss(T, U, C if order == 2 else None, order=order, K=K, seed=0, m=M)
    assert got == pytest.approx(want, rel=1e-12)


def test_training_lowers_loss():
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    U = O.init_uniform(g.n_nodes, 16, seed=0)
    C = np.zeros_like(U)
    before = O.eval_loss(T, U, C, order=2, K=5, seed=0, m=20000)
    O.train(T, U, C, order=2, K=5, n_samples=100_000, seed=0, batch=256)
    after = O.eval_loss(T, U, C, order=2, K=5, seed=0, m=20000)
    assert after < 0.9 * before


def test_init_is_uniform_on_the_stated_interval():
    """Initial U rows are uniform on [-0.5/d, 0.5/d) (the workload's
    initialisation): every value in range and exact in FP32, the
    distribution passes a Kolmogorov-Smirnov test, row i does not depend on
    the table size, and seeds give different tables."""
    from scipy.stats import kstest
    for dim in (16, 128):
        U = O.init_uniform(4000, dim, seed=5)
        lo, hi = -0.5 / dim, 0.5 / dim
        assert U.min() >= lo and U.max() < hi
        assert np.array_equal(U.astype(np.float32).astype(np.float64), U)
        assert kstest(U.ravel(), "uniform", args=(lo, hi - lo)).pvalue > 1e-3
        np.testing.assert_array_equal(O.init_uniform(100, dim, seed=5), U[:100])
        assert not np.array_equal(O.init_uniform(100, dim, seed=6), U[:100])
        # neighbouring values are not correlated
        assert abs(np.corrcoef(U[:, 0], U[:, 1])[0, 1]) < 0.1
