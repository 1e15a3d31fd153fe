"""Pins of the oracle's per-pair immediate updates (Algorithm 1's local path,
LineUpdate applied pair after pair):

* with K = 0 every sample is one call reading the state before it, so the
  pairwise run equals the (separately pinned) minibatch run at B = 1 exactly;
* each call moves U[u] and Ctx[y] by -eta times the central-difference
  gradient of the pair's loss plus the decay term, evaluated at the values
  before the call, on a tiny graph where negatives repeat and, in order 1,
  equal u (the later call sees the earlier call's writes);
* the same on walk pairs;
* eta = 0 leaves the tables unchanged.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I


def _tables(g, order, dim, seed=1):
    U = O.init_uniform(g.n_nodes, dim, seed)
    # a non-zero C so that the first calls already move U
    C = O.init_uniform(g.n_nodes, dim, seed + 7) if order == 2 else None
    return U, C


@pytest.mark.parametrize("order", [1, 2])
def test_k0_equals_minibatch_b1(order):
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    U1, C1 = _tables(g, order, 16)
    U2, C2 = U1.copy(), None if C1 is None else C1.copy()
    kw = dict(order=order, K=0, n_samples=3000, seed=3, lam=1e-3, lr_total=3000)
    O.train(T, U1, C1, batch=1, **kw)
    O.train_pairwise(T, U2, C2, batch=1, **kw)
    assert np.array_equal(U1, U2)
    if order == 2:
        assert np.array_equal(C1, C2)


def _log_sigmoid(s):
    return -np.logaddexp(0.0, -s)


def _grad(f, x, h=1e-6):
    out = np.empty_like(x)
    for k in range(len(x)):
        e = np.zeros_like(x)
        e[k] = h
        out[k] = (f(x + e) - f(x - e)) / (2 * h)
    return out


def _replay(recs, U, C, order, etas, lam, alpha):
    """The calls of the local path in order, each a gradient step on the
    pair's loss (-log sigma(s) or -alpha log sigma(-s), plus lam/2 |.|^2 on
    both rows) taken by central differences at the values before the call;
    U[u] is written first, then Ctx[y]."""
    Ctx = C if order == 2 else U
    for rec, eta in zip(recs, etas):
        u = rec[0]
        for j, y in enumerate(rec[1:]):
            x, c = U[u].copy(), Ctx[y].copy()
            if j == 0:
                loss_x = lambda z: -_log_sigmoid(z @ c) + 0.5 * lam * (z @ z)
                loss_c = lambda z: -_log_sigmoid(x @ z) + 0.5 * lam * (z @ z)
            else:
                loss_x = lambda z: -alpha * _log_sigmoid(-(z @ c)) + 0.5 * lam * (z @ z)
                loss_c = lambda z: -alpha * _log_sigmoid(-(x @ z)) + 0.5 * lam * (z @ z)
            U[u] = x - eta * _grad(loss_x, x)
            Ctx[y] = c - eta * _grad(loss_c, c)


@pytest.mark.parametrize("order", [1, 2])
@pytest.mark.parametrize("walk", [False, True])
def test_each_call_is_a_gradient_step_on_the_current_rows(order, walk):
    # 6 nodes: with K = 4 negatives repeat, and in order 1 they hit u
    src = np.array([0, 0, 1, 2, 3, 4, 5, 1])
    dst = np.array([1, 2, 2, 3, 4, 5, 0, 4])
    g = I.canonicalize(6, src, dst, np.array([1.0, 2.0, 0.5, 1.0, 3.0, 1.0, 1.0, 2.0]), symmetrize=True)
    T = O.Tables(g)
    dim, K, n, B, lam, alpha, seed = 4, 4, 40, 3, 0.01, 0.7, 11
    U, C = _tables(g, order, dim)
    U *= 40.0  # scores of order 1, so that sigma is not flat
    if C is not None:
        C *= 40.0
    Ur, Cr = U.copy(), None if C is None else C.copy()
    wk = (O.walk_cumw(g), 5, 2) if walk else None
    O.train_pairwise(T, U, C, order=order, K=K, n_samples=n, seed=seed, batch=B, lam=lam, alpha_neg=alpha,
                     lr0=0.5, sample_offset=17, lr_total=100, walk=wk)
    recs = O.sample_walk(T, wk[0], seed, 17, n, K, 5, 2) if walk else O.sample(T, seed, 17, n, K)
    if order == 1:
        assert any(u in r[2:] for u, r in zip(recs[:, 0], recs)), "no negative equal to u: the case is not covered"
    assert any(len(set(r[2:])) < K for r in recs), "no repeated negative: the case is not covered"
    etas = [O.lib().orc_batch_lr(0.5, 1, 1e-4, 100, 17 + (t // B) * B) for t in range(n)]
    _replay(recs, Ur, Cr, order, etas, lam, alpha)
    np.testing.assert_allclose(U, Ur, rtol=0, atol=1e-7)
    if order == 2:
        np.testing.assert_allclose(C, Cr, rtol=0, atol=1e-7)
    assert np.abs(U - _tables(g, order, dim)[0] * 40.0).max() > 1e-2  # training moved the rows


def test_zero_lr_leaves_tables_unchanged():
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    U, C = _tables(g, 2, 8)
    U0, C0 = U.copy(), C.copy()
    O.train_pairwise(T, U, C, order=2, K=5, n_samples=2000, seed=1, batch=64, lr0=0.0)
    assert np.array_equal(U, U0) and np.array_equal(C, C0)


def test_cpu_hogwild_context_baseline():
    """The multi-threaded CPU Hogwild (FP32, context for the benchmark): one
    thread is the per-pair run in FP32 (within 1e-5 of FP64); four threads
    racing on the rows land near the same loss."""
    g = I.tiny_chung_lu()
    T = O.Tables(g)
    kw = dict(order=2, K=5, n_samples=50_000, seed=3, batch=256)
    U, C = _tables(g, 2, 32)
    U0, C0 = U.astype(np.float32), C.astype(np.float32)
    O.train_pairwise(T, U, C, **kw)
    U1, C1 = U0.copy(), C0.copy()
    O.train_hogwild_cpu(T, U1, C1, threads=1, **kw)
    assert max(np.abs(U1 - U).max(), np.abs(C1 - C).max()) <= 1e-5
    U4, C4 = U0.copy(), C0.copy()
    O.train_hogwild_cpu(T, U4, C4, threads=4, **kw)
    l_seq = O.eval_loss(T, U, C, order=2, K=5, seed=9, m=5000)
    l_mt = O.eval_loss(T, U4.astype(np.float64), C4.astype(np.float64), order=2, K=5, seed=9, m=5000)
    assert abs(l_mt - l_seq) <= 0.05 * l_seq
