"""Warm-start MLP through the C ABI against the FP64 oracle.

* initial weights bit-exact (Philox domain 7);
* inputs (log degree, mean known-neighbour row) within FP32 summation
  bounds, and within one BF16 rounding for BF16 activations; the same bits
  for a row subset (repeated rows and hubs of many arc chunks included) as
  for the full pass;
* loss and gradients against the oracle's backpropagation, element by
  element: |g - g_oracle| <= tol max|g_oracle| + tol |g_oracle| per tensor,
  tol 1e-5 (FP32 activations) or 1e-3 (BF16 activations, oracle rounding x
  and h to BF16 at the same points);
* Adam training steps, predictions into table rows, determinism, errors;
* the gain of the warm start over the random rows LINE starts from (an
  empirical claim: measured, not pinned).
"""
import numpy as np
import pytest

from oracle import mlp as OM
from paper_2604_09419_gb300 import inputs as I
from tests import gpu_util as G

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    c = G.context()
    yield c
    c.close()


def trained_tables(name, dim, n, seed):
    U, C = G.oracle_run(name, 2, dim, 5, n, seed, 256, seed + 1)
    return U, C


def flat(p):
    return np.concatenate([p["W1"].ravel(), p["b1"], p["W2"].ravel(), p["b2"]])


def unflat(v, dim, hidden):
    P = OM.in_width(dim)
    n1 = hidden * P
    n2 = dim * hidden
    return {"W1": v[:n1].reshape(hidden, P).astype(np.float64), "b1": v[n1:n1 + hidden].astype(np.float64),
            "W2": v[n1 + hidden:n1 + hidden + n2].reshape(dim, hidden).astype(np.float64),
            "b2": v[n1 + hidden + n2:].astype(np.float64)}


def setup(ctx, name, dim, act, hidden=64, seed=11, known_frac=0.1):
    from paper_2604_09419_gb300 import line as L
    g = G.graph(name)
    G.upload(ctx, g)
    U, C = trained_tables(name, dim, 60_000, 5)
    U, C = G.upload_tables(ctx, 2, U, C)
    held, _ = I.hold_out_nodes(g, known_frac, seed=1)
    known = (~held).astype(np.uint8)
    ctx.mlp_create(2, hidden=hidden, act_dtype=act, seed=seed)
    ctx.mlp_features(known)
    X = OM.features(g.n_nodes, g.src, g.dst, g.w, U, known.astype(bool), act_bf16=(act == L.DTYPE_BF16))
    return g, U, known, X


@pytest.mark.parametrize("dim,hidden", [(16, 32), (128, 256)])
def test_init_bit_exact(ctx, dim, hidden):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(2, dim, L.DTYPE_F32, seed=1)
    ctx.mlp_create(2, hidden=hidden, act_dtype=L.DTYPE_F32, seed=99)
    got = ctx.mlp_get_params()
    want = flat(OM.init_params(dim, hidden, 99)).astype(np.float32)
    assert got.shape == want.shape and np.array_equal(got, want)


@pytest.mark.parametrize("name,dim", [("tiny", 16), ("rmat14", 128)])
@pytest.mark.parametrize("act", [0, 1])
def test_features_match_oracle(ctx, name, dim, act):
    g, U, known, X = setup(ctx, name, dim, act)
    got = np.empty(X.shape, np.float32)
    ctx.mlp_get_features(got)
    # FP32 sum of cnt rows: |error of the mean| <= (cnt + 2) 2^-24 max|U|
    ok = known.astype(bool)[g.dst]
    cnt = np.bincount(g.src[ok], minlength=g.n_nodes).astype(np.float64)
    bound = (cnt[:, None] + 2) * 2.0 ** -24 * np.abs(U).max() + 2.0 ** -23 * np.abs(X)
    if act == 1:
        bound = bound + 2.0 ** -7 * np.abs(X)  # at most one BF16 ulp (8 significant bits) apart
    err = np.abs(got.astype(np.float64) - X)
    assert (err <= bound).all(), float((err - bound).max())


def test_features_of_a_row_subset(ctx):
    """Inputs recomputed for some rows after the graph changed equal a full
    recomputation for those rows (same bits); the other rows keep theirs."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    held, kept = I.hold_out_nodes(g, 0.1, seed=3)
    G.upload(ctx, kept)
    U, C = trained_tables("rmat14", 64, 40_000, 6)
    G.upload_tables(ctx, 2, U, C)
    known = (~held).astype(np.uint8)
    ctx.mlp_create(2, hidden=32, act_dtype=L.DTYPE_BF16, seed=1)
    ctx.mlp_features(known)
    before = np.empty((g.n_nodes, 80), np.float32)
    ctx.mlp_get_features(before)
    G.upload(ctx, g)  # the held-out nodes' arcs arrive; tables and MLP are kept
    rows = np.flatnonzero(held).astype(np.int32)
    ctx.mlp_features_rows(known, rows)
    part = np.empty_like(before)
    ctx.mlp_get_features(part)
    ctx.mlp_features(known)
    full = np.empty_like(before)
    ctx.mlp_get_features(full)
    assert np.array_equal(part[rows], full[rows])
    rest = np.flatnonzero(~held)
    assert np.array_equal(part[rest], before[rest])
    assert not np.array_equal(before[rows], full[rows])  # their inputs did change
    with pytest.raises(L.LineError) as ei:
        ctx.mlp_features_rows(known, np.array([0, g.n_nodes], np.int32))
    assert ei.value.status == L.LINE_ERR_ARG


def test_features_of_repeated_rows_and_hubs(ctx):
    """A row list that names hubs many times (more often than the graph has
    hubs) and spans hubs of one and of many arc chunks gives the inputs of
    the full pass for those rows, bit for bit."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    G.upload(ctx, g)
    U, C = trained_tables("rmat14", 64, 40_000, 6)
    G.upload_tables(ctx, 2, U, C)
    held, _ = I.hold_out_nodes(g, 0.1, seed=3)
    known = (~held).astype(np.uint8)
    deg = np.bincount(g.src, minlength=g.n_nodes)
    assert deg.max() > 2048 and ((deg > 256) & (deg <= 2048)).any()  # hubs of one and of two chunks
    hubs = np.flatnonzero(deg > 256).astype(np.int32)
    rows = np.concatenate([np.repeat(hubs, 40), np.arange(0, g.n_nodes, 5, dtype=np.int32), hubs[::-1]])
    assert len(rows) > g.n_arcs // 256 + 1
    ctx.mlp_create(2, hidden=32, act_dtype=L.DTYPE_F32, seed=1)
    ctx.mlp_features_rows(known, rows)
    part = np.empty((g.n_nodes, 80), np.float32)
    ctx.mlp_get_features(part)
    ctx.mlp_features(known)
    full = np.empty_like(part)
    ctx.mlp_get_features(full)
    assert np.array_equal(part[rows], full[rows]) and part[hubs].any()


def test_features_of_a_sample_alone(ctx):
    """Inputs of a node sample computed without a pass over every node equal
    those of the full pass for those rows, and the other rows stay zero: the
    warm start can fit on a sample of the kept nodes."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    G.upload(ctx, g)
    U, C = trained_tables("rmat14", 64, 40_000, 6)
    G.upload_tables(ctx, 2, U, C)
    held, _ = I.hold_out_nodes(g, 0.1, seed=3)
    known = (~held).astype(np.uint8)
    rows = np.flatnonzero(~held)[::7].astype(np.int32)
    ctx.mlp_create(2, hidden=32, act_dtype=L.DTYPE_BF16, seed=1)
    ctx.mlp_features_rows(known, rows)
    part = np.empty((g.n_nodes, 80), np.float32)
    ctx.mlp_get_features(part)
    ctx.mlp_features(known)
    full = np.empty_like(part)
    ctx.mlp_get_features(full)
    assert np.array_equal(part[rows], full[rows]) and part[rows].any()
    others = np.setdiff1d(np.arange(g.n_nodes), rows)
    assert not part[others].any()


def elementwise_excess(got, want, tol):
    """Largest excess of |got - want| over tol max|want| + tol |want|, taken
    element by element (<= 0 when every element is within the bound)."""
    bound = tol * np.abs(want).max() + tol * np.abs(want)
    return float((np.abs(got - want) - bound).max())


@pytest.mark.parametrize("act,tol", [(0, 1e-5), (1, 1e-3)])
def test_loss_and_gradients_match_oracle(ctx, act, tol):
    """Every element of every gradient tensor (W1, b1, W2, b2) against the
    oracle's backpropagation, on a minibatch that includes nodes whose input
    row is all zeros (no arcs); the input padding columns of W1 get exactly
    zero gradient on both sides."""
    dim, hidden = 128, 256
    g, U, known, X = setup(ctx, "rmat14", dim, act, hidden=hidden)
    rng = np.random.default_rng(3)
    # a parameter point with non-zero biases (both sides start from it)
    p = OM.init_params(dim, hidden, 11)
    p["b1"] = rng.normal(size=hidden) * 0.1
    p["b2"] = rng.normal(size=dim) * 0.01
    pv = flat(p).astype(np.float32)
    ctx.mlp_set_params(pv)
    p = unflat(pv, dim, hidden)
    zero_rows = np.flatnonzero(~X.any(axis=1))[:64]
    assert zero_rows.size >= 16  # isolated nodes: log(1 + 0) = 0 and no neighbours
    rows = np.concatenate([np.flatnonzero(known)[:3000], zero_rows]).astype(np.int32)
    grads = np.empty(pv.shape, np.float32)
    loss = ctx.mlp_grad(rows, grads)
    L, gw = OM.loss_and_grads(p, X[rows], U[rows], act_bf16=(act == 1))
    assert abs(loss - L) <= tol * L
    got = unflat(grads, dim, hidden)
    for k in ("W1", "b1", "W2", "b2"):
        ex = elementwise_excess(got[k], gw[k], tol)
        assert ex <= 0, (k, ex)
    pad = slice(dim + 1, OM.in_width(dim))
    assert not got["W1"][:, pad].any() and not gw["W1"][:, pad].any()


def test_gradients_of_small_and_ragged_batches_bf16(ctx):
    """BF16 activations at d = 128, hidden 256 (the tensor-core forward and
    weight-gradient kernels): batches of 1, 17, 64, 65 and 200 rows, so the
    batch is below, at and just past one 64-row slice of the weight gradient
    and always a partial 128-row tile of the forward products; every element
    of every gradient against the oracle."""
    from paper_2604_09419_gb300 import line as L
    dim, hidden = 128, 256
    g, U, known, X = setup(ctx, "rmat14", dim, L.DTYPE_BF16, hidden=hidden)
    rng = np.random.default_rng(21)
    p = OM.init_params(dim, hidden, 11)
    p["b1"] = rng.normal(size=hidden) * 0.1
    p["b2"] = rng.normal(size=dim) * 0.01
    pv = flat(p).astype(np.float32)
    ctx.mlp_set_params(pv)
    p = unflat(pv, dim, hidden)
    kept = np.flatnonzero(known)
    for B in (1, 17, 64, 65, 200):
        rows = rng.choice(kept, size=B, replace=False).astype(np.int32)
        grads = np.empty(pv.shape, np.float32)
        loss = ctx.mlp_grad(rows, grads)
        Lo, gw = OM.loss_and_grads(p, X[rows], U[rows], act_bf16=True)
        assert abs(loss - Lo) <= 1e-3 * Lo, (B, loss, Lo)
        got = unflat(grads, dim, hidden)
        for k in ("W1", "b1", "W2", "b2"):
            ex = elementwise_excess(got[k], gw[k], 1e-3)
            assert ex <= 0, (B, k, ex)


def test_training_steps_match_oracle(ctx):
    dim, hidden = 16, 32
    g, U, known, X = setup(ctx, "tiny", dim, 0, hidden=hidden)
    nodes = np.flatnonzero(known).astype(np.int32)
    losses = ctx.mlp_train(nodes, steps=12, batch=128, lr=1e-3, seed=4)
    p = OM.init_params(dim, hidden, 11)
    st = {}
    want = OM.train(p, X, U, nodes, steps=12, batch=128, seed=4, lr=1e-3, state=st)
    np.testing.assert_allclose(losses, want, rtol=1e-5)

    def close():
        got = unflat(ctx.mlp_get_params(), dim, hidden)
        for k in p:
            # Adam moves every weight by about lr per step: compare on that scale
            assert np.abs(got[k] - p[k]).max() <= 1e-3 * 1e-3 * 15, k

    close()
    # a second call continues the step count and the optimiser state
    more = ctx.mlp_train(nodes, steps=3, batch=128, lr=1e-3, seed=4, step_offset=12)
    want = OM.train(p, X, U, nodes, steps=3, batch=128, seed=4, lr=1e-3, step_offset=12, state=st)
    np.testing.assert_allclose(more, want, rtol=1e-5)
    close()


def test_training_bf16_tracks_oracle_and_is_deterministic(ctx):
    from paper_2604_09419_gb300 import line as L
    dim, hidden = 128, 256
    g, U, known, X = setup(ctx, "rmat14", dim, L.DTYPE_BF16, hidden=hidden)
    nodes = np.flatnonzero(known).astype(np.int32)
    p0 = ctx.mlp_get_params()
    losses = ctx.mlp_train(nodes, steps=20, batch=512, lr=1e-3, seed=8)
    p1 = ctx.mlp_get_params()
    p = OM.init_params(dim, hidden, 11)
    want = OM.train(p, X, U, nodes, steps=20, batch=512, seed=8, lr=1e-3, act_bf16=True)
    np.testing.assert_allclose(losses, want, rtol=1e-3)
    assert losses[-1] < losses[0]
    ctx.mlp_set_params(p0)
    again = ctx.mlp_train(nodes, steps=20, batch=512, lr=1e-3, seed=8)
    assert np.array_equal(again, losses) and np.array_equal(ctx.mlp_get_params(), p1)


def test_recreate_same_shape_starts_over(ctx):
    """line_mlp_create over an MLP of the same shape keeps its memory but
    starts over: initial weights, cleared inputs, zero optimiser state."""
    from paper_2604_09419_gb300 import line as L
    dim, hidden = 128, 256
    g, U, known, X = setup(ctx, "rmat14", dim, L.DTYPE_BF16, hidden=hidden)
    nodes = np.flatnonzero(known).astype(np.int32)
    p0 = ctx.mlp_get_params()
    losses = ctx.mlp_train(nodes, steps=6, batch=512, lr=1e-3, seed=8)
    p1 = ctx.mlp_get_params()
    for _ in range(2):
        ctx.mlp_create(2, hidden=hidden, act_dtype=L.DTYPE_BF16, seed=11)
        assert np.array_equal(ctx.mlp_get_params(), p0)
        few = nodes[:10]
        ctx.mlp_features_rows(known, few)
        feats = np.empty((g.n_nodes, OM.in_width(dim)), np.float32)
        ctx.mlp_get_features(feats)
        others = np.ones(g.n_nodes, bool)
        others[few] = False
        assert not feats[others].any() and feats[few].any()
        ctx.mlp_features(known)
        again = ctx.mlp_train(nodes, steps=6, batch=512, lr=1e-3, seed=8)
        assert np.array_equal(again, losses) and np.array_equal(ctx.mlp_get_params(), p1)
    # another width, then this one again
    ctx.mlp_create(2, hidden=64, act_dtype=L.DTYPE_BF16, seed=11)
    ctx.mlp_create(2, hidden=hidden, act_dtype=L.DTYPE_BF16, seed=11)
    assert np.array_equal(ctx.mlp_get_params(), p0)


def test_predict_bf16_activations_on_the_tensor_cores(ctx):
    """BF16 activations at d = 128, hidden 256: both forward products run on
    the tensor cores (activations by TMA, weights as BF16 hi/lo pairs).
    Predictions of 1, 77, 128 and 40,000 rows (a partial tile, one tile, and
    313 tiles, so that every CTA takes several tiles and both accumulators
    alternate) against the oracle's FP64 forward pass with x and h rounded to
    BF16, element by element, within 1e-3.  That bound allows for the
    roundings of h to BF16 that fall the other way (a sum off by a few parts
    in 10^6 changes about one h value in 10^3, and a row has 256).  The
    product itself is pinned by the median error: the hi/lo weights carry
    about 17 significant bits, so the typical output is within 1e-5 of the
    largest (TF32 weights, 11 bits, would give about 1e-4)."""
    from paper_2604_09419_gb300 import line as L
    dim, hidden = 128, 256
    g, U, known, X = setup(ctx, "rmat14", dim, L.DTYPE_BF16, hidden=hidden)
    rng = np.random.default_rng(9)
    p = OM.init_params(dim, hidden, 11)
    p["b1"] = rng.normal(size=hidden) * 0.1
    p["b2"] = rng.normal(size=dim) * 0.01
    pv = flat(p).astype(np.float32)
    ctx.mlp_set_params(pv)
    p = unflat(pv, dim, hidden)
    for n_rows in (1, 77, 128, 40_000):
        rows = rng.integers(0, g.n_nodes, n_rows).astype(np.int32)
        y = np.empty((n_rows, dim), np.float32)
        ctx.mlp_predict(rows, y)
        want = OM.predict(p, X[rows], act_bf16=True)
        ex = elementwise_excess(y, want, 1e-3)
        assert ex <= 0, (n_rows, ex)
        med = float(np.median(np.abs(y - want))) / float(np.abs(want).max())
        assert med <= 1e-5, (n_rows, med)


@pytest.mark.parametrize("table_dtype", [0, 1])
def test_predict_into_rows(ctx, table_dtype):
    from paper_2604_09419_gb300 import line as L
    dim, hidden = 16, 32
    g = G.graph("tiny")
    G.upload(ctx, g)
    U, C = trained_tables("tiny", dim, 60_000, 5)
    U, C = G.upload_tables(ctx, 2, U, C, dtype=table_dtype)
    held, _ = I.hold_out_nodes(g, 0.2, seed=2)
    known = (~held).astype(np.uint8)
    ctx.mlp_create(2, hidden=hidden, act_dtype=L.DTYPE_F32, seed=3)
    ctx.mlp_features(known)
    rows = np.flatnonzero(held).astype(np.int32)
    y = np.empty((len(rows), dim), np.float32)
    ctx.mlp_predict(rows, y)
    X = OM.features(g.n_nodes, g.src, g.dst, g.w, U, known.astype(bool))
    want = OM.predict(OM.init_params(dim, hidden, 3), X[rows])
    np.testing.assert_allclose(y, want, rtol=1e-5, atol=1e-6)
    before, _ = G.tables(ctx, g, 2, dim)
    ctx.mlp_predict(rows)
    after, _ = G.tables(ctx, g, 2, dim)
    stored = y if table_dtype == 0 else G.bf16_round(y)
    assert np.array_equal(after[rows], stored)
    rest = np.flatnonzero(~held)
    assert np.array_equal(after[rest], before[rest])


def test_mlp_errors(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(2, 16, L.DTYPE_F32, seed=1)
    rows = np.arange(4, dtype=np.int32)
    with pytest.raises(L.LineError) as ei:  # no MLP after a graph of another size
        G.upload(ctx, G.graph("rmat14"))
        ctx.mlp_grad(rows)
    assert ei.value.status == L.LINE_ERR_STATE
    G.upload(ctx, g)
    ctx.init_embeddings(2, 16, L.DTYPE_F32, seed=1)
    ctx.mlp_create(2, hidden=16, act_dtype=L.DTYPE_F32, seed=1)
    with pytest.raises(L.LineError) as ei:  # no features yet
        ctx.mlp_grad(rows)
    assert ei.value.status == L.LINE_ERR_STATE
    ctx.mlp_features(np.ones(g.n_nodes, np.uint8))
    with pytest.raises(L.LineError) as ei:
        ctx.mlp_create(3, 16, L.DTYPE_F32, 1)
    assert ei.value.status == L.LINE_ERR_ARG
    ctx.mlp_create(2, hidden=16, act_dtype=L.DTYPE_F32, seed=1)
    ctx.mlp_features(np.ones(g.n_nodes, np.uint8))
    with pytest.raises(L.LineError) as ei:
        ctx.mlp_train(np.array([0, g.n_nodes], np.int32), steps=2, batch=64)
    assert ei.value.status == L.LINE_ERR_ARG
    # still usable
    assert np.isfinite(ctx.mlp_grad(rows))


def incident_pairs(g, held, hs, hd, seed):
    """Held-out edges with a held-out endpoint, and as many non-edges with one."""
    inc = held[hs] | held[hd]
    ps, pd = hs[inc], hd[inc]
    ns, nd = I.non_edges(g, 40 * len(ps) + 1000, seed=seed)
    m = held[ns] | held[nd]
    return ps, pd, ns[m][:len(ps)], nd[m][:len(ps)]


def test_warm_start_gain_over_random_rows(ctx):
    """R-MAT 14 with 10% of edges and 10% of nodes held out.  LINE (order 2,
    d = 128) trains on the kept nodes; the MLP learns their rows and
    initialises the held-out nodes' rows.  Scored by the inner product of U
    rows, the warm-started rows must separate the held-out nodes' held-out
    edges from non-edges far better than the random rows plain LINE gives
    them (and better than the mean-neighbour input alone), and after the same
    short refinement on the graph with the held-out nodes' edges the warm
    start must still lead in loss and in AUC over all held-out edges."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    tr, hs, hd = I.split_edges(g, 0.1, seed=4)
    ans, ad = I.non_edges(g, len(hs), seed=7)
    held, kept = I.hold_out_nodes(tr, 0.1, seed=5)
    ps, pd, ns, nd = incident_pairs(g, held, hs, hd, seed=6)
    assert len(ps) > 1000 and len(ns) == len(ps)
    G.upload(ctx, kept)
    ctx.init_embeddings(2, 128, L.DTYPE_F32, seed=7)
    ctx.train_steps(2, 128, 5, 20 * kept.n_arcs, 8, batch=4096)
    G.upload(ctx, tr)  # same node count: the tables are kept
    U0, C0 = G.tables(ctx, tr, 2, 128)
    rows = np.flatnonzero(held).astype(np.int32)
    ctx.mlp_create(2, hidden=256, act_dtype=L.DTYPE_BF16, seed=9)
    ctx.mlp_features((~held).astype(np.uint8))
    train_nodes = np.flatnonzero(~held & (np.bincount(kept.src, minlength=g.n_nodes) > 0)).astype(np.int32)
    losses = ctx.mlp_train(train_nodes, steps=400, batch=1024, lr=1e-3, seed=10)
    assert losses[-20:].mean() < 0.5 * losses[:5].mean()
    X = np.empty((g.n_nodes, 144), np.float32)
    ctx.mlp_get_features(X)
    auc_random, _ = ctx.eval_auc(2, ps, pd, ns, nd)
    ctx.mlp_predict(rows)
    auc_mlp, _ = ctx.eval_auc(2, ps, pd, ns, nd)
    U_mlp, _ = G.tables(ctx, tr, 2, 128)
    U_mean = U0.copy()
    U_mean[rows] = X[rows, 1:129]
    ctx.set_embeddings(2, L.WHICH_U, U_mean, L.DTYPE_F32)
    auc_mean, _ = ctx.eval_auc(2, ps, pd, ns, nd)

    def refine(U):
        ctx.set_embeddings(2, L.WHICH_U, U, L.DTYPE_F32)
        ctx.set_embeddings(2, L.WHICH_C, C0, L.DTYPE_F32)
        ctx.train_steps(2, 128, 5, tr.n_arcs, 11, batch=4096, lr0=0.0025, total=tr.n_arcs)
        return ctx.eval_auc(2, hs, hd, ans, ad)[0], ctx.eval_loss(2, 5, 12, 200_000)

    auc_r, loss_r = refine(U0)
    auc_m, loss_m = refine(U_mlp)
    print(f"held-out-node edges AUC: random {auc_random:.4f}, mean-neighbour {auc_mean:.4f}, MLP {auc_mlp:.4f}; "
          f"after refinement, all held-out edges: random {auc_r:.4f} (loss {loss_r:.1f}), "
          f"MLP {auc_m:.4f} (loss {loss_m:.1f})")
    assert auc_mlp > auc_random + 0.2 and auc_mlp > auc_mean
    assert auc_m > auc_r and loss_m < loss_r
