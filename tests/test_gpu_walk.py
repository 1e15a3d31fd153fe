"""The walk sampler on the GPU (Algorithms 2-3, the local walk) against the
oracle, through the C ABI:

* the records of the walk sampler bit-exact (weighted root arc, weighted
  steps by running FP64 weight sums, dead ends stepping back, the windowed
  pairs, the edge sampler's negatives), on graphs with hubs of thousands of
  arcs, non-integer weights and dead ends, from sample windows that start
  inside a walk;
* FP32 training with walk pairs within 1e-5 of the FP64 oracle, in both
  orders, both modes, with walks split across pre-pass chunks, and for the
  concurrent two-order call;
* walk reuse (each walk's pairs serving r passes): samples bit-exact and
  training within 1e-5 in the minibatch and the one-worker Hogwild schedule;
* argument errors.
"""
import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = 1e-5


@pytest.fixture(scope="module")
def ctx():
    c = G.context()
    yield c
    c.close()


def _graph(name):
    if name == "hub":
        # node 0 -> 1 .. 5000 with lognormal weights; every other node -> 0 and
        # to two neighbours; node 5001 is a dead end reached from node 1
        rng = np.random.default_rng(7)
        n = 5002
        src = np.concatenate([np.zeros(5000, np.int64), np.arange(1, 5001), np.arange(1, 5001), [1]])
        dst = np.concatenate([np.arange(1, 5001), np.zeros(5000, np.int64), (np.arange(1, 5001) % 5000) + 1, [5001]])
        w = np.concatenate([rng.lognormal(0, 1, 5000), rng.uniform(0.5, 2, 10000), [3.0]])
        return I.canonicalize(n, src, dst, w, symmetrize=False)
    return G.graph(name)


_cache = {}


def _setup(ctx, name):
    if name not in _cache:
        g = _graph(name)
        _cache[name] = (g, O.Tables(g), O.walk_cumw(g))
    g, T, cw = _cache[name]
    G.upload(ctx, g)
    return g, T, cw


def _gpu_walk(ctx, K, seed, L, W, t0, count):
    out = np.empty((count, K + 2), np.int32)
    ctx.sample_walk_debug(K, seed, L, W, t0, count, out)
    return out


@pytest.mark.parametrize("name", ["tiny", "dchung", "hub"])
@pytest.mark.parametrize("L,W", [(1, 1), (5, 5), (20, 3), (80, 10), (1024, 16)])
def test_walk_samples_bit_exact(ctx, name, L, W):
    g, T, cw = _setup(ctx, name)
    P = O.walk_pairs_per_walk(L, W)
    seed = 0x5EED1234ABC
    for t0, count, K in [(0, 20_000, 5), (P // 2 + 3, 7777, 0), ((1 << 33) + 11, 3000, 2)]:
        got = _gpu_walk(ctx, K, seed, L, W, t0, count)
        want = O.sample_walk(T, cw, seed, t0, count, K, L, W)
        assert np.array_equal(got, want), (name, L, W, t0)


@pytest.mark.parametrize("name", ["tiny", "dchung"])
def test_walk_samples_with_reuse_bit_exact(ctx, name):
    g, T, cw = _setup(ctx, name)
    L, W, r = 30, 2, 3
    P = O.walk_pairs_per_walk(L, W)
    for t0, count, K in [(0, 20_000, 5), (r * P + P // 2, 5000, 1)]:
        out = np.empty((count, K + 2), np.int32)
        ctx.sample_walk_debug(K, 77, L, W, t0, count, out, reuse=r)
        assert np.array_equal(out, O.sample_walk(T, cw, 77, t0, count, K, L, W, reuse=r)), (name, t0)


def test_walk_training_with_reuse(ctx):
    from paper_2604_09419_gb300 import line as L_
    g, T, cw = _setup(ctx, "tiny")
    n, B = 40_000, 512
    for mode in (L_.MODE_BATCHED, L_.MODE_HOGWILD):
        ctx.init_embeddings(2, 32, L_.DTYPE_F32, seed=1)
        kw = {"hogwild_workers": 1} if mode == L_.MODE_HOGWILD else {}
        ctx.train_steps(2, 32, 5, n, 3, batch=B, walk_length=20, window=2, walk_reuse=4, mode=mode, **kw)
        U, C = G.tables(ctx, g, 2, 32)
        Uo = O.init_uniform(g.n_nodes, 32, 1)
        Co = np.zeros_like(Uo)
        fn = O.train_pairwise if mode == L_.MODE_HOGWILD else O.train
        fn(T, Uo, Co, order=2, K=5, n_samples=n, seed=3, batch=B, walk=(cw, 20, 2, 4))
        err = max(np.abs(U - Uo).max(), np.abs(C - Co).max())
        assert err <= TOL, (mode, err)


def test_walk_tables_follow_a_new_graph(ctx):
    """The per-node arc offsets and weight sums are rebuilt with the graph."""
    for name in ("hub", "tiny", "hub"):
        g, T, cw = _setup(ctx, name)
        got = _gpu_walk(ctx, 1, 3, 30, 4, 100, 5000)
        assert np.array_equal(got, O.sample_walk(T, cw, 3, 100, 5000, 1, 30, 4)), name


def _train_walk(ctx, name, order, dim, K, n, B, L, W, seed=5, **okw):
    from paper_2604_09419_gb300 import line as L_
    g, T, cw = _setup(ctx, name)
    ctx.init_embeddings(order, dim, L_.DTYPE_F32, seed=1)
    ctx.train_steps(order, dim, K, n, seed, batch=B, walk_length=L, window=W, **okw)
    U, C = G.tables(ctx, g, order, dim)
    Uo = O.init_uniform(g.n_nodes, dim, 1)
    Co = np.zeros_like(Uo) if order == 2 else None
    O.train(T, Uo, Co, order=order, K=K, n_samples=n, seed=seed, batch=B, walk=(cw, L, W))
    err = np.abs(U - Uo).max()
    if order == 2:
        err = max(err, np.abs(C - Co).max())
    return U, C, err


@pytest.mark.parametrize("name,order,dim,K,n,B,L,W", [
    ("tiny", 2, 32, 5, 60_000, 256, 20, 3),
    ("tiny", 1, 64, 5, 60_000, 1024, 80, 10),
    ("dchung", 2, 128, 5, 50_000, 4096, 80, 10),
    ("hub", 2, 16, 3, 40_000, 500, 7, 7),
])
def test_walk_training_parity(ctx, name, order, dim, K, n, B, L, W):
    _, _, err = _train_walk(ctx, name, order, dim, K, n, B, L, W)
    assert err <= TOL, err


def test_walks_split_across_chunks_and_persistent_mode(ctx):
    from paper_2604_09419_gb300 import line as L_
    # one batch per chunk: the 755 pairs of each walk span several chunks
    U1, C1, err = _train_walk(ctx, "tiny", 2, 32, 5, 30_000, 256, 80, 10, chunk_batches=1)
    assert err <= TOL, err
    U2, C2, err = _train_walk(ctx, "tiny", 2, 32, 5, 30_000, 256, 80, 10, mode=L_.MODE_PERSISTENT)
    assert err <= TOL, err
    assert np.array_equal(U1, U2) and np.array_equal(C1, C2)


def test_walk_resume_split_is_bitwise(ctx):
    from paper_2604_09419_gb300 import line as L_
    g, _, _ = _setup(ctx, "tiny")
    n, B, Lw, W = 40_000, 256, 40, 5
    ctx.init_embeddings(2, 32, L_.DTYPE_F32, seed=1)
    ctx.train_steps(2, 32, 5, n, 5, batch=B, total=n, walk_length=Lw, window=W)
    full = G.tables(ctx, g, 2, 32)
    ctx.init_embeddings(2, 32, L_.DTYPE_F32, seed=1)
    split = 256 * 41  # inside a walk of 185 pairs
    ctx.train_steps(2, 32, 5, split, 5, batch=B, total=n, walk_length=Lw, window=W)
    ctx.train_steps(2, 32, 5, n - split, 5, batch=B, total=n, sample_offset=split, walk_length=Lw, window=W)
    U, C = G.tables(ctx, g, 2, 32)
    assert np.array_equal(U, full[0]) and np.array_equal(C, full[1])


def test_train_orders_with_walks(ctx):
    from paper_2604_09419_gb300 import line as L_
    g, T, cw = _setup(ctx, "dchung")
    n, B, K, dim = 40_000, 1024, 5, 32
    for o in (1, 2):
        ctx.init_embeddings(o, dim, L_.DTYPE_F32, seed=1)
    ctx.train_orders(dim, K, n, 9, batch=B, walk_length=30, window=4)
    for o in (1, 2):
        U, C = G.tables(ctx, g, o, dim)
        Uo = O.init_uniform(g.n_nodes, dim, 1)
        Co = np.zeros_like(Uo) if o == 2 else None
        O.train(T, Uo, Co, order=o, K=K, n_samples=n, seed=9, batch=B, walk=(cw, 30, 4))
        err = np.abs(U - Uo).max()
        if o == 2:
            err = max(err, np.abs(C - Co).max())
        assert err <= TOL, (o, err)


def test_walk_argument_errors(ctx):
    from paper_2604_09419_gb300 import line as L_
    _setup(ctx, "tiny")
    ctx.init_embeddings(2, 32, L_.DTYPE_F32, seed=1)
    with pytest.raises(L_.LineError) as ei:
        ctx.train_steps(2, 32, 5, 1000, 5, walk_length=10, window=2, walk_reuse=1025)
    assert ei.value.status == L_.LINE_ERR_ARG
    with pytest.raises(L_.LineError) as ei:
        ctx.sample_walk_debug(2, 1, 10, 2, 0, 10, np.empty((10, 4), np.int32), reuse=0)
    assert ei.value.status == L_.LINE_ERR_ARG
    for Lw, W in [(10, 0), (10, 11), (1025, 4), (-1, 1)]:
        with pytest.raises(L_.LineError) as ei:
            ctx.train_steps(2, 32, 5, 1000, 5, walk_length=Lw, window=W)
        assert ei.value.status == L_.LINE_ERR_ARG
        if Lw >= 1:
            with pytest.raises(L_.LineError) as ei:
                ctx.sample_walk_debug(2, 1, Lw, W, 0, 10, np.empty((10, 4), np.int32))
            assert ei.value.status == L_.LINE_ERR_ARG


def test_full_size_rmat20_walks(ctx):
    """The rmat20walk benchmark workload (R-MAT 20, L=100, W=2, d=128, K=5,
    B=4096) in the benchmark's launch configuration (both orders
    concurrently): sampled windows bit-exact, and a training prefix the
    oracle finishes in seconds within 1e-5."""
    from paper_2604_09419_gb300 import line as L_
    g = G.graph("rmat20")
    G.upload(ctx, g)
    T = G.oracle_tables("rmat20")
    cw = O.walk_cumw(g)
    total = 335_544_320
    for t0 in (0, total - 200_000):
        out = np.empty((200_000, 7), np.int32)
        ctx.sample_walk_debug(5, 1000, 100, 2, t0, 200_000, out)
        assert np.array_equal(out, O.sample_walk(T, cw, 1000, t0, 200_000, 5, 100, 2)), t0
    n = 4096 * 48
    for o in (1, 2):
        ctx.init_embeddings(o, 128, L_.DTYPE_F32, seed=o)
    ctx.train_orders(128, 5, n, 1000, batch=4096, total=total, walk_length=100, window=2)
    for o in (1, 2):
        U, C = G.tables(ctx, g, o, 128)
        Uo = O.init_uniform(g.n_nodes, 128, o)
        Co = np.zeros_like(Uo) if o == 2 else None
        O.train(T, Uo, Co, order=o, K=5, n_samples=n, seed=1000, batch=4096, lr_total=total, walk=(cw, 100, 2))
        err = np.abs(U - Uo).max()
        if o == 2:
            err = max(err, np.abs(C - Co).max())
        assert err <= TOL, (o, err)
