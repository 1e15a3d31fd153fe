"""GPU path vs the FP64 oracle, through the C ABI.

* alias tables bit-exact (Eq. 1 and Algorithm 3's weight-proportional pick);
* sampled indices bit-exact (Algorithm 1's positive + K negatives per sample);
* FP32 embeddings within 1e-5 max-abs of the FP64 oracle (minibatch LINE,
  Eq. 2-4), across dims, orders, batch sizes, K, lambda and alpha_neg;
* bitwise determinism, resume equivalence, schedule equivalence;
* the loss of the GPU tables against the oracle's loss of the same tables.
"""
import numpy as np
import pytest

import oracle as O
from tests import gpu_util as G

pytestmark = pytest.mark.gpu

TOL = 1e-5  # FP32 GPU vs FP64 oracle, max abs (the target's stated bound)


@pytest.fixture(scope="module")
def ctx():
    c = G.context()
    yield c
    c.close()


@pytest.mark.parametrize("name", ["tiny", "rmat14", "dchung", "two", "isolated"])
def test_alias_tables_bit_exact(ctx, name):
    from paper_2604_09419_gb300 import line as L
    g = G.graph(name)
    T = G.oracle_tables(name)
    G.upload(ctx, g)
    thr, alias = G.gpu_alias(ctx, g, L.TABLE_EDGE)
    assert np.array_equal(thr, T.thr_e) and np.array_equal(alias, T.alias_e)
    thr, alias = G.gpu_alias(ctx, g, L.TABLE_NEG)
    assert np.array_equal(thr, T.thr_n) and np.array_equal(alias, T.alias_n)


def test_alias_rebuilds_in_one_context(ctx):
    """One context, graphs of growing, shrinking and equal sizes, weighted
    and unit-weight (the graph buffers of an earlier build are reused when
    large enough): both alias tables bit-exact after every build."""
    import dataclasses

    import torch

    from paper_2604_09419_gb300 import line as L
    tiny = G.graph("tiny")
    unit = dataclasses.replace(tiny, w=np.ones(tiny.n_arcs, np.float32))
    seq = [("rmat14", G.graph("rmat14"), True), ("tiny", tiny, True), ("tiny unit", unit, False),
           ("dchung", G.graph("dchung"), True), ("rmat14", G.graph("rmat14"), True)]
    for name, g, weighted in seq:
        T = O.Tables(g)
        w = torch.from_numpy(g.w).cuda() if weighted else None
        ctx.build_alias(g.n_nodes, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(), w)
        for which, (thr_o, alias_o) in ((L.TABLE_EDGE, (T.thr_e, T.alias_e)), (L.TABLE_NEG, (T.thr_n, T.alias_n))):
            thr, alias = G.gpu_alias(ctx, g, which)
            assert np.array_equal(thr, thr_o) and np.array_equal(alias, alias_o), (name, which)


def test_alias_host_buffers(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    T = G.oracle_tables("rmat14")
    G.upload(ctx, g, host=True)
    thr, alias = G.gpu_alias(ctx, g, L.TABLE_NEG)
    assert np.array_equal(thr, T.thr_n) and np.array_equal(alias, T.alias_n)


@pytest.mark.parametrize("name", ["tiny", "dchung"])
def test_samples_bit_exact(ctx, name):
    g = G.graph(name)
    T = G.oracle_tables(name)
    G.upload(ctx, g)
    # a whole tiny run (100,000 samples, K = 5), and windows with t_hi != 0
    for t0, count, K, domain in [(0, 100_000, 5, 0), ((3 << 32) - 17, 5000, 5, 0), (12345, 3000, 0, 3),
                                 (99, 2000, 32, 0)]:
        got = G.gpu_samples(ctx, K, 0xABCDEF12345, t0, count, domain)
        want = O.sample(T, 0xABCDEF12345, t0, count, K, domain)
        assert np.array_equal(got, want), (t0, count, K)


def _train_both(ctx, name, order, dim, K, n, B, seed=5, init_seed=1, check_tol=True, **kw):
    from paper_2604_09419_gb300 import line as L
    g = G.graph(name)
    G.upload(ctx, g)
    ctx.init_embeddings(order, dim, L.DTYPE_F32, seed=init_seed)
    okw = {k: v for k, v in kw.items() if k in ("mode", "chunk_batches", "warps_per_block")}
    lam = kw.get("lam", 0.0)
    alpha = kw.get("alpha_neg", 1.0)
    ctx.train_steps(order, dim, K, n, seed, batch=B, lam=lam, alpha_neg=alpha, **okw)
    U, C = G.tables(ctx, g, order, dim)
    Uo, Co = G.oracle_run(name, order, dim, K, n, seed, B, init_seed, lam=lam, alpha_neg=alpha)
    err = np.abs(U - Uo).max()
    if order == 2:
        err = max(err, np.abs(C - Co).max())
    if check_tol:
        assert err <= TOL, err
    return U, C, err


@pytest.mark.parametrize("order", [2, 1])
def test_tiny_config_parity(ctx, order):
    """Tiny Chung-Lu, d=16, K=5, 100,000 samples, B=256 (390 full batches + 160), lr 0.025 linear."""
    _, _, err = _train_both(ctx, "tiny", order, 16, 5, 100_000, 256)
    print(f"tiny order {order}: max |GPU - oracle| = {err:.3e}")


@pytest.mark.parametrize("dim", [32, 64, 128, 256])
def test_dims(ctx, dim):
    _train_both(ctx, "tiny", 2, dim, 5, 20_000, 128)


@pytest.mark.parametrize("B,n,K", [(1, 300, 5), (7, 1000, 3), (5000, 3000, 5), (256, 10_000, 0), (64, 5000, 1),
                                   (100, 4000, 32)])
def test_batch_and_k_edge_cases(ctx, B, n, K):
    _train_both(ctx, "tiny", 2, 16, K, n, B)


def test_decay_and_alpha(ctx):
    _train_both(ctx, "tiny", 2, 32, 5, 30_000, 256, lam=1e-3, alpha_neg=0.5)
    _train_both(ctx, "tiny", 1, 32, 5, 30_000, 256, lam=1e-3, alpha_neg=0.5)


def test_weighted_directed_graph(ctx):
    _train_both(ctx, "dchung", 2, 64, 5, 50_000, 512)


def test_ragged_rmat(ctx):
    """R-MAT scale 14: hub rows appear many times per batch (long segments)."""
    _train_both(ctx, "rmat14", 2, 128, 5, 40_000, 4096)
    _train_both(ctx, "rmat14", 1, 128, 5, 40_000, 4096)


def _run(ctx, g, order, dim, K, n, B, seed=5, **kw):
    from paper_2604_09419_gb300 import line as L
    ctx.init_embeddings(order, dim, L.DTYPE_F32, seed=1)
    ctx.train_steps(order, dim, K, n, seed, batch=B, **kw)
    return G.tables(ctx, g, order, dim)


def test_determinism_and_schedules(ctx):
    g = G.graph("rmat14")
    G.upload(ctx, g)
    a = _run(ctx, g, 2, 64, 5, 60_000, 1024)
    b = _run(ctx, g, 2, 64, 5, 60_000, 1024)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    for cb in (1, 3, 7):
        c = _run(ctx, g, 2, 64, 5, 60_000, 1024, chunk_batches=cb)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]), cb
    for wpb in (1, 4, 16):
        c = _run(ctx, g, 2, 64, 5, 60_000, 1024, warps_per_block=wpb)
        assert np.array_equal(a[0], c[0]) and np.array_equal(a[1], c[1]), wpb


def test_graph_replay_matches_direct_launches_and_oracle(ctx):
    """Full chunks replayed from captured CUDA graphs (several chunks per
    set, a partial last chunk) give the same bits as direct launches, and the
    oracle's tables within the FP32 bound."""
    g = G.graph("tiny")
    G.upload(ctx, g)
    n, B = 100_000, 256
    direct = _run(ctx, g, 2, 16, 5, n, B, chunk_batches=16, graph=0)
    for cb in (16, 5):
        replay = _run(ctx, g, 2, 16, 5, n, B, chunk_batches=cb, graph=1)
        assert np.array_equal(direct[0], replay[0]) and np.array_equal(direct[1], replay[1]), cb
    U, C = G.oracle_run("tiny", 2, 16, 5, n, 5, B, 1)
    assert np.abs(replay[0] - U).max() <= TOL and np.abs(replay[1] - C).max() <= TOL
    # first order and BF16 tables through the same path
    d1 = _run(ctx, g, 1, 32, 5, 60_000, B, chunk_batches=8, graph=0)
    r1 = _run(ctx, g, 1, 32, 5, 60_000, B, chunk_batches=8, graph=1)
    assert np.array_equal(d1[0], r1[0])


def test_autotune_keeps_tables_and_returns_a_valid_configuration(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    G.upload(ctx, g)
    ctx.init_embeddings(2, 64, L.DTYPE_F32, seed=1)
    U0, C0 = G.tables(ctx, g, 2, 64)
    ctx.reset_stats()
    o, rate = ctx.autotune(2, 64, 5, batches=[1024, 4096], trial_samples=65_536, try_persistent=True)
    assert rate > 0 and o.batch in (1024, 4096) and o.chunk_batches >= 1 and o.graph == 1
    assert o.mode in (L.MODE_BATCHED, L.MODE_PERSISTENT)
    U1, C1 = G.tables(ctx, g, 2, 64)
    assert np.array_equal(U0, U1) and np.array_equal(C0, C1)
    assert ctx.stats().total_samples == 0
    # the tuned configuration trains to the same bits as the defaults at its batch size
    a = _run(ctx, g, 2, 64, 5, 50_000, o.batch)
    b = _run(ctx, g, 2, 64, 5, 50_000, o.batch, opts=o)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    # both orders at once: both tables untouched
    ctx.init_embeddings(1, 64, L.DTYPE_F32, seed=3)
    ctx.init_embeddings(2, 64, L.DTYPE_F32, seed=4)
    V1, _ = G.tables(ctx, g, 1, 64)
    V2, W2 = G.tables(ctx, g, 2, 64)
    o2, rate2 = ctx.autotune(1, 64, 5, batches=[2048, 4096], trial_samples=65_536, both_orders=True)
    assert rate2 > 0 and o2.batch in (2048, 4096)
    X1, _ = G.tables(ctx, g, 1, 64)
    X2, Y2 = G.tables(ctx, g, 2, 64)
    assert np.array_equal(V1, X1) and np.array_equal(V2, X2) and np.array_equal(W2, Y2)


def test_tables_recreated_in_place_with_another_type(ctx):
    """init_embeddings reuses the tables' memory: a run after tables of the
    other type (same addresses, replayed CUDA graphs of full chunks) equals
    the run of a fresh context."""
    g = G.graph("rmat14")
    n = 5 * (1 << 18) + 777

    def run(c, dtype):
        c.init_embeddings(2, 16, dtype, seed=2)
        c.train_steps(2, 16, 5, n, 9, batch=4096, total=n)
        return G.tables(c, g, 2, 16)

    fresh = {}
    for dtype in (0, 1):
        c = G.context()
        G.upload(c, g)
        fresh[dtype] = run(c, dtype)
        c.close()
    G.upload(ctx, g)
    for dtype in (0, 1, 0, 1):
        U, C = run(ctx, dtype)
        assert np.array_equal(U, fresh[dtype][0]) and np.array_equal(C, fresh[dtype][1]), dtype


@pytest.mark.parametrize("dtype", [0, 1])
def test_train_orders_long_call_equals_two_sequential_calls(ctx, dtype):
    """A call longer than one slice (the orders are issued in alternate
    slices of about 2^24 samples) with a ragged last batch: bitwise the
    tables of one train_steps call per order."""
    g = G.graph("rmat14")
    G.upload(ctx, g)
    n = (1 << 24) + 3 * 4096 + 1000 + 17
    B = 4096
    ctx.init_embeddings(1, 16, dtype, seed=1)
    ctx.init_embeddings(2, 16, dtype, seed=2)
    ctx.train_steps(1, 16, 5, n, 9, batch=B, total=n)
    ctx.train_steps(2, 16, 5, n, 9, batch=B, total=n)
    want1, _ = G.tables(ctx, g, 1, 16)
    want2 = G.tables(ctx, g, 2, 16)
    ctx.init_embeddings(1, 16, dtype, seed=1)
    ctx.init_embeddings(2, 16, dtype, seed=2)
    ctx.train_orders(16, 5, n, 9, batch=B, total=n)
    got1, _ = G.tables(ctx, g, 1, 16)
    got2 = G.tables(ctx, g, 2, 16)
    assert np.array_equal(want1, got1)
    assert np.array_equal(want2[0], got2[0]) and np.array_equal(want2[1], got2[1])


@pytest.mark.parametrize("dtype,cb,dim,K,extra", [(0, 0, 64, 5, {}), (0, 3, 64, 5, {}), (1, 2, 64, 5, {}),
                                                   (0, 0, 128, 5, {}), (0, 3, 128, 5, {}), (1, 2, 128, 5, {}),
                                                   (1, 0, 128, 5, {}), (0, 2, 128, 3, {"lam": 1e-3, "alpha_neg": 0.5}),
                                                   (0, 2, 128, 8, {})])
def test_train_orders_equals_two_sequential_calls(ctx, dtype, cb, dim, K, extra):
    """Both orders trained together on two streams give the tables of two
    separate calls: at the bench's d = 128 and at d = 64, for the register
    gather (K <= 7) and the staged one (K = 8), FP32 and BF16, with graph
    replays of full chunks (cb > 0) and with weight decay and a negative
    weight."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat14")
    G.upload(ctx, g)
    n, B = 80_000, 1024
    ctx.init_embeddings(1, dim, dtype, seed=1)
    ctx.init_embeddings(2, dim, dtype, seed=2)
    for order in (1, 2):
        ctx.train_steps(order, dim, K, n, 9, batch=B, chunk_batches=cb, total=2 * n, **extra)
    ctx.train_steps(1, dim, K, n, 9, batch=B, chunk_batches=cb, total=2 * n, sample_offset=n, **extra)
    ctx.train_steps(2, dim, K, n, 9, batch=B, chunk_batches=cb, total=2 * n, sample_offset=n, **extra)
    want1, _ = G.tables(ctx, g, 1, dim)
    want2 = G.tables(ctx, g, 2, dim)
    ctx.init_embeddings(1, dim, dtype, seed=1)
    ctx.init_embeddings(2, dim, dtype, seed=2)
    ctx.reset_stats()
    ctx.train_orders(dim, K, n, 9, batch=B, chunk_batches=cb, total=2 * n, **extra)
    ctx.train_orders(dim, K, n, 9, batch=B, chunk_batches=cb, total=2 * n, sample_offset=n, **extra)
    st = ctx.stats()
    assert st.update_samples == 4 * n
    got1, _ = G.tables(ctx, g, 1, dim)
    got2 = G.tables(ctx, g, 2, dim)
    assert np.array_equal(want1, got1)
    assert np.array_equal(want2[0], got2[0]) and np.array_equal(want2[1], got2[1])
    # both orders must exist with the given dim
    ctx.init_embeddings(1, 32, dtype, seed=1)
    with pytest.raises(L.LineError) as ei:
        ctx.train_orders(dim, K, n, 9)
    assert ei.value.status == L.LINE_ERR_STATE


def test_resume_split_is_bitwise(ctx):
    from paper_2604_09419_gb300 import line as L
    g = G.graph("tiny")
    G.upload(ctx, g)
    n, B = 50_000, 256
    full = _run(ctx, g, 2, 32, 5, n, B)
    ctx.init_embeddings(2, 32, L.DTYPE_F32, seed=1)
    split = 256 * 77
    ctx.train_steps(2, 32, 5, split, 5, batch=B, total=n)
    ctx.train_steps(2, 32, 5, n - split, 5, batch=B, total=n, sample_offset=split)
    U, C = G.tables(ctx, g, 2, 32)
    assert np.array_equal(U, full[0]) and np.array_equal(C, full[1])


def test_loss_matches_oracle_on_the_same_tables(ctx):
    """The GPU loss of oracle-trained tables, installed through the ABI,
    against the oracle's loss of the same (FP32-rounded) tables."""
    g = G.graph("tiny")
    G.upload(ctx, g)
    T = G.oracle_tables("tiny")
    U, C = G.oracle_run("tiny", 2, 16, 5, 50_000, 7, 256, 3)
    U, C = G.upload_tables(ctx, 2, U, C)
    for m in (1, 1000, 65_537):
        got = ctx.eval_loss(2, 5, 9, m)
        want = O.eval_loss(T, U, C, order=2, K=5, seed=9, m=m)
        assert abs(got - want) <= 1e-9 * abs(want), (m, got, want)
    U1, _ = G.oracle_run("tiny", 1, 16, 5, 20_000, 8, 256, 4)
    U1 = G.upload_tables(ctx, 1, U1)
    got = ctx.eval_loss(1, 5, 9, 4000)
    want = O.eval_loss(T, U1, None, order=1, K=5, seed=9, m=4000)
    assert abs(got - want) <= 1e-9 * abs(want)


def test_untouched_rows_and_zero_lr(ctx):
    g = G.graph("isolated")
    G.upload(ctx, g)
    from paper_2604_09419_gb300 import line as L
    ctx.init_embeddings(2, 16, L.DTYPE_F32, seed=3)
    U0, C0 = G.tables(ctx, g, 2, 16)
    ctx.train_steps(2, 16, 5, 5000, 1, batch=64, lr0=0.0)
    U1, C1 = G.tables(ctx, g, 2, 16)
    assert np.array_equal(U0, U1) and np.array_equal(C0, C1)
    ctx.train_steps(2, 16, 5, 5000, 1, batch=64)
    U2, C2 = G.tables(ctx, g, 2, 16)
    # nodes 41.. have degree 0: never drawn, rows unchanged
    assert np.array_equal(U2[41:], U0[41:]) and not C2[41:].any()
    assert not np.array_equal(U2[:41], U0[:41])


@pytest.mark.parametrize("name,order,dim,B,n", [("tiny", 2, 16, 256, 100_000), ("tiny", 1, 16, 256, 50_000),
                                               ("rmat14", 2, 128, 4096, 200_000), ("rmat14", 1, 128, 4096, 100_000),
                                               ("dchung", 2, 64, 1000, 50_000), ("tiny", 2, 256, 64, 20_000)])
def test_persistent_matches_batched_bitwise(ctx, name, order, dim, B, n):
    from paper_2604_09419_gb300 import line as L
    g = G.graph(name)
    G.upload(ctx, g)
    a = _run(ctx, g, order, dim, 5, n, B, mode=L.MODE_BATCHED)
    for cb in (0, 1, 5):
        b = _run(ctx, g, order, dim, 5, n, B, mode=L.MODE_PERSISTENT, chunk_batches=cb)
        assert np.array_equal(a[0], b[0]), cb
        if order == 2:
            assert np.array_equal(a[1], b[1]), cb


def test_persistent_parity_with_oracle(ctx):
    from paper_2604_09419_gb300 import line as L
    _train_both(ctx, "tiny", 2, 16, 5, 100_000, 256, mode=L.MODE_PERSISTENT)
    _train_both(ctx, "rmat14", 1, 128, 5, 40_000, 4096, mode=L.MODE_PERSISTENT)


def test_full_size_rmat20_prefix(ctx):
    """The benchmark's workload (R-MAT 20, d=128, K=5, B=4096) in the benchmark's
    launch configuration, on a prefix the oracle finishes in seconds."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("rmat20")
    G.upload(ctx, g)
    T = G.oracle_tables("rmat20")
    # alias tables and windows of draws at full size
    thr, alias = G.gpu_alias(ctx, g, L.TABLE_NEG)
    assert np.array_equal(thr, T.thr_n) and np.array_equal(alias, T.alias_n)
    thr, alias = G.gpu_alias(ctx, g, L.TABLE_EDGE)
    assert np.array_equal(thr, T.thr_e) and np.array_equal(alias, T.alias_e)
    for t0 in (0, 335_544_320 - 1_000_000):
        assert np.array_equal(G.gpu_samples(ctx, 5, 1000, t0, 1_000_000), O.sample(T, 1000, t0, 1_000_000, 5))
    n, total = 4096 * 48, 335_544_320
    for order, mode in ((2, L.MODE_PERSISTENT), (1, L.MODE_PERSISTENT), (2, L.MODE_BATCHED)):
        ctx.init_embeddings(order, 128, L.DTYPE_F32, seed=order)
        ctx.train_steps(order, 128, 5, n, 1000, batch=4096, total=total, mode=mode)
        U, C = G.tables(ctx, g, order, 128)
        Uo = O.init_uniform(g.n_nodes, 128, order)
        Co = np.zeros_like(Uo) if order == 2 else None
        O.train(T, Uo, Co, order=order, K=5, n_samples=n, seed=1000, batch=4096, lr_total=total)
        err = np.abs(U - Uo).max()
        if order == 2:
            err = max(err, np.abs(C - Co).max())
        print(f"rmat20 order {order} mode {mode}: max |GPU - oracle| = {err:.3e}")
        assert err <= TOL


def bf16_ulp(x):
    """Spacing of BF16 values at |x| (8 significant bits; the smallest normal
    binade's spacing below it)."""
    e = np.floor(np.log2(np.maximum(np.abs(x), 2.0 ** -126)))
    return 2.0 ** (e - 7)


def test_bf16_tables(ctx):
    """BF16 storage with FP32 arithmetic and stochastic rounding, against the
    oracle's BF16 mode (the FP64 batch sum, rounded to FP32, then
    stochastically to BF16 with the same bits).

    Batch by batch from the oracle's state: the GPU's FP32 sums differ from
    the FP64 sums by a few FP32 units in the last place, which flips a
    stochastic rounding with probability of about 2^-16 per unit, so each
    batch agrees to within one BF16 unit in the last place everywhere and
    exactly almost everywhere.  Over a whole run the flips carry forward, and
    the error against the oracle's BF16 run and against FP64 is stated."""
    from paper_2604_09419_gb300 import line as L
    g = G.graph("tiny")
    T = G.oracle_tables("tiny")
    G.upload(ctx, g)
    dim, n, B, seed = 64, 100_000, 256, 3
    ctx.init_embeddings(2, dim, L.DTYPE_BF16, seed=1)
    U0, C0 = G.tables(ctx, g, 2, dim)
    # the initial table is the FP32 initialisation rounded to nearest BF16
    Ui = O.round_bf16_rn(O.init_uniform(g.n_nodes, dim, 1))
    assert np.array_equal(U0.astype(np.float64), Ui) and not C0.any()
    ctx.train_steps(2, dim, 5, 5000, seed, batch=B, lr0=0.0)
    U1, C1 = G.tables(ctx, g, 2, dim)
    assert np.array_equal(U0, U1) and np.array_equal(C0, C1)
    # batch by batch (lambda != 0 on the second half), resynchronised to the
    # oracle after every batch
    Uo, Co = Ui.copy(), np.zeros_like(Ui)
    n_vals = n_exact = 0
    worst = 0.0
    for b in range(24):
        lam = 0.0 if b < 12 else 1e-3
        ctx.set_embeddings(2, L.WHICH_U, Uo.astype(np.float32))
        ctx.set_embeddings(2, L.WHICH_C, Co.astype(np.float32))
        ctx.train_steps(2, dim, 5, B, seed, batch=B, total=n, sample_offset=b * B, lam=lam)
        Ug, Cg = G.tables(ctx, g, 2, dim)
        O.train(T, Uo, Co, order=2, K=5, n_samples=B, seed=seed, batch=B, lr_total=n, sample_offset=b * B,
                lam=lam, bf16=True)
        for Xg, Xo in ((Ug, Uo), (Cg, Co)):
            d = np.abs(Xg.astype(np.float64) - Xo)
            lim = np.maximum(bf16_ulp(np.maximum(np.abs(Xg), np.abs(Xo))), 1e-9)
            worst = max(worst, float((d / lim).max()))
            n_vals += d.size
            n_exact += int((d == 0).sum())
    frac = n_exact / n_vals
    print(f"bf16 per batch (24 batches of {B}, d={dim}): {frac:.6f} of values bit-exact, "
          f"max difference {worst:.2f} BF16 ulp")
    assert worst <= 1.0 and frac >= 0.999
    # a whole run: both schedules bitwise equal; error against the oracle's
    # BF16 run and against FP64 stated
    runs = []
    for mode in (L.MODE_BATCHED, L.MODE_PERSISTENT):
        ctx.init_embeddings(2, dim, L.DTYPE_BF16, seed=1)
        ctx.train_steps(2, dim, 5, n, seed, batch=B, mode=mode)
        runs.append(G.tables(ctx, g, 2, dim))
    assert np.array_equal(runs[0][0], runs[1][0]) and np.array_equal(runs[0][1], runs[1][1])
    Ub, Cb = runs[0]
    gb = np.concatenate([Ub.ravel(), Cb.ravel()]).astype(np.float64)
    Uo, Co = Ui.copy(), np.zeros_like(Ui)
    O.train(T, Uo, Co, order=2, K=5, n_samples=n, seed=seed, batch=B, bf16=True)
    ob = np.concatenate([Uo.ravel(), Co.ravel()])
    Uf, Cf = Ui.copy(), np.zeros_like(Ui)
    O.train(T, Uf, Cf, order=2, K=5, n_samples=n, seed=seed, batch=B)
    of = np.concatenate([Uf.ravel(), Cf.ravel()])
    scale = np.abs(of).max()
    e_bf, e_64 = np.abs(gb - ob), np.abs(gb - of)
    print(f"bf16 whole run ({n} samples): vs oracle BF16 max {e_bf.max():.3e} rms {np.sqrt((e_bf ** 2).mean()):.3e} "
          f"({(e_bf == 0).mean():.4f} exact); vs FP64 max {e_64.max():.3e} rms {np.sqrt((e_64 ** 2).mean()):.3e}; "
          f"oracle BF16 vs FP64 max {np.abs(ob - of).max():.3e}; max |x| {scale:.3f}")
    assert e_bf.max() < 0.05 * scale and e_64.max() < 0.1 * scale
    # unbiased rounding: the mean signed error against FP64 is small against its spread
    diff = (gb - of)[gb != of]
    assert abs(diff.mean()) < 5 * diff.std() / np.sqrt(diff.size)
