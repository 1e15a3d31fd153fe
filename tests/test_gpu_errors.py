"""Error handling of the C ABI on the GPU, with failures made on the host side
or by a bounded device wait (nothing here faults, traps or hangs the GPU)."""
import numpy as np
import pytest

from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def test_bounded_wait_times_out_cleanly():
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    assert ctx.debug_wait_timeout(1000) == L.LINE_ERR_TIMEOUT
    # the context stays usable afterwards
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(2, 16, L.DTYPE_F32, 0)
    ctx.train_steps(2, 16, 5, 1000, 1, batch=64)
    ctx.close()


def test_bad_arguments_and_state():
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    lr = L.LR(0.025, 1, 1e-4, 0)
    o = L.train_opts_default()
    import ctypes
    # no graph yet
    st = L.lib.line_train_steps(ctx.h, 2, 16, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o))
    assert st == L.LINE_ERR_STATE
    g = G.graph("tiny")
    G.upload(ctx, g)
    # tables not initialised / wrong dim
    assert L.lib.line_train_steps(ctx.h, 2, 16, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_ERR_STATE
    ctx.init_embeddings(2, 16, L.DTYPE_F32, 0)
    assert L.lib.line_train_steps(ctx.h, 2, 32, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_ERR_STATE
    assert L.lib.line_train_steps(ctx.h, 3, 16, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_ERR_ARG
    assert L.lib.line_train_steps(ctx.h, 2, 16, 33, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_ERR_ARG
    o.batch = 0
    assert L.lib.line_train_steps(ctx.h, 2, 16, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_ERR_ARG
    assert L.lib.line_init_embeddings(ctx.h, 2, 48, 0, 0) == L.LINE_ERR_ARG
    # argument errors are not sticky
    o.batch = 64
    assert L.lib.line_train_steps(ctx.h, 2, 16, 5, ctypes.byref(lr), 100, 1, ctypes.byref(o)) == L.LINE_OK
    ctx.close()


def test_graph_validation():
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    g = G.graph("tiny")
    bad_order = g.src[::-1].copy()
    with pytest.raises(L.LineError) as e:
        ctx.build_alias(g.n_nodes, bad_order, g.dst, g.w)
    assert e.value.status == L.LINE_ERR_VALIDATE
    bad_w = g.w.copy()
    bad_w[7] = -1.0
    with pytest.raises(L.LineError) as e:
        ctx.build_alias(g.n_nodes, g.src, g.dst, bad_w)
    assert e.value.status == L.LINE_ERR_VALIDATE
    bad_id = g.dst.copy()
    bad_id[3] = g.n_nodes
    with pytest.raises(L.LineError) as e:
        ctx.build_alias(g.n_nodes, g.src, bad_id, g.w)
    assert e.value.status == L.LINE_ERR_VALIDATE
    # a valid graph still builds on the same context
    G.upload(ctx, g)
    assert ctx.graph_info() == (g.n_nodes, g.n_arcs)
    ctx.close()


def test_set_get_roundtrip():
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(2, 32, L.DTYPE_F32, 0)
    rng = np.random.default_rng(0)
    rows = np.array([5, 0, 999, 17], np.int32)
    vals = rng.normal(size=(4, 32)).astype(np.float32)
    U0, _ = G.tables(ctx, g, 2, 32)
    ctx.set_embeddings(2, L.WHICH_U, vals, L.DTYPE_F32, rows)
    U1, _ = G.tables(ctx, g, 2, 32)
    want = U0.copy()
    want[rows] = vals
    assert np.array_equal(U1, want)
    with pytest.raises(L.LineError):
        ctx.set_embeddings(2, L.WHICH_U, vals, L.DTYPE_F32, np.array([1, 2, 3, 5000], np.int32))
    ctx.close()


def test_allocation_failure_is_reported_and_not_sticky():
    """A real device allocation failure (tables of 2^29 nodes x 256 FP32
    values, 549 GB, far above the GPU's memory; the first allocation already
    fails, so nothing large is ever held): LINE_ERR_OOM, nothing is kept,
    and the context goes on working."""
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    n = 1 << 29
    ctx.build_alias(n, np.array([0, 1], np.int32), np.array([1, 0], np.int32), None)
    with pytest.raises(L.LineError) as e:
        ctx.init_embeddings(2, 256, L.DTYPE_F32, 0)
    assert e.value.status == L.LINE_ERR_OOM
    g = G.graph("tiny")
    G.upload(ctx, g)
    ctx.init_embeddings(2, 16, L.DTYPE_F32, 0)
    ctx.train_steps(2, 16, 5, 1000, 1, batch=64)
    ctx.close()
