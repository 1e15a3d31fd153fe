"""The seeded graph generators: determinism and canonical form (no GPU)."""
import numpy as np

from paper_2604_09419_gb300 import inputs as I


def _canonical(g):
    assert g.src.dtype == np.int32 and g.dst.dtype == np.int32 and g.w.dtype == np.float32
    assert np.all(g.src[1:] >= g.src[:-1])
    key = g.src.astype(np.int64) * g.n_nodes + g.dst
    assert np.all(key[1:] > key[:-1])  # sorted, no duplicates
    assert not np.any(g.src == g.dst)
    assert np.all(g.w > 0)
    assert g.src.min() >= 0 and g.dst.max() < g.n_nodes


def _symmetric(g):
    fwd = g.src.astype(np.int64) * g.n_nodes + g.dst
    rev = g.dst.astype(np.int64) * g.n_nodes + g.src
    order = np.argsort(rev)
    assert np.array_equal(fwd, rev[order])
    assert np.array_equal(g.w, g.w[order])


def test_tiny_chung_lu():
    a, b = I.tiny_chung_lu(), I.tiny_chung_lu()
    assert np.array_equal(a.src, b.src) and np.array_equal(a.dst, b.dst)
    _canonical(a)
    _symmetric(a)
    assert a.n_nodes == 1000
    assert 9500 <= a.n_arcs // 2 <= 10500
    assert np.all(a.w == 1.0)
    deg = np.diff(a.row_ptr())
    assert deg[0] > 20 * np.median(deg)  # power-law head


def test_rmat_small():
    g = I.rmat(12, seed=1)
    _canonical(g)
    _symmetric(g)
    assert np.array_equal(g.w, np.round(g.w))  # merged duplicates are integer weights
    assert g.w.max() > 1
    deg = np.diff(g.row_ptr())
    assert deg.max() > 50 * max(1, np.median(deg))
    assert not np.array_equal(I.rmat(12, seed=2).dst, g.dst)


def test_directed_chung_lu_small():
    g = I.chung_lu_directed(n=5000, m=50000, seed=0)
    _canonical(g)
    assert g.directed
    deg = np.bincount(g.src, minlength=g.n_nodes)
    assert deg[:10].sum() > deg[-1000:].sum()
    # lognormal(0, 1) weights: median log-weight near 0, spread near 1
    lw = np.log(g.w.astype(np.float64))
    assert abs(np.median(lw)) < 0.1 and 0.8 < lw.std() < 1.3


def test_split_edges():
    g = I.tiny_chung_lu()
    train, hs, hd = I.split_edges(g, 0.1, seed=0)
    _symmetric(train)
    assert np.all(hs < hd)
    held = set(zip(hs.tolist(), hd.tolist()))
    tr = set(zip(train.src.tolist(), train.dst.tolist()))
    assert not any((s, d) in tr or (d, s) in tr for s, d in held)
    assert abs(len(held) - 0.1 * g.n_arcs / 2) < 0.03 * g.n_arcs / 2
