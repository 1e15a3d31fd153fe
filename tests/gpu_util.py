"""Helpers shared by the GPU tests: graph upload through the C ABI, table
read-back, and cached oracle tables."""
import functools

import numpy as np

import oracle as O
from paper_2604_09419_gb300 import inputs as I


def context():
    import torch

    from paper_2604_09419_gb300 import line as L
    torch.cuda.set_device(0)
    return L.Context(0, torch.cuda.current_stream().cuda_stream)


def upload(ctx, g, host=False):
    """Build the alias tables of graph g (device buffers, or host arrays)."""
    import torch
    if host:
        ctx.build_alias(g.n_nodes, g.src, g.dst, g.w)
    else:
        ctx.build_alias(g.n_nodes, torch.from_numpy(g.src).cuda(), torch.from_numpy(g.dst).cuda(),
                        torch.from_numpy(g.w).cuda())


def tables(ctx, g, order, dim):
    from paper_2604_09419_gb300 import line as L
    U = L.table_numpy(ctx, g.n_nodes, dim, order, L.WHICH_U)
    C = L.table_numpy(ctx, g.n_nodes, dim, order, L.WHICH_C) if order == 2 else None
    return U, C


def gpu_alias(ctx, g, which):
    from paper_2604_09419_gb300 import line as L
    n = g.n_arcs if which == L.TABLE_EDGE else g.n_nodes
    thr = np.empty(n, np.uint32)
    alias = np.empty(n, np.uint32)
    ctx.get_alias(which, thr, alias)
    return thr, alias


def gpu_samples(ctx, K, seed, t0, count, domain=0):
    out = np.empty((count, K + 2), np.int32)
    ctx.sample_debug(K, seed, domain, t0, count, out)
    return out


@functools.lru_cache(maxsize=8)
def graph(name):
    if name == "tiny":
        return I.tiny_chung_lu()
    if name == "rmat14":
        return I.rmat(14, seed=3)
    if name == "dchung":
        return I.chung_lu_directed(n=20000, m=300000, seed=1)
    if name == "rmat20":
        return I.rmat20()
    if name == "two":
        return I.canonicalize(2, np.array([0]), np.array([1]), None, symmetrize=True)
    if name == "isolated":
        # a star plus isolated nodes: most nodes have degree 0
        return I.canonicalize(5000, np.zeros(40, np.int64), np.arange(1, 41), None, symmetrize=True)
    raise KeyError(name)


@functools.lru_cache(maxsize=8)
def oracle_tables(name):
    return O.Tables(graph(name))


def oracle_run(name, order, dim, K, n, seed, B, init_seed, **kw):
    T = oracle_tables(name)
    g = graph(name)
    U = O.init_uniform(g.n_nodes, dim, init_seed)
    C = np.zeros_like(U) if order == 2 else None
    O.train(T, U, C, order=order, K=K, n_samples=n, seed=seed, batch=B, **kw)
    return U, C


def bf16_round(x) -> np.ndarray:
    """Round to the nearest BF16 value (ties to even), returned as float32."""
    b = np.ascontiguousarray(x, np.float32).view(np.uint32).astype(np.uint64)
    b = (b + 0x7FFF + ((b >> 16) & 1)) >> 16 << 16
    return b.astype(np.uint32).view(np.float32)


def upload_tables(ctx, order, U, C=None, dtype=0):
    """Install host tables (e.g. the oracle's) as the context's tables of
    `order`; returns the FP64 copies of the values actually stored (FP32, or
    BF16-rounded when dtype is BF16)."""
    from paper_2604_09419_gb300 import line as L
    dim = U.shape[1]
    ctx.init_embeddings(order, dim, dtype, seed=0)
    out = []
    for which, X in ((L.WHICH_U, U), (L.WHICH_C, C)):
        if X is None:
            continue
        X32 = np.ascontiguousarray(X, np.float32)
        if dtype == L.DTYPE_BF16:
            X32 = bf16_round(X32)
        ctx.set_embeddings(order, which, X32, L.DTYPE_F32)
        out.append(X32.astype(np.float64))
    return out if len(out) > 1 else out[0]
