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
