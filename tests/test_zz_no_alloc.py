"""line_eval_loss_noalloc: the loss evaluation for callers that cannot
allocate device memory while they run (a service that reserved all device
memory up front, a latency-bound loop where cudaMalloc/cudaFree would
synchronise the device).  Its scratch is one fixed device array that every
call reuses, so two calls in a row must each agree with the allocating
line_eval_loss; sizes beyond the array are refused; and the calls leave the
device's free memory unchanged.

Both calls run the same loss kernel and the same fixed-order FP64 sum, so
they agree bit for bit.  This file is named to be collected last.
"""
import ctypes

import pytest
import torch

from tests import gpu_util as G

pytestmark = pytest.mark.gpu


def test_noalloc_loss_matches_allocating_call_twice_in_a_row():
    from paper_2604_09419_gb300 import line as L
    ctx = G.context()
    try:
        g = G.graph("tiny")
        G.upload(ctx, g)
        ctx.init_embeddings(2, 16, L.DTYPE_F32, seed=1)
        ctx.train_steps(2, 16, 5, 20_000, 3, batch=256)
        # first a large call, then a smaller one: the second must not see
        # anything the first left in the shared array
        for m, seed in ((L.NOALLOC_MAX_SAMPLES, 9), (1000, 4)):
            want = ctx.eval_loss(2, 5, seed, m)
            got = ctx.eval_loss_noalloc(2, 5, seed, m)
            assert got == want, (m, got, want)
        # no device memory is taken by further calls
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info()
        for m, seed in ((L.NOALLOC_MAX_SAMPLES, 11), (77, 12), (L.NOALLOC_MAX_SAMPLES, 13)):
            ctx.eval_loss_noalloc(2, 5, seed, m)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info()
        assert free1 == free0, (free0, free1)
        # first order, BF16 tables
        ctx.init_embeddings(1, 32, L.DTYPE_BF16, seed=2)
        ctx.train_steps(1, 32, 5, 10_000, 5, batch=128)
        want = ctx.eval_loss(1, 5, 7, 4096)
        assert ctx.eval_loss_noalloc(1, 5, 7, 4096) == want
        # sizes outside the fixed array are refused before any work
        out = ctypes.c_double()
        for m in (0, L.NOALLOC_MAX_SAMPLES + 1):
            st = L.lib.line_eval_loss_noalloc(ctx.h, 2, 5, 1, m, ctypes.byref(out))
            assert st == L.LINE_ERR_ARG
            assert "fixed scratch" in ctx.last_error()
        # the context is still usable
        want = ctx.eval_loss(2, 5, 3, 2048)
        assert ctx.eval_loss_noalloc(2, 5, 3, 2048) == want
    finally:
        ctx.close()
