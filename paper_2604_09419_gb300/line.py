"""Python binding of the LINE C ABI (``include/line.h``).

Argument marshalling only: every function here forwards to the entry point of
the same name in ``_build/libline.so``.  Buffers may be CUDA tensors (device
pointers) or NumPy arrays / CPU tensors (host pointers); the library copies
with unified addressing.  There is no fallback: if the shared library is
missing or cannot be loaded, importing this module raises.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libline.so")

NOALLOC_MAX_SAMPLES = 1 << 20
LINE_OK, LINE_ERR_ARG, LINE_ERR_OOM, LINE_ERR_CUDA, LINE_ERR_TIMEOUT, LINE_ERR_STATE, LINE_ERR_VALIDATE = (
    0, -1, -2, -3, -4, -5, -6)
DTYPE_F32, DTYPE_BF16 = 0, 1
TABLE_EDGE, TABLE_NEG = 0, 1
WHICH_U, WHICH_C = 0, 1
MODE_BATCHED, MODE_PERSISTENT, MODE_HOGWILD = 0, 1, 2
SCORE_DOT, SCORE_COSINE = 0, 1


class GraphDesc(ctypes.Structure):
    _fields_ = [("n_nodes", ctypes.c_int64), ("n_arcs", ctypes.c_int64), ("src", ctypes.c_void_p),
                ("dst", ctypes.c_void_p), ("w", ctypes.c_void_p)]


class LR(ctypes.Structure):
    _fields_ = [("lr0", ctypes.c_double), ("schedule", ctypes.c_int), ("floor_frac", ctypes.c_double),
                ("total", ctypes.c_uint64)]


class TrainOpts(ctypes.Structure):
    _fields_ = [("batch", ctypes.c_int64), ("lambda_", ctypes.c_double), ("alpha_neg", ctypes.c_double),
                ("sample_offset", ctypes.c_uint64), ("mode", ctypes.c_int), ("spin_limit", ctypes.c_int64),
                ("chunk_batches", ctypes.c_int), ("warps_per_block", ctypes.c_int), ("timing", ctypes.c_int),
                ("graph", ctypes.c_int), ("walk_length", ctypes.c_int), ("window", ctypes.c_int),
                ("hogwild_workers", ctypes.c_int), ("walk_reuse", ctypes.c_int)]


class TuneOpts(ctypes.Structure):
    _fields_ = [("batches", ctypes.c_void_p), ("n_batches", ctypes.c_int), ("trial_samples", ctypes.c_uint64),
                ("try_persistent", ctypes.c_int), ("both_orders", ctypes.c_int)]


class Stats(ctypes.Structure):
    _fields_ = [("update_launches", ctypes.c_int64), ("update_ms", ctypes.c_double),
                ("update_samples", ctypes.c_uint64), ("prepass_launches", ctypes.c_int64),
                ("prepass_ms", ctypes.c_double), ("total_ms", ctypes.c_double), ("total_samples", ctypes.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError(f"libline.so not built ({LIB_PATH}); run __graft_entry__.build()")
    L = ctypes.CDLL(LIB_PATH)
    vp, i64, u64, u32, i32, dbl = (ctypes.c_void_p, ctypes.c_int64, ctypes.c_uint64, ctypes.c_uint32,
                                   ctypes.c_int, ctypes.c_double)
    sigs = {
        "line_train_opts_default": (None, [ctypes.POINTER(TrainOpts)]),
        "line_status_string": (ctypes.c_char_p, [i32]),
        "line_create": (i32, [ctypes.POINTER(vp), i32, vp]),
        "line_destroy": (None, [vp]),
        "line_last_error": (ctypes.c_char_p, [vp]),
        "line_build_alias": (i32, [vp, ctypes.POINTER(GraphDesc)]),
        "line_get_graph_info": (i32, [vp, ctypes.POINTER(i64), ctypes.POINTER(i64)]),
        "line_get_alias": (i32, [vp, i32, vp, vp]),
        "line_sample_debug": (i32, [vp, i32, u64, u32, u64, i64, vp]),
        "line_sample_walk_debug": (i32, [vp, i32, u64, i32, i32, i32, u64, i64, vp]),
        "line_init_embeddings": (i32, [vp, i32, i32, i32, u64]),
        "line_train_steps": (i32, [vp, i32, i32, i32, ctypes.POINTER(LR), u64, u64, ctypes.POINTER(TrainOpts)]),
        "line_train_orders": (i32, [vp, i32, i32, ctypes.POINTER(LR), u64, u64, ctypes.POINTER(TrainOpts)]),
        "line_get_embeddings": (i32, [vp, i32, i32, vp, i32]),
        "line_set_embeddings": (i32, [vp, i32, i32, vp, i32, vp, i64]),
        "line_eval_loss": (i32, [vp, i32, i32, u64, i64, ctypes.POINTER(dbl)]),
        "line_eval_loss_noalloc": (i32, [vp, i32, i32, u64, i64, ctypes.POINTER(dbl)]),
        "line_eval_auc": (i32, [vp, i32, i32, vp, vp, i64, vp, vp, i64, vp, vp, ctypes.POINTER(dbl)]),
        "line_mlp_create": (i32, [vp, i32, i32, i32, u64]),
        "line_mlp_features": (i32, [vp, vp]),
        "line_mlp_features_rows": (i32, [vp, vp, vp, i64]),
        "line_mlp_get_features": (i32, [vp, vp]),
        "line_mlp_get_params": (i32, [vp, vp, ctypes.POINTER(i64)]),
        "line_mlp_set_params": (i32, [vp, vp]),
        "line_mlp_grad": (i32, [vp, vp, i64, vp, ctypes.POINTER(dbl)]),
        "line_mlp_train": (i32, [vp, vp, i64, i64, i64, dbl, u64, u64, vp]),
        "line_mlp_predict": (i32, [vp, vp, i64, vp]),
        "line_autotune": (i32, [vp, i32, i32, i32, ctypes.POINTER(LR), ctypes.POINTER(TuneOpts),
                                ctypes.POINTER(TrainOpts), ctypes.POINTER(dbl)]),
        "line_get_stats": (i32, [vp, ctypes.POINTER(Stats)]),
        "line_reset_stats": (i32, [vp]),
        "line_synchronize": (i32, [vp]),
        "line_debug_wait_timeout": (i32, [vp, i64]),
    }
    for name, (res, args) in sigs.items():
        f = getattr(L, name)
        f.restype = res
        f.argtypes = args
    return L


lib = _load()
EXPORTED = ("line_train_opts_default", "line_status_string", "line_create", "line_destroy", "line_last_error",
            "line_build_alias", "line_get_graph_info", "line_get_alias", "line_sample_debug", "line_sample_walk_debug",
            "line_init_embeddings", "line_train_steps", "line_train_orders", "line_get_embeddings", "line_set_embeddings",
            "line_eval_loss", "line_eval_loss_noalloc", "line_eval_auc", "line_mlp_create", "line_mlp_features", "line_mlp_features_rows",
            "line_mlp_get_features", "line_mlp_get_params", "line_mlp_set_params", "line_mlp_grad", "line_mlp_train",
            "line_mlp_predict", "line_autotune", "line_get_stats", "line_reset_stats", "line_synchronize", "line_debug_wait_timeout")


class LineError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{lib.line_status_string(status).decode()} ({status}): {msg}")
        self.status = status


def ptr(x) -> int | None:
    """Address of a CUDA tensor, CPU tensor or NumPy array (None for None)."""
    if x is None:
        return None
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    if hasattr(x, "data_ptr"):
        assert x.is_contiguous()
        return x.data_ptr()
    raise TypeError(type(x))


def train_opts_default() -> TrainOpts:
    o = TrainOpts()
    lib.line_train_opts_default(ctypes.byref(o))
    return o


class Context:
    """Owns one ``line_ctx``; methods mirror the C entry points."""

    def __init__(self, device: int = 0, stream: int | None = None):
        h = ctypes.c_void_p()
        st = lib.line_create(ctypes.byref(h), device, stream)
        if st != LINE_OK:
            raise LineError(st, "line_create failed")
        self.h = h

    def close(self):
        if self.h:
            lib.line_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def _ck(self, st):
        if st != LINE_OK:
            raise LineError(st, lib.line_last_error(self.h).decode())
        return st

    def last_error(self) -> str:
        return lib.line_last_error(self.h).decode()

    def build_alias(self, n_nodes, src, dst, w=None):
        g = GraphDesc(n_nodes, int(src.shape[0]), ptr(src), ptr(dst), ptr(w))
        return self._ck(lib.line_build_alias(self.h, ctypes.byref(g)))

    def graph_info(self):
        n, m = ctypes.c_int64(), ctypes.c_int64()
        self._ck(lib.line_get_graph_info(self.h, ctypes.byref(n), ctypes.byref(m)))
        return n.value, m.value

    def get_alias(self, table, thr, alias):
        return self._ck(lib.line_get_alias(self.h, table, ptr(thr), ptr(alias)))

    def sample_debug(self, K, seed, domain, t0, count, out):
        return self._ck(lib.line_sample_debug(self.h, K, seed, domain, t0, count, ptr(out)))

    def sample_walk_debug(self, K, seed, walk_length, window, t0, count, out, reuse=1):
        return self._ck(lib.line_sample_walk_debug(self.h, K, seed, walk_length, window, reuse, t0, count, ptr(out)))

    def init_embeddings(self, order, dim, dtype=DTYPE_F32, seed=0):
        return self._ck(lib.line_init_embeddings(self.h, order, dim, dtype, seed))

    def train_steps(self, order, dim, K, n_samples, seed, *, lr0=0.025, schedule=1, floor_frac=1e-4, total=0,
                    opts: TrainOpts | None = None, check=True, **kw):
        lr = LR(lr0, schedule, floor_frac, total)
        o = opts if opts is not None else train_opts_default()
        for k, v in kw.items():
            setattr(o, "lambda_" if k == "lam" else k, v)
        st = lib.line_train_steps(self.h, order, dim, K, ctypes.byref(lr), n_samples, seed, ctypes.byref(o))
        return self._ck(st) if check else st

    def train_orders(self, dim, K, n_samples, seed, *, lr0=0.025, schedule=1, floor_frac=1e-4, total=0,
                     opts: TrainOpts | None = None, **kw):
        """Both orders' tables on the same samples, concurrently (same bits as two train_steps calls)."""
        lr = LR(lr0, schedule, floor_frac, total)
        o = opts if opts is not None else train_opts_default()
        for k, v in kw.items():
            setattr(o, "lambda_" if k == "lam" else k, v)
        return self._ck(lib.line_train_orders(self.h, dim, K, ctypes.byref(lr), n_samples, seed, ctypes.byref(o)))

    def get_embeddings(self, order, which, dst, dtype=DTYPE_F32):
        return self._ck(lib.line_get_embeddings(self.h, order, which, ptr(dst), dtype))

    def set_embeddings(self, order, which, src, dtype=DTYPE_F32, rows=None):
        n = int(src.shape[0]) if rows is None else int(rows.shape[0])
        return self._ck(lib.line_set_embeddings(self.h, order, which, ptr(src), dtype, ptr(rows), n))

    def eval_loss(self, order, K, seed, m) -> float:
        out = ctypes.c_double()
        self._ck(lib.line_eval_loss(self.h, order, K, seed, m, ctypes.byref(out)))
        return out.value

    def eval_loss_noalloc(self, order, K, seed, m) -> float:
        """line_eval_loss with no device allocation (scratch in a fixed array)."""
        out = ctypes.c_double()
        self._ck(lib.line_eval_loss_noalloc(self.h, order, K, seed, m, ctypes.byref(out)))
        return out.value

    def eval_auc(self, orders, pos_src, pos_dst, neg_src, neg_dst, scores=None, score=SCORE_DOT):
        """Link-prediction AUC; returns (auc, (#(neg < pos), #(neg == pos)))."""
        out = ctypes.c_double()
        counts = np.zeros(2, np.uint64)
        self._ck(lib.line_eval_auc(self.h, orders, score, ptr(pos_src), ptr(pos_dst), int(pos_src.shape[0]), ptr(neg_src),
                                   ptr(neg_dst), int(neg_src.shape[0]), ptr(scores), counts.ctypes.data,
                                   ctypes.byref(out)))
        return out.value, (int(counts[0]), int(counts[1]))

    def autotune(self, order, dim, K, *, batches=None, trial_samples=0, try_persistent=False, both_orders=False,
                 lr0=0.025, schedule=1, floor_frac=1e-4, total=0, opts: TrainOpts | None = None):
        """Fastest launch configuration on scratch copies of the tables;
        returns (TrainOpts, samples/s)."""
        lr = LR(lr0, schedule, floor_frac, total)
        o = opts if opts is not None else train_opts_default()
        arr = None if not batches else np.asarray(batches, np.int64)
        t = TuneOpts(None if arr is None else arr.ctypes.data, 0 if arr is None else len(arr), trial_samples,
                     1 if try_persistent else 0, 1 if both_orders else 0)
        rate = ctypes.c_double()
        self._ck(lib.line_autotune(self.h, order, dim, K, ctypes.byref(lr), ctypes.byref(t), ctypes.byref(o),
                                   ctypes.byref(rate)))
        return o, rate.value

    # ---- warm-start MLP
    def mlp_create(self, order, hidden=256, act_dtype=DTYPE_BF16, seed=0):
        return self._ck(lib.line_mlp_create(self.h, order, hidden, act_dtype, seed))

    def mlp_features(self, known):
        return self._ck(lib.line_mlp_features(self.h, ptr(known)))

    def mlp_features_rows(self, known, rows):
        return self._ck(lib.line_mlp_features_rows(self.h, ptr(known), ptr(rows), int(rows.shape[0])))

    def mlp_get_features(self, out):
        return self._ck(lib.line_mlp_get_features(self.h, ptr(out)))

    def mlp_n_params(self) -> int:
        n = ctypes.c_int64()
        self._ck(lib.line_mlp_get_params(self.h, None, ctypes.byref(n)))
        return n.value

    def mlp_get_params(self) -> np.ndarray:
        out = np.empty(self.mlp_n_params(), np.float32)
        self._ck(lib.line_mlp_get_params(self.h, out.ctypes.data, None))
        return out

    def mlp_set_params(self, params):
        return self._ck(lib.line_mlp_set_params(self.h, ptr(params)))

    def mlp_grad(self, rows, grads_out=None) -> float:
        loss = ctypes.c_double()
        self._ck(lib.line_mlp_grad(self.h, ptr(rows), int(rows.shape[0]), ptr(grads_out), ctypes.byref(loss)))
        return loss.value

    def mlp_train(self, nodes, steps, batch, lr=1e-3, seed=0, step_offset=0, losses=True):
        out = np.empty(steps, np.float64) if losses else None
        self._ck(lib.line_mlp_train(self.h, ptr(nodes), int(nodes.shape[0]), steps, batch, lr, seed, step_offset,
                                    None if out is None else out.ctypes.data))
        return out

    def mlp_predict(self, rows, y_out=None):
        return self._ck(lib.line_mlp_predict(self.h, ptr(rows), int(rows.shape[0]), ptr(y_out)))

    def stats(self) -> Stats:
        s = Stats()
        self._ck(lib.line_get_stats(self.h, ctypes.byref(s)))
        return s

    def reset_stats(self):
        return self._ck(lib.line_reset_stats(self.h))

    def synchronize(self):
        return self._ck(lib.line_synchronize(self.h))

    def debug_wait_timeout(self, spin_limit) -> int:
        return lib.line_debug_wait_timeout(self.h, spin_limit)


def table_numpy(ctx: Context, n_nodes: int, dim: int, order: int, which: int) -> np.ndarray:
    """Copy a table into a new host FP32 array (through the C ABI)."""
    out = np.empty((n_nodes, dim), np.float32)
    ctx.get_embeddings(order, which, out, DTYPE_F32)
    return out
