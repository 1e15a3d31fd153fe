"""FP64 serial CPU oracle for the LINE training step (arXiv 2604.09419).

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The library
(``paper_2604_09419_gb300``) never calls it and shares no code with it.

The arithmetic lives in ``line_oracle.c`` (plain loops, FP64, no FMA
contraction); this module compiles it with gcc on first use and wraps it with
ctypes.  Each function names the passage of the paper it follows:

* ``neg_weights`` - Eq. 1: q(v) ∝ d(v)^0.75, d = weighted out-degree;
* ``alias_build`` - the discrete distributions of Eq. 1 and Algorithm 3
  (edge pick ∝ weight) as alias tables over exact integer masses;
* ``sample`` - Algorithm 1: one positive arc and K negatives per sample;
* ``train`` - Algorithm 1 with Eq. 2-3 (LineUpdate) and the batch-summed
  deltas of Eq. 4;
* ``eval_loss`` - the negative-sampling objective whose gradients give the
  scalars g of Algorithm 1.

All functions are pinned by ``tests/test_oracle_*.py``: Philox known-answer
vectors, hand-derived alias tables, exact integer invariants, brute-force
enumeration, chi-square frequencies, finite differences of the loss and
closed-form small cases.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "line_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None

_u32p = np.ctypeslib.ndpointer(dtype=np.uint32, flags="C_CONTIGUOUS")
_u64p = np.ctypeslib.ndpointer(dtype=np.uint64, flags="C_CONTIGUOUS")
_i32p = np.ctypeslib.ndpointer(dtype=np.int32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(dtype=np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(dtype=np.float64, flags="C_CONTIGUOUS")
_i64 = ctypes.c_int64
_u64 = ctypes.c_uint64
_u32 = ctypes.c_uint32
_int = ctypes.c_int
_dbl = ctypes.c_double

TABLE_ARGS = [_i64, _i64, _i32p, _i32p, _u32p, _u32p, _u32p, _u32p]


def build(force: bool = False) -> str:
    """Compile ``line_oracle.c`` into ``_build/liboracle.so`` (gcc, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-std=c11", "-Wall", "-shared",
                               "-fPIC", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build()
            L = ctypes.CDLL(path)
            L.orc_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
            L.orc_philox4x32_10.restype = None
            L.orc_draw_words.argtypes = [_u64, _u32, _u32, _u64, _i64, _u32p]
            L.orc_draw_words.restype = None
            L.orc_neg_weights.argtypes = [_i64, _i64, _i32p, ctypes.c_void_p, _f64p]
            L.orc_neg_weights.restype = _int
            L.orc_fixed_sum.argtypes = [_i64, _f64p]
            L.orc_fixed_sum.restype = _dbl
            L.orc_alias_masses.argtypes = [_i64, _f64p, _u64p]
            L.orc_alias_masses.restype = _int
            L.orc_alias_pair.argtypes = [_i64, _u64p, _u32p, _u32p]
            L.orc_alias_pair.restype = _int
            L.orc_alias_build.argtypes = [_i64, _f64p, _u64p, _u32p, _u32p]
            L.orc_alias_build.restype = _int
            L.orc_alias_draw.argtypes = [_i64, _u32p, _u32p, _u32, _u32, _u32]
            L.orc_alias_draw.restype = _u32
            L.orc_sample.argtypes = TABLE_ARGS + [_u64, _u32, _u64, _i64, _int, _i32p]
            L.orc_sample.restype = _int
            L.orc_init_uniform.argtypes = [_i64, _int, _u64, _f64p]
            L.orc_init_uniform.restype = None
            L.orc_batch_lr.argtypes = [_dbl, _int, _dbl, _u64, _u64]
            L.orc_batch_lr.restype = _dbl
            L.orc_train.argtypes = TABLE_ARGS + [_int, _int, _int, _dbl, _int, _dbl, _u64, _u64, _u64,
                                                 _i64, _dbl, _dbl, _u64, _f64p, ctypes.c_void_p, ctypes.c_void_p,
                                                 _int, _int, _int]
            L.orc_train_bf16.argtypes = L.orc_train.argtypes
            L.orc_train_bf16.restype = _int
            L.orc_splitmix64_mix.argtypes = [_u64]
            L.orc_splitmix64_mix.restype = _u64
            L.orc_fmix32.argtypes = [_u32]
            L.orc_fmix32.restype = _u32
            L.orc_sr_bits.argtypes = [_u64, _u32, _u64, _u64, _u32]
            L.orc_sr_bits.restype = _u64
            L.orc_bf16_sr_bits.argtypes = [ctypes.c_float, _u32]
            L.orc_bf16_sr_bits.restype = ctypes.c_uint16
            L.orc_bf16_rn_bits.argtypes = [ctypes.c_float]
            L.orc_bf16_rn_bits.restype = ctypes.c_uint16
            L.orc_train_pairwise.argtypes = L.orc_train.argtypes
            L.orc_train_pairwise.restype = _int
            _f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
            L.orc_train_hogwild_mt.argtypes = TABLE_ARGS + [_int, _int, _int, _dbl, _int, _dbl, _u64, _u64, _u64,
                                                            _i64, _dbl, _dbl, _u64, _f32p, ctypes.c_void_p, _int]
            L.orc_train_hogwild_mt.restype = _int
            L.orc_walk_cumw.argtypes = [_i64, _i32p, ctypes.c_void_p, _f64p]
            L.orc_walk_cumw.restype = None
            L.orc_walk_pairs_per_walk.argtypes = [_int, _int]
            L.orc_walk_pairs_per_walk.restype = _i64
            L.orc_sample_walk.argtypes = TABLE_ARGS + [_f64p, _u64, _u64, _i64, _int, _int, _int, _int, _i32p]
            L.orc_sample_walk.restype = _int
            L.orc_train.restype = _int
            L.orc_eval_loss.argtypes = TABLE_ARGS + [_int, _int, _int, _u64, _i64, _f64p, ctypes.c_void_p]
            L.orc_eval_loss.restype = _dbl
            _lib = L
    return _lib


def philox(ctr, key) -> np.ndarray:
    """Philox4x32-10 of one 128-bit counter under one 64-bit key (SC'11)."""
    out = np.zeros(4, np.uint32)
    lib().orc_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def draw_words(seed: int, domain: int, call: int, t0: int, count: int) -> np.ndarray:
    """[count][4] Philox words of draws t0.. of one (domain, call)."""
    out = np.zeros((count, 4), np.uint32)
    lib().orc_draw_words(seed, domain, call, t0, count, out.reshape(-1))
    return out


def neg_weights(g) -> np.ndarray:
    """Eq. 1 numerator: x_v = d(v)^0.75, d(v) = sum of v's out-arc weights (FP64)."""
    x = np.zeros(g.n_nodes, np.float64)
    w = np.ascontiguousarray(g.w, np.float32)
    rc = lib().orc_neg_weights(g.n_nodes, g.n_arcs, np.ascontiguousarray(g.src, np.int32),
                               w.ctypes.data, x)
    if rc:
        raise ValueError(f"orc_neg_weights failed ({rc})")
    return x


def fixed_sum(x) -> float:
    x = np.ascontiguousarray(x, np.float64)
    return lib().orc_fixed_sum(x.size, x)


def alias_masses(x) -> np.ndarray:
    x = np.ascontiguousarray(x, np.float64)
    m = np.zeros(x.size, np.uint64)
    rc = lib().orc_alias_masses(x.size, x, m)
    if rc:
        raise ValueError(f"orc_alias_masses failed ({rc})")
    return m


def alias_pair(m):
    m = np.ascontiguousarray(m, np.uint64)
    thr = np.zeros(m.size, np.uint32)
    alias = np.zeros(m.size, np.uint32)
    rc = lib().orc_alias_pair(m.size, m, thr, alias)
    if rc:
        raise ValueError(f"orc_alias_pair failed ({rc})")
    return thr, alias


def alias_build(x):
    """Alias table of the distribution ∝ x: returns (masses, thr, alias)."""
    x = np.ascontiguousarray(x, np.float64)
    n = x.size
    m = np.zeros(n, np.uint64)
    thr = np.zeros(n, np.uint32)
    alias = np.zeros(n, np.uint32)
    rc = lib().orc_alias_build(n, x, m, thr, alias)
    if rc:
        raise ValueError(f"orc_alias_build failed ({rc})")
    return m, thr, alias


def alias_draw(thr, alias, w0: int, w1: int, w2: int) -> int:
    return int(lib().orc_alias_draw(thr.size, thr, alias, w0, w1, w2))


class Tables:
    """The graph plus both alias tables, as the oracle's functions take them."""

    def __init__(self, g):
        self.g = g
        self.n_nodes = g.n_nodes
        self.n_arcs = g.n_arcs
        self.src = np.ascontiguousarray(g.src, np.int32)
        self.dst = np.ascontiguousarray(g.dst, np.int32)
        self.edge_x = np.ascontiguousarray(g.w, np.float64)
        self.neg_x = neg_weights(g)
        self.m_e, self.thr_e, self.alias_e = alias_build(self.edge_x)
        self.m_n, self.thr_n, self.alias_n = alias_build(self.neg_x)

    def args(self):
        return (self.n_nodes, self.n_arcs, self.src, self.dst, self.thr_e, self.alias_e,
                self.thr_n, self.alias_n)


def sample(T: Tables, seed: int, t0: int, count: int, K: int, domain: int = 0) -> np.ndarray:
    """Records [count, K+2] = (u, v, n_1..n_K) for samples t0 .. t0+count-1."""
    out = np.zeros((count, K + 2), np.int32)
    lib().orc_sample(*T.args(), seed, domain, t0, count, K, out)
    return out


def init_uniform(n: int, dim: int, seed: int) -> np.ndarray:
    U = np.zeros((n, dim), np.float64)
    lib().orc_init_uniform(n, dim, seed, U)
    return U


def batch_lr(lr0, schedule, floor_frac, total, t0) -> float:
    return lib().orc_batch_lr(lr0, schedule, floor_frac, total, t0)


def walk_cumw(g) -> np.ndarray:
    """Cumulative arc weights per node, FP64 in arc order (the walk sampler's table)."""
    cw = np.zeros(g.n_arcs, np.float64)
    w = None if g.w is None else np.ascontiguousarray(g.w, np.float32)
    lib().orc_walk_cumw(g.n_arcs, np.ascontiguousarray(g.src, np.int32), None if w is None else w.ctypes.data, cw)
    return cw


def walk_pairs_per_walk(L: int, W: int) -> int:
    return lib().orc_walk_pairs_per_walk(L, W)


def sample_walk(T: Tables, cw: np.ndarray, seed: int, t0: int, count: int, K: int, L: int, W: int,
                reuse: int = 1) -> np.ndarray:
    """[count][K+2] records of the walk sampler (Algorithms 2-3, local walk);
    with reuse r each walk's pairs serve r passes in a row."""
    out = np.zeros((count, K + 2), np.int32)
    rc = lib().orc_sample_walk(*T.args(), cw, seed, t0, count, K, L, W, reuse, out.reshape(-1))
    if rc:
        raise ValueError(f"orc_sample_walk failed ({rc})")
    return out


def _walk_args(walk):
    if walk is None:
        return None, 0, 0, 1
    return (walk[0], walk[1], walk[2], walk[3] if len(walk) > 3 else 1)


def train(T: Tables, U: np.ndarray, C, *, order: int, K: int, lr0: float = 0.025, schedule: int = 1,
          lr_floor_frac: float = 1e-4, lr_total: int = 0, n_samples: int, seed: int, batch: int,
          lam: float = 0.0, alpha_neg: float = 1.0, sample_offset: int = 0, walk=None, bf16: bool = False):
    """Minibatch-synchronous LINE in place on FP64 tables U (and C for order 2).
    walk: None (arcs drawn by weight) or (cw, L, W) or (cw, L, W, reuse) for
    the walk sampler.  bf16: the tables hold BF16 values and every row
    written after a batch is rounded to FP32, then stochastically to BF16
    (``bf16_sr`` with the bits of ``sr_bits``)."""
    assert U.dtype == np.float64 and U.flags.c_contiguous
    dim = U.shape[1]
    cptr = None
    if order == 2:
        assert C is not None and C.dtype == np.float64 and C.flags.c_contiguous and C.shape == U.shape
        cptr = C.ctypes.data
    cw, L, W, R = _walk_args(walk)
    fn = lib().orc_train_bf16 if bf16 else lib().orc_train
    rc = fn(*T.args(), order, dim, K, lr0, schedule, lr_floor_frac, lr_total, n_samples,
            seed, batch, lam, alpha_neg, sample_offset, U, cptr,
            None if cw is None else cw.ctypes.data, L, W, R)
    if rc:
        raise ValueError(f"orc_train failed ({rc})")


def splitmix64_mix(z: int) -> int:
    """The SplitMix64 output function (Steele, Lea, Flood, OOPSLA 2014)."""
    return int(lib().orc_splitmix64_mix(z & 0xFFFFFFFFFFFFFFFF))


def fmix32(h: int) -> int:
    """MurmurHash3's 32-bit finaliser (Appleby)."""
    return int(lib().orc_fmix32(h & 0xFFFFFFFF))


def sr_bits(seed: int, table: int, row: int, t0: int, k4: int) -> int:
    """The 64 stochastic-rounding bits of values 4 k4 .. 4 k4 + 3 of `row`
    of table `table` (0 U, 1 C) written by the batch starting at sample t0:
    fmix32 of (lo32(s) + (2 row + table) 0x9E3779B1 + 2 k4 + j) for j = 0, 1
    (low, high word), with s the SplitMix64 output of seed ^ t0 0x9E3779B97F4A7C15."""
    return int(lib().orc_sr_bits(seed & 0xFFFFFFFFFFFFFFFF, table, row, t0, k4))


def bf16_sr_bits(x: float, r16: int) -> int:
    """BF16 bit pattern of the FP32 value x rounded stochastically with 16 bits r16."""
    return int(lib().orc_bf16_sr_bits(float(np.float32(x)), r16))


def bf16_rn_bits(x: float) -> int:
    """BF16 bit pattern of the FP32 value x rounded to nearest, ties to even."""
    return int(lib().orc_bf16_rn_bits(float(np.float32(x))))


def bf16_value(h: int) -> float:
    """The value of a BF16 bit pattern."""
    return float(np.array([h << 16], np.uint32).view(np.float32)[0])


def round_bf16_rn(x: np.ndarray) -> np.ndarray:
    """Values of an FP32-exact array rounded to BF16 (nearest even), as FP64."""
    f = np.ascontiguousarray(x, np.float32).ravel()
    out = np.empty(f.size, np.float64)
    fn = lib().orc_bf16_rn_bits
    for i, v in enumerate(f.tolist()):
        out[i] = bf16_value(int(fn(v)))
    return out.reshape(np.shape(x))


def train_pairwise(T: Tables, U: np.ndarray, C, *, order: int, K: int, lr0: float = 0.025, schedule: int = 1,
                   lr_floor_frac: float = 1e-4, lr_total: int = 0, n_samples: int, seed: int, batch: int,
                   lam: float = 0.0, alpha_neg: float = 1.0, sample_offset: int = 0, walk=None):
    """Per-pair immediate LINE updates (Algorithm 1's local path with
    LineUpdate) in place on FP64 tables; `batch` only sets the steps of the
    learning-rate schedule."""
    assert U.dtype == np.float64 and U.flags.c_contiguous
    dim = U.shape[1]
    cptr = None
    if order == 2:
        assert C is not None and C.dtype == np.float64 and C.flags.c_contiguous and C.shape == U.shape
        cptr = C.ctypes.data
    cw, L, W, R = _walk_args(walk)
    rc = lib().orc_train_pairwise(*T.args(), order, dim, K, lr0, schedule, lr_floor_frac, lr_total, n_samples,
                                  seed, batch, lam, alpha_neg, sample_offset, U, cptr,
                                  None if cw is None else cw.ctypes.data, L, W, R)
    if rc:
        raise ValueError(f"orc_train_pairwise failed ({rc})")


def train_hogwild_cpu(T: Tables, U: np.ndarray, C, *, order: int, K: int, lr0: float = 0.025, schedule: int = 1,
                      lr_floor_frac: float = 1e-4, lr_total: int = 0, n_samples: int, seed: int, batch: int,
                      lam: float = 0.0, alpha_neg: float = 1.0, sample_offset: int = 0, threads: int = 1):
    """Multi-threaded CPU Hogwild in FP32 (context for the benchmark, not a
    reference): the per-pair updates on FP32 tables U (and C), in place."""
    assert U.dtype == np.float32 and U.flags.c_contiguous
    cptr = None
    if order == 2:
        assert C is not None and C.dtype == np.float32 and C.flags.c_contiguous and C.shape == U.shape
        cptr = C.ctypes.data
    rc = lib().orc_train_hogwild_mt(*T.args(), order, U.shape[1], K, lr0, schedule, lr_floor_frac, lr_total,
                                    n_samples, seed, batch, lam, alpha_neg, sample_offset, U, cptr, threads)
    if rc:
        raise ValueError(f"orc_train_hogwild_mt failed ({rc})")


def eval_loss(T: Tables, U: np.ndarray, C, *, order: int, K: int, seed: int, m: int) -> float:
    U = np.ascontiguousarray(U, np.float64)
    cptr = None
    if order == 2:
        C = np.ascontiguousarray(C, np.float64)
        cptr = C.ctypes.data
    return lib().orc_eval_loss(*T.args(), order, U.shape[1], K, seed, m, U, cptr)
