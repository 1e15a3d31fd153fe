"""FP64 oracle of the MLP warm start for new or held-out nodes.

TEST INFRASTRUCTURE: only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this module.

The paper trains LINE embeddings for a fixed graph (Algorithm 1); nodes that
arrive later, or whose rows were never trained, start from random rows.  The
warm start regresses a node's trained U row on two inputs every node has: its
log weighted degree and the mean trained U row of its neighbours, and
initialises the rows of new nodes with the prediction.  Definitions, for
embedding dimension d, hidden width H and P = the input width rounded up to a
multiple of 16 (d + 1 = 129 -> 144):

* features:  x[0] = log(1 + d_w(v)), d_w = weighted out-degree;
  x[1 .. d] = mean of U[w] over arcs v -> w with w known (0 if none);
  x[d+1 .. P) = 0;
* network:   a = W1 x + b1 (W1: H x P), h = GELU(a) = a/2 (1 + erf(a/sqrt 2)),
  y = W2 h + b2 (W2: d x H);
* loss of a minibatch of B nodes with targets t = U[v]:
  L = sum (y - t)^2 / (B d);
* gradients: backpropagation of L (written out below, pinned by finite
  differences);
* optimiser: Adam (Kingma and Ba, ICLR 2015, Algorithm 1) with bias
  correction, beta1 = 0.9, beta2 = 0.999, eps = 1e-8;
* initialisation: b1 = b2 = 0; W1[j][i] = s1 * u, s1 = fl32(1/sqrt(d+1)), for
  i <= d (0 for the padding columns); W2[j][i] = s2 * u, s2 = fl32(1/sqrt(H));
  u = ((w0 >> 8) - 2^23) 2^-23 where w0 is word 0 of the Philox draw of
  domain 7, call 1, counter index = the parameter's flat index in
  [W1, b1, W2, b2];
* minibatches: sample j of (global) step s is node nodes[mulhi64(w1:w0, n)],
  words of the Philox draw of domain 7, call 0, counter index s B + j.

``act_bf16`` rounds the activations x and h to BF16 (nearest, ties to even)
where the library stores them in BF16; everything else is FP64 here.
"""
from __future__ import annotations

import math

import numpy as np

DOMAIN = 7
BETA1, BETA2, EPS = 0.9, 0.999, 1e-8


def in_width(dim: int) -> int:
    return (dim + 1 + 15) // 16 * 16


def bf16(x) -> np.ndarray:
    """Round to BF16 (8 significant bits, nearest, ties to even), as FP64."""
    x = np.asarray(x, np.float64)
    m, e = np.frexp(x)
    return np.ldexp(np.round(m * 256.0) / 256.0, e)


def gelu(a):
    from scipy.special import erf
    return 0.5 * a * (1.0 + erf(a / math.sqrt(2.0)))


def gelu_grad(a):
    from scipy.special import erf
    return 0.5 * (1.0 + erf(a / math.sqrt(2.0))) + a * np.exp(-0.5 * a * a) / math.sqrt(2.0 * math.pi)


def features(n_nodes, src, dst, w, U, known, act_bf16=False) -> np.ndarray:
    """[n_nodes][P] inputs of every node (FP64; BF16-rounded if act_bf16)."""
    U = np.asarray(U, np.float64)
    dim = U.shape[1]
    X = np.zeros((n_nodes, in_width(dim)), np.float64)
    src = np.asarray(src, np.int64)
    dst = np.asarray(dst, np.int64)
    w = np.ones(len(src)) if w is None else np.asarray(w, np.float64)
    deg = np.zeros(n_nodes)
    np.add.at(deg, src, w)
    X[:, 0] = np.log1p(deg)
    ok = np.asarray(known, bool)[dst]
    acc = np.zeros((n_nodes, dim))
    cnt = np.zeros(n_nodes)
    np.add.at(acc, src[ok], U[dst[ok]])
    np.add.at(cnt, src[ok], 1.0)
    has = cnt > 0
    X[has, 1:dim + 1] = acc[has] / cnt[has, None]
    return bf16(X) if act_bf16 else X


def init_params(dim: int, hidden: int, seed: int) -> dict:
    """The initial parameters (FP32 values, held in FP64)."""
    from oracle import draw_words
    P = in_width(dim)
    n1, n2 = hidden * P, dim * hidden
    words = draw_words(seed, DOMAIN, 1, 0, n1 + hidden + n2 + dim)[:, 0].astype(np.int64)
    u = ((words >> 8) - (1 << 23)).astype(np.float64) * 2.0 ** -23
    s1 = float(np.float32(1.0 / math.sqrt(dim + 1)))
    s2 = float(np.float32(1.0 / math.sqrt(hidden)))
    # one FP32 rounding of the exact product, as the library computes it
    W1 = (u[:n1] * s1).astype(np.float32).astype(np.float64).reshape(hidden, P)
    W1[:, dim + 1:] = 0.0
    W2 = (u[n1 + hidden:n1 + hidden + n2] * s2).astype(np.float32).astype(np.float64).reshape(dim, hidden)
    return {"W1": W1, "b1": np.zeros(hidden), "W2": W2, "b2": np.zeros(dim)}


def batch_nodes(nodes, step: int, batch: int, seed: int) -> np.ndarray:
    """The minibatch of global step `step`: nodes[mulhi64(w1:w0, n)]."""
    from oracle import draw_words
    nodes = np.asarray(nodes)
    n = len(nodes)
    wd = draw_words(seed, DOMAIN, 0, step * batch, batch)
    idx = [((int(a[1]) << 32 | int(a[0])) * n) >> 64 for a in wd]
    return nodes[np.array(idx, np.int64)]


def forward(p: dict, X, act_bf16=False):
    """(a, h, y) for the rows of X."""
    a = X @ p["W1"].T + p["b1"]
    h = gelu(a)
    if act_bf16:
        h = bf16(h)
    y = h @ p["W2"].T + p["b2"]
    return a, h, y


def loss_and_grads(p: dict, X, T, act_bf16=False):
    """Minibatch loss L = sum (y - t)^2 / (B d) and its gradients."""
    B, dim = T.shape
    a, h, y = forward(p, X, act_bf16)
    r = y - T
    L = float((r * r).sum()) / (B * dim)
    dy = 2.0 * r / (B * dim)
    g = {"W2": dy.T @ h, "b2": dy.sum(axis=0)}
    da = (dy @ p["W2"]) * gelu_grad(a)
    g["W1"] = da.T @ X
    g["b1"] = da.sum(axis=0)
    return L, g


def adam_step(p: dict, g: dict, state: dict, lr: float) -> None:
    """One Adam update in place; state holds m, v per parameter and the step t."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m_" + k, np.zeros_like(p[k]))
        v = state.setdefault("v_" + k, np.zeros_like(p[k]))
        m *= BETA1
        m += (1.0 - BETA1) * g[k]
        v *= BETA2
        v += (1.0 - BETA2) * g[k] * g[k]
        mhat = m / (1.0 - BETA1 ** t)
        vhat = v / (1.0 - BETA2 ** t)
        p[k] -= lr * mhat / (np.sqrt(vhat) + EPS)


def train(p: dict, X_all, T_all, nodes, steps: int, batch: int, seed: int, lr: float = 1e-3,
          act_bf16=False, step_offset: int = 0, state: dict | None = None) -> list:
    """`steps` Adam steps on minibatches of `nodes`; returns the loss of each
    step (before its update)."""
    state = {} if state is None else state
    losses = []
    for s in range(step_offset, step_offset + steps):
        b = batch_nodes(nodes, s, batch, seed)
        L, g = loss_and_grads(p, X_all[b], T_all[b], act_bf16)
        losses.append(L)
        adam_step(p, g, state, lr)
    return losses


def predict(p: dict, X, act_bf16=False) -> np.ndarray:
    return forward(p, X, act_bf16)[2]
