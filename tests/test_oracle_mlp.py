"""Pins of the warm-start MLP oracle: BF16 rounding against a library
conversion, GELU against math.erf, gradients against finite differences,
Adam against its closed-form first steps, features on a hand-built graph,
the initialisation and minibatch draws against Philox words computed one by
one."""
import math

import numpy as np
import pytest

import oracle as O
from oracle import mlp as M


def test_bf16_rounding_matches_torch_and_hand_values():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=2000) * 10.0 ** rng.integers(-6, 6, 2000),
                        [1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -(1.0 + 2 ** -8 + 2 ** -20), 0.0, 65504.0]])
    x32 = x.astype(np.float32)
    want = torch.from_numpy(x32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(M.bf16(x32.astype(np.float64)), want)
    assert M.bf16(1.0 + 2 ** -8) == 1.0  # a tie goes to the even neighbour
    assert M.bf16(1.0 + 3 * 2 ** -9) == 1.0 + 2 ** -7
    assert M.bf16(-(1.0 + 2 ** -8 + 2 ** -20)) == -(1.0 + 2 ** -7)


def test_gelu_and_its_derivative():
    a = np.linspace(-6, 6, 97)
    want = np.array([0.5 * v * (1.0 + math.erf(v / math.sqrt(2.0))) for v in a])
    np.testing.assert_allclose(M.gelu(a), want, rtol=0, atol=1e-15)
    h = 1e-6
    fd = (M.gelu(a + h) - M.gelu(a - h)) / (2 * h)
    np.testing.assert_allclose(M.gelu_grad(a), fd, rtol=0, atol=1e-8)
    assert M.gelu(np.array([0.0]))[0] == 0.0 and M.gelu_grad(np.array([0.0]))[0] == 0.5


def tiny_params(rng, dim=4, hidden=6):
    P = M.in_width(dim)
    return {"W1": rng.normal(size=(hidden, P)) * 0.5, "b1": rng.normal(size=hidden) * 0.1,
            "W2": rng.normal(size=(dim, hidden)) * 0.5, "b2": rng.normal(size=dim) * 0.1}


def test_gradients_match_central_differences():
    rng = np.random.default_rng(1)
    p = tiny_params(rng)
    X = rng.normal(size=(5, M.in_width(4)))
    T = rng.normal(size=(5, 4))
    L, g = M.loss_and_grads(p, X, T)
    h = 1e-6
    for k in p:
        fd = np.zeros_like(p[k])
        for idx in np.ndindex(p[k].shape):
            old = p[k][idx]
            p[k][idx] = old + h
            Lp, _ = M.loss_and_grads(p, X, T)
            p[k][idx] = old - h
            Lm, _ = M.loss_and_grads(p, X, T)
            p[k][idx] = old
            fd[idx] = (Lp - Lm) / (2 * h)
        err = np.abs(fd - g[k]).max() / max(np.abs(g[k]).max(), 1e-12)
        assert err < 1e-6, (k, err)


def test_loss_closed_form_and_zero_network():
    rng = np.random.default_rng(2)
    p = tiny_params(rng)
    p["W1"][:] = 0.0
    p["b1"][:] = 0.0
    X = rng.normal(size=(3, M.in_width(4)))
    T = rng.normal(size=(3, 4))
    # h = GELU(0) = 0, so y = b2 and L = mean (b2 - t)^2
    L, g = M.loss_and_grads(p, X, T)
    assert L == pytest.approx(float(((p["b2"] - T) ** 2).mean()), rel=1e-15)
    assert not g["W2"].any()
    np.testing.assert_allclose(g["b2"], 2 * (p["b2"] - T).sum(axis=0) / 12, rtol=1e-14)


def test_adam_first_two_steps_closed_form():
    p = {"w": np.array([1.0, -2.0, 0.5])}
    g1 = np.array([0.1, -3.0, 0.0])
    st = {}
    M.adam_step(p, {"w": g1}, st, lr=0.01)
    # step 1: mhat = g, vhat = g^2
    want = np.array([1.0, -2.0, 0.5]) - 0.01 * g1 / (np.abs(g1) + 1e-8)
    np.testing.assert_allclose(p["w"], want, rtol=0, atol=1e-15)
    g2 = np.array([0.3, 1.0, 2.0])
    M.adam_step(p, {"w": g2}, st, lr=0.01)
    m = 0.9 * 0.1 * g1 + 0.1 * g2
    v = 0.999 * 0.001 * g1 * g1 + 0.001 * g2 * g2
    mhat = m / (1 - 0.81)
    vhat = v / (1 - 0.999 ** 2)
    np.testing.assert_allclose(p["w"], want - 0.01 * mhat / (np.sqrt(vhat) + 1e-8), rtol=0, atol=1e-14)


def test_features_hand_graph():
    # arcs: 0->1 (w 2), 0->2 (w 3), 0->3 (w 1), 1->0 (w 2), 4 isolated
    src = np.array([0, 0, 0, 1])
    dst = np.array([1, 2, 3, 0])
    w = np.array([2.0, 3.0, 1.0, 2.0])
    U = np.arange(5 * 2, dtype=np.float64).reshape(5, 2)  # dim 2 -> width 16
    known = np.array([1, 1, 1, 0, 1], bool)  # node 3 is unknown
    X = M.features(5, src, dst, w, U, known)
    assert X.shape == (5, 16)
    assert X[0, 0] == pytest.approx(math.log(7.0)) and X[1, 0] == pytest.approx(math.log(3.0))
    np.testing.assert_allclose(X[0, 1:3], (U[1] + U[2]) / 2)  # node 3 excluded
    np.testing.assert_allclose(X[1, 1:3], U[0])
    assert not X[4].any() and not X[2].any() and not X[:, 3:].any()


def test_init_params_match_philox_words_one_by_one():
    dim, hidden, seed = 4, 6, 77
    p = M.init_params(dim, hidden, seed)
    P = M.in_width(dim)
    n1 = hidden * P

    def u(idx):
        w0 = int(O.philox([idx & 0xFFFFFFFF, idx >> 32, 1, 7], [seed & 0xFFFFFFFF, seed >> 32])[0])
        return ((w0 >> 8) - (1 << 23)) / float(1 << 23)

    s1 = float(np.float32(1 / math.sqrt(dim + 1)))
    s2 = float(np.float32(1 / math.sqrt(hidden)))
    for j, i in [(0, 0), (3, 4), (5, 2)]:
        assert p["W1"][j, i] == float(np.float32(u(j * P + i) * s1))
    assert not p["W1"][:, dim + 1:].any() and not p["b1"].any() and not p["b2"].any()
    for j, i in [(0, 0), (3, 5)]:
        assert p["W2"][j, i] == float(np.float32(u(n1 + hidden + j * hidden + i) * s2))
    assert np.abs(p["W1"]).max() <= s1 and np.abs(p["W2"]).max() <= s2


def test_batch_nodes_match_philox_words_one_by_one():
    nodes = np.array([5, 9, 11, 40, 41, 77, 1000], np.int32)
    seed, step, B = 3, 12, 9
    got = M.batch_nodes(nodes, step, B, seed)
    for j in range(B):
        t = step * B + j
        w = O.philox([t & 0xFFFFFFFF, t >> 32, 0, 7], [seed, 0])
        r = int(w[1]) << 32 | int(w[0])
        assert got[j] == nodes[(r * len(nodes)) >> 64]


def test_training_learns_a_smooth_map():
    """A sanity check of the whole loop: the MLP fits targets that are a
    smooth function of the inputs."""
    rng = np.random.default_rng(4)
    dim, hidden = 8, 32
    P = M.in_width(dim)
    n = 512
    X = np.zeros((n, P))
    X[:, :dim + 1] = rng.normal(size=(n, dim + 1))
    T = np.tanh(X[:, 1:dim + 1] @ rng.normal(size=(dim, dim)) * 0.5)
    p = M.init_params(dim, hidden, 5)
    losses = M.train(p, X, T, np.arange(n), steps=300, batch=64, seed=6, lr=3e-3)
    assert np.mean(losses[-20:]) < 0.3 * np.mean(losses[:5])
