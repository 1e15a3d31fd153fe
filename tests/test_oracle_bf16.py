"""Pins of the oracle's BF16 storage mode (a target addition; the paper's
tables are FP32): the SplitMix64 output function and MurmurHash3's fmix32
(the two parts of the rounding bits) against published vectors, the
statistics of the bits, the stochastic-rounding rule, round-to-nearest for
initial tables, and the wiring of both into the minibatch oracle
(Algorithm 1 with the batch-summed deltas of Eq. 4).

Runs on the CPU (no GPU)."""
import os

import numpy as np
import pytest

import oracle as O
from paper_2604_09419_gb300 import inputs as I

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "splitmix64_seed1234567.txt")
GAMMA = 0x9E3779B97F4A7C15
M64 = (1 << 64) - 1


def f32_of_bits(b: int) -> float:
    return float(np.array([b], np.uint32).view(np.float32)[0])


def bits_of_f32(x: float) -> int:
    return int(np.array([x], np.float32).view(np.uint32)[0])


def test_splitmix64_published_vectors():
    want = [int(line.split()[1]) for line in open(GOLDEN) if line.strip() and not line.startswith("#")]
    x = 1234567
    got = []
    for _ in want:
        x = (x + GAMMA) & M64
        got.append(O.splitmix64_mix(x))
    assert got == want


MURMUR = os.path.join(os.path.dirname(__file__), "golden", "murmur3_x86_32.txt")


def murmur3_x86_32(data: bytes, seed: int) -> int:
    """MurmurHash3_x86_32 (Appleby): 4-byte blocks mixed into the state, the
    tail, the length, then the finaliser - here the oracle's fmix32."""
    M = 0xFFFFFFFF
    c1, c2 = 0xCC9E2D51, 0x1B873593

    def rotl(x, r):
        return ((x << r) | (x >> (32 - r))) & M

    h = seed
    n = len(data)
    for i in range(0, n - n % 4, 4):
        k = int.from_bytes(data[i:i + 4], "little")
        h ^= (rotl((k * c1) & M, 15) * c2) & M
        h = (rotl(h, 13) * 5 + 0xE6546B64) & M
    tail = data[n - n % 4:]
    if tail:
        k = int.from_bytes(tail, "little")
        h ^= (rotl((k * c1) & M, 15) * c2) & M
    return O.fmix32(h ^ n)


def test_fmix32_published_vectors():
    n = 0
    for line in open(MURMUR):
        if not line.strip() or line.startswith("#"):
            continue
        data_hex, seed_hex, want_hex = line.split()
        data = b"" if data_hex == "-" else bytes.fromhex(data_hex)
        seed, want = int(seed_hex, 16), int(want_hex, 16)
        if not data:
            assert O.fmix32(seed) == want, (seed_hex, want_hex)
        assert murmur3_x86_32(data, seed) == want, (data_hex, seed_hex, want_hex)
        n += 1
    assert n == 7


def test_sr_bits_uncorrelated_across_batches():
    # the property stochastic rounding relies on over training: for a fixed
    # row and column group, the bits of consecutive batches are uniform and
    # independent (lag-1 correlation and chi-square over 64 bins)
    for table, row, k4 in ((0, 0, 0), (1, 12345, 17), (0, 1 << 20, 31)):
        w = np.array([O.sr_bits(9, table, row, 4096 * b, k4) for b in range(6000)], np.uint64)
        for i in range(4):
            r = ((w >> np.uint64(16 * i)) & np.uint64(0xFFFF)).astype(np.float64)
            assert abs(np.corrcoef(r[:-1], r[1:])[0, 1]) < 0.06
            hist = np.bincount((r.astype(np.int64) >> 10), minlength=64)
            exp = r.size / 64
            assert ((hist - exp) ** 2 / exp).sum() < 110  # 63 degrees of freedom, p ~ 0.0002


def test_sr_bits_uniform_and_distinct():
    # distinct (table, row, batch, column group) give distinct words, and the
    # 16-bit slices are uniform (chi-square over 256 bins) and uncorrelated
    # between neighbouring column groups and rows
    words = set()
    vals = []
    for table in (0, 1):
        for row in range(64):
            for t0 in (0, 256, 1 << 33):
                for k4 in range(8):
                    w = O.sr_bits(77, table, row, t0, k4)
                    words.add(w)
                    vals.append(w)
    assert len(words) == len(vals)
    v = np.array(vals, np.uint64)
    r16 = np.concatenate([((v >> np.uint64(16 * i)) & np.uint64(0xFFFF)).astype(np.int64) for i in range(4)])
    hist = np.bincount(r16 >> 8, minlength=256)
    exp = r16.size / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    assert chi2 < 340  # 255 degrees of freedom, p ~ 0.0003
    a = np.array([O.sr_bits(5, 0, r, 0, 0) & 0xFFFF for r in range(4000)], np.float64)
    b = np.array([O.sr_bits(5, 0, r, 0, 1) & 0xFFFF for r in range(4000)], np.float64)
    c = np.array([O.sr_bits(5, 0, r + 1, 0, 0) & 0xFFFF for r in range(4000)], np.float64)
    assert abs(np.corrcoef(a, b)[0, 1]) < 0.06 and abs(np.corrcoef(a, c)[0, 1]) < 0.06
    # the seed and the batch start change the bits
    assert O.sr_bits(5, 0, 3, 0, 0) != O.sr_bits(6, 0, 3, 0, 0) != O.sr_bits(6, 0, 3, 256, 0)


def test_bf16_sr_hand_cases():
    one = bits_of_f32(1.0)
    # a BF16 value stays itself for every r
    for r in (0, 1, 0x7FFF, 0x8000, 0xFFFF):
        assert O.bf16_sr_bits(1.0, r) == one >> 16
        assert O.bf16_sr_bits(-2.5, r) == bits_of_f32(-2.5) >> 16
    # halfway between 1.0 and the next BF16 value (1 + 2^-7): up iff r >= 2^15
    half = f32_of_bits(one | 0x8000)
    assert O.bf16_sr_bits(half, 0x7FFF) == 0x3F80 and O.bf16_sr_bits(half, 0x8000) == 0x3F81
    # a quarter of the way: up iff r >= 3 * 2^14
    quarter = f32_of_bits(one | 0x4000)
    assert O.bf16_sr_bits(quarter, 0xBFFF) == 0x3F80 and O.bf16_sr_bits(quarter, 0xC000) == 0x3F81
    # negative values round in magnitude: away from zero when the bits carry
    nh = f32_of_bits(bits_of_f32(-1.0) | 0x8000)
    assert O.bf16_sr_bits(nh, 0x8000) == 0xBF81 and O.bf16_sr_bits(nh, 0x7FFF) == 0xBF80
    # carry into the exponent: just below 2.0 rounds up to 2.0
    below2 = f32_of_bits(bits_of_f32(2.0) - 1)
    assert O.bf16_sr_bits(below2, 1) == bits_of_f32(2.0) >> 16
    # overflow: the largest finite FP32 value can round up to infinity
    big = f32_of_bits(0x7F7FFFFF)
    assert O.bf16_sr_bits(big, 1) == 0x7F80 and O.bf16_sr_bits(big, 0) == 0x7F7F
    # infinities and NaN pass unchanged
    assert O.bf16_sr_bits(float("inf"), 0xFFFF) == 0x7F80
    assert O.bf16_sr_bits(float("-inf"), 0xFFFF) == 0xFF80
    nan = f32_of_bits(0x7FC00001)
    assert O.bf16_sr_bits(nan, 0xFFFF) == 0x7FC0
    # signed zero and a subnormal
    assert O.bf16_sr_bits(0.0, 0xFFFF) == 0 and O.bf16_sr_bits(-0.0, 0xFFFF) == 0x8000
    sub = f32_of_bits(0x00008000)
    assert O.bf16_sr_bits(sub, 0x7FFF) == 0 and O.bf16_sr_bits(sub, 0x8000) == 1


@pytest.mark.parametrize("x", [1.00390625 + 2 ** -10, -3.14159, 1e-3, -7.7e-6, 123456.7, 2.0 ** -130])
def test_bf16_sr_is_unbiased_exactly(x):
    # over all 2^16 equally likely bit patterns the mean of the rounded value
    # is the FP32 value exactly (the defining property of stochastic rounding)
    xf = float(np.float32(x))
    tot = 0.0
    for r in range(1 << 16):
        tot += O.bf16_value(O.bf16_sr_bits(xf, r))
    assert tot / 65536.0 == xf


def test_bf16_rn_against_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(3)
    xs = np.concatenate([rng.standard_normal(3000).astype(np.float32),
                         (rng.standard_normal(500) * 1e-39).astype(np.float32),
                         np.array([1.00390625, 1.01171875, -1.00390625, 3.4e38, 0.0, -0.0], np.float32)])
    want = torch.from_numpy(xs).to(torch.bfloat16).view(torch.int16).numpy().astype(np.uint16)
    got = np.array([O.bf16_rn_bits(float(v)) for v in xs], np.uint16)
    assert np.array_equal(got, want)
    # ties go to even: 1 + 2^-8 -> 1.0, 1 + 3 * 2^-8 -> 1 + 2^-6
    assert O.bf16_rn_bits(1.00390625) == 0x3F80 and O.bf16_rn_bits(1.01171875) == 0x3F82


@pytest.fixture(scope="module")
def tiny():
    g = I.tiny_chung_lu()
    return g, O.Tables(g)


def bf16_start(n, dim, seed):
    return O.round_bf16_rn(O.init_uniform(n, dim, seed))


def test_train_bf16_one_batch_is_the_fp64_batch_rounded(tiny):
    # one batch: every touched row is X_b + dX (the FP64 oracle's batch) in
    # FP32, then rounded with the bits of its (table, row, batch start, k/4)
    g, T = tiny
    dim, B, seed, t0 = 16, 256, 9, 512
    U0 = bf16_start(g.n_nodes, dim, 1)
    C0 = O.round_bf16_rn(U0[::-1].copy() * 0.5)
    for order in (1, 2):
        Uf, Cf = U0.copy(), (C0.copy() if order == 2 else None)
        O.train(T, Uf, Cf, order=order, K=5, n_samples=B, seed=seed, batch=B, sample_offset=t0, lr_total=4096,
                lam=1e-3)
        Ub, Cb = U0.copy(), (C0.copy() if order == 2 else None)
        O.train(T, Ub, Cb, order=order, K=5, n_samples=B, seed=seed, batch=B, sample_offset=t0, lr_total=4096,
                lam=1e-3, bf16=True)
        for table, (X0, Xf, Xb) in enumerate([(U0, Uf, Ub)] + ([(C0, Cf, Cb)] if order == 2 else [])):
            touched = np.nonzero(np.any(Xf != X0, axis=1))[0]
            assert touched.size > 50
            untouched = np.setdiff1d(np.arange(g.n_nodes), touched)
            assert np.array_equal(Xb[untouched], X0[untouched])
            for v in touched[:40]:
                for k in range(dim):
                    r = O.sr_bits(seed, table, int(v), t0, k // 4)
                    h = O.bf16_sr_bits(float(np.float32(Xf[v, k])), (r >> (16 * (k % 4))) & 0xFFFF)
                    assert Xb[v, k] == O.bf16_value(h), (order, table, v, k)


def test_train_bf16_invariants(tiny):
    g, T = tiny
    dim, B = 16, 256
    U0 = bf16_start(g.n_nodes, dim, 1)
    # lr 0: nothing changes (a BF16 value rounds to itself)
    U, C = U0.copy(), np.zeros_like(U0)
    O.train(T, U, C, order=2, K=5, n_samples=5000, seed=3, batch=B, lr0=0.0, bf16=True)
    assert np.array_equal(U, U0) and not C.any()
    # every stored value is a BF16 value
    U, C = U0.copy(), np.zeros_like(U0)
    O.train(T, U, C, order=2, K=5, n_samples=20_000, seed=3, batch=B, bf16=True)
    for X in (U, C):
        b = X.astype(np.float32).view(np.uint32)
        assert not np.any(b & 0xFFFF) and np.array_equal(X.astype(np.float32).astype(np.float64), X)
    # close to the FP64 run and unbiased against it
    Uf, Cf = U0.copy(), np.zeros_like(U0)
    O.train(T, Uf, Cf, order=2, K=5, n_samples=20_000, seed=3, batch=B)
    d = np.concatenate([(U - Uf).ravel(), (C - Cf).ravel()])
    scale = max(np.abs(Uf).max(), np.abs(Cf).max())
    assert np.abs(d).max() < 0.05 * scale
    nz = d[d != 0]
    assert abs(nz.mean()) < 5 * nz.std() / np.sqrt(nz.size)
