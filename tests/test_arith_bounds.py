"""Host checks of the bounds the kernels' lazy arithmetic relies on (no GPU).

* shoup_one (common.cuh) is shoup_approx with w = 1 bit for bit.

* shoup_approx (common.cuh): the quotient built from x1*s1 + hi(x1*s0) + hi(x0*s1 +
  lo(x1*s0)) is within 1 of floor(x*w'/2^64), so x*w - q_hat*p is in [0, 3p), for
  every 64-bit x.  The emulation below follows the 32-bit instruction sequence.
* The lazy forward NTT: with T in [0, 3p), X' = X + T and Y' = X + 4p - T grow by < 4p
  per stage; inputs below 8p and 17 stages stay below 2^64 for p < 2^57.
* The split basis conversion: reduced sources split at W = ceil(bits/2) bits; two
  accumulators of 2*32 products below 2^(2W+2) stay below 2^62 when W <= 27.
"""
import random

import pytest

M32, M64 = (1 << 32) - 1, (1 << 64) - 1


def shoup_approx(x, w, p):
    ws = (w << 64) // p
    x0, x1, s0, s1 = x & M32, x >> 32, ws & M32, ws >> 32
    T = x1 * s0
    U = x0 * s1 + (T & M32)
    assert U <= M64
    q_hat = x1 * s1 + (T >> 32) + (U >> 32)
    # low words on 32-bit halves: x*w + q_hat*(2^64 - p) mod 2^64
    w0, w1 = w & M32, w >> 32
    n = (1 << 64) - p
    n0, n1 = n & M32, n >> 32
    q0, q1 = q_hat & M32, (q_hat >> 32) & M32
    acc = (x0 * w0 + q0 * n0) & M64
    hi = ((acc >> 32) + x0 * w1 + x1 * w0 + q0 * n1 + q1 * n0) & M32
    r = (acc & M32) | (hi << 32)
    return q_hat, (x * ws) >> 64, r


def shoup_one(x, p):
    """shoup_one (common.cuh): shoup_approx with w = 1, the low word as
    x + q_hat*(2^64 - p) with x as the addend of the wide multiply-add."""
    ones = (1 << 64) // p
    x0, x1, s0, s1 = x & M32, x >> 32, ones & M32, ones >> 32
    T = x1 * s0
    U = x0 * s1 + (T & M32)
    q_hat = x1 * s1 + (T >> 32) + (U >> 32)
    n = (1 << 64) - p
    n0, n1 = n & M32, n >> 32
    q0, q1 = q_hat & M32, (q_hat >> 32) & M32
    acc = (q0 * n0 + x) & M64
    hi = ((acc >> 32) + q0 * n1 + q1 * n0) & M32
    return q_hat, (acc & M32) | (hi << 32)


@pytest.mark.parametrize("p", [18014398506729473, 1125899906826241, 144115188075593729, 65537, 7681])
def test_shoup_one_equals_shoup_approx_with_w_one(p):
    rng = random.Random(p + 1)
    for _ in range(20000):
        x = rng.choice([rng.randrange(0, 1 << 64), rng.randrange(0, min(80 * p, 1 << 64)), M64, 0, 3 * p - 1])
        q_hat, r = shoup_one(x, p)
        q_ref, _, r_ref = shoup_approx(x, 1, p)
        assert q_hat == q_ref and r == r_ref
        assert r == x - q_hat * p and 0 <= r < 3 * p


@pytest.mark.parametrize("p", [18014398506729473, 1125899906826241, 144115188075593729, 65537, 7681])
def test_shoup_approx_quotient_and_range(p):
    rng = random.Random(p)
    for _ in range(20000):
        w = rng.randrange(1, p)
        x = rng.choice([rng.randrange(0, 1 << 64), rng.randrange(0, min(80 * p, 1 << 64)), M64, 0, 8 * p - 1, p])
        assert 0 <= x <= M64
        q_hat, q, r = shoup_approx(x, w, p)
        assert q - 1 <= q_hat <= q
        assert r == x * w - q_hat * p
        assert 0 <= r < 3 * p


def test_lazy_forward_ntt_growth_bound():
    for logN in range(10, 18):
        p_max = (1 << 57) - 1
        bound = (8 + 4 * logN) * p_max
        assert bound < (1 << 64), logN


def test_split_conversion_accumulator_bound():
    for bits in range(20, 55):
        W = (bits + 1) // 2
        if W > 27:
            continue
        n_src = 32
        prod_max = ((1 << (W + 2)) - 1) * ((1 << W) - 1)  # yh < 2^(W+2) with y < 3q, constants < 2^W
        assert 2 * n_src * prod_max < (1 << 62)
