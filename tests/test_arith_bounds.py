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


# ---------------------------------------------------------------- tensor-core basis conversion
def _f16_bits(v):
    """The host encoder of byte values in bconv_tc_kernel's operand images (exact below 2048)."""
    if v == 0:
        return 0
    e = v.bit_length() - 1
    mant = v << (10 - e) if e <= 10 else v >> (e - 10)
    return ((e + 15) << 10) | (mant & 0x3FF)


def test_tc_operand_encodings_are_exact():
    np = pytest.importorskip("numpy")
    for v in list(range(256)) + [2048, 4096]:
        assert np.array([v], dtype=np.float16).view(np.uint16)[0] == _f16_bits(v)
    # device side: (0x6400 | b) is the f16 1024 + b; subtracting 1024 leaves b exactly
    for b in range(256):
        h = np.array([0x6400 | b], dtype=np.uint16).view(np.float16)[0]
        assert float(h) == 1024 + b and float(np.float16(h - np.float16(1024))) == b
    assert 2048.0 * 4096.0 == 2.0 ** 23


def shoup_u32(x, w, p):
    """shoup_u32 (common.cuh): x < 2^32, exact quotient hi(x*s1 + hi(x*s0)), result in [0, 2p)."""
    ws = (w << 64) // p
    s0, s1 = ws & M32, ws >> 32
    T = x * s0
    U = x * s1 + (T >> 32)
    assert U <= M64
    q = U >> 32
    assert q == (x * ws) >> 64
    n = (1 << 64) - p
    acc = (x * (w & M32) + q * (n & M32)) & M64
    m = (x * (w >> 32) + q * (n >> 32)) & M32
    r = (acc + (m << 32)) & M64
    assert r == x * w - q * p and r < 2 * p
    return r


def _tc_lazy(nsrc, tmin):
    """The host's tc_lazy: the epilogue's low word stays below 5t for the smallest prime."""
    lo_max = nsrc * 7 * 255 * 255 * (1 + (1 << 8) + (1 << 16) + (1 << 24) + (1 << 32))
    return lo_max < 5 * tmin


def _tc_convert(ys, Cs, t, sub, lazy):
    """bconv_tc_kernel for one coefficient and one target t: byte products summed
    as the tensor core does (integers, every partial sum exact in f32), the f32
    bits read as integers, the epilogue's 64- and 32-bit arithmetic."""
    import struct

    S = [0] * 8
    for y, C in zip(ys, Cs):
        for j in range(7):
            mj = ((1 << (8 * j)) * C) % t
            yj = (y >> (8 * j)) & 0xFF
            for c in range(7):
                S[c] += yj * ((mj >> (8 * c)) & 0xFF)
    b = []
    for c in range(7):
        f = 2.0 ** 23 + S[c]
        assert f < 2.0 ** 24  # every partial sum is an exact f32 integer
        bits = struct.unpack("<I", struct.pack("<f", f))[0]
        assert bits == 0x4B000000 + S[c]
        b.append(bits)
    lo_bias = 0x4B000000 * (1 + (1 << 8) + (1 << 16) + (1 << 24) + (1 << 32))
    lo = b[0] + (b[1] << 8) + (b[2] << 16) + (b[3] << 24) + (b[4] << 32)
    assert lo <= M64
    hi = (b[5] + (b[6] << 8) - 0x4B000000 * 257) & M32
    assert hi == S[5] + (S[6] << 8)
    assert lo - lo_bias + (hi << 40) == sum(S[c] << (8 * c) for c in range(7))
    # the staged offset [-sub]_t - lo_bias, added modulo 2^64 as the kernel does
    off = ((t - sub % t) % t - lo_bias) & M64
    fold = shoup_u32(hi, (1 << 40) % t, t)
    v = (lo + fold + off) & M64
    assert v == lo - lo_bias + fold + (t - sub % t) % t  # no wrap in the true sum
    assert v <= M64
    if lazy:
        assert v < 8 * t  # the lazy forward NTT's input bound
    else:
        _, v = shoup_one(v, t)
    return v


@pytest.mark.parametrize("bits,nsrc", [(54, 9), (54, 16), (55, 16), (50, 4), (50, 16)])
def test_tc_conversion_arithmetic(bits, nsrc):
    rng = random.Random(bits * 100 + nsrc)
    for trial in range(60):
        t = rng.randrange(1 << (bits - 1), 1 << bits) | 1
        qs = [rng.randrange(1 << (bits - 1), 1 << bits) | 1 for _ in range(nsrc)]
        if trial % 3 == 0:  # largest byte sums: every byte of y and of M' near 255
            t = (1 << bits) - rng.randrange(1, 1000, 2)
            ys = [q - 1 for q in qs]
        else:
            ys = [rng.randrange(q) for q in qs]
        if trial % 5 == 1:  # the smallest prime the lazy bound allows
            t = (1 << (bits - 1)) + 1
        Cs = [rng.randrange(t) for _ in range(nsrc)]
        sub = rng.randrange(t)
        lazy = _tc_lazy(nsrc, 1 << (bits - 1))
        out = _tc_convert(ys, Cs, t, sub, lazy)
        assert out < (8 if lazy else 3) * t
        assert out % t == (sum(y * C for y, C in zip(ys, Cs)) - sub) % t


def test_tc_lazy_holds_at_the_key_switching_shapes():
    # 54-bit primes with max(alpha, k + 1) = 9 sources: no final reduction
    assert _tc_lazy(9, 1 << 53)
    assert not _tc_lazy(16, 1 << 49)


def test_tc_byte_sums_stay_below_two_to_23_at_sixteen_sources():
    # the bound the kernel relies on: 16 sources x 7 bytes x 255^2
    assert 16 * 7 * 255 * 255 < 2 ** 23
