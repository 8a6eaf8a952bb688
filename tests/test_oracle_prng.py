"""Pins of the key-compression generator (Sec. 5.3): the oracle regenerates
the uniform half a_j of a key-switching key from a 64-bit seed with SplitMix64
(Steele, Lea and Flood, OOPSLA 2014) and per-element rejection to [0, q).

* published values: SplitMix64 seeded with 0 starts 0xE220A8397B1DCDAF,
  0x6E789E6AA1B965F4, 0x06C45D188009454F;
* a second implementation (numpy, synth.splitmix64) of the same definition
  gives the same element for every (digit, limb, coefficient) sampled;
* the values are residues (< q) and look uniform (mean and top-bit balance).
"""
import numpy as np
import pytest

import synth

PUBLISHED_SEED0 = [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]


def _params(oracle_lib, bits=50, logN=6, L=4, k=2, dnum=2):
    return oracle_lib.Params(logN, L, k, dnum, primes=oracle_lib.gen_primes(bits, 12, L + k))


def _reference(P, seed, j, l, n):
    q = int(P.primes[l])
    b = q.bit_length()
    e = (j * (P.L + P.k) + l) * P.N + n
    draws = synth.splitmix64(seed, 16, offset=16 * e)
    v = 0
    for x in draws:
        v = int(x) >> (64 - b)
        if v < q:
            return v
    return v % q


def test_splitmix64_published_values():
    assert [int(x) for x in synth.splitmix64(0, 3)] == PUBLISHED_SEED0


def test_first_element_of_seed_zero_is_the_published_draw(oracle_lib):
    P = _params(oracle_lib)
    q = int(P.primes[0])
    b = q.bit_length()
    first = PUBLISHED_SEED0[0] >> (64 - b)
    second = PUBLISHED_SEED0[1] >> (64 - b)
    want = first if first < q else (second if second < q else None)
    assert want is not None
    assert oracle_lib.prng_key_a_element(P, 0, 0, 0, 0) == want


@pytest.mark.parametrize("bits", [50, 54, 60])
def test_prng_matches_independent_implementation(oracle_lib, bits):
    P = _params(oracle_lib, bits=bits)
    seed = synth.stream_seed("pin/prng/seed")
    a = oracle_lib.prng_key_a(P, seed)
    rng = np.random.default_rng(7)
    for _ in range(200):
        j = int(rng.integers(P.dnum))
        l = int(rng.integers(P.L + P.k))
        n = int(rng.integers(P.N))
        assert int(a[j, l, n]) == _reference(P, seed, j, l, n)


def test_prng_values_are_uniform_residues(oracle_lib):
    P = _params(oracle_lib, logN=10)
    a = oracle_lib.prng_key_a(P, 987654321)
    for l, q in enumerate(P.primes):
        col = a[:, l, :].astype(np.float64).ravel()
        assert np.all(a[:, l, :] < np.uint64(q))
        assert abs(col.mean() / q - 0.5) < 0.02
        assert abs(np.mean(col > q / 2) - 0.5) < 0.03
    # different seeds give different keys
    assert not np.array_equal(a, oracle_lib.prng_key_a(P, 987654322))
