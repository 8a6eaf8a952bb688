"""Oracle pins for Automorph (table "CKKS Subroutines"): X -> X^g."""
import numpy as np
import pytest

from tests.crt import automorph_int


def _rand(q, N, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(0, 1 << 62, size=N, dtype=np.uint64) % np.uint64(q)).astype(np.uint64)


@pytest.mark.parametrize("logN", [3, 6, 10])
def test_coeff_automorph_definition(oracle_lib, logN):
    N = 1 << logN
    q = oracle_lib.gen_primes(50, 12, 1)[0]
    a = _rand(q, N, 7)
    for g in [5, pow(5, 3, 2 * N), 2 * N - 1, 3]:
        got = [int(x) for x in oracle_lib.automorph_coeff(a, logN, g, q)]
        assert got == [c % q for c in automorph_int([int(x) for x in a], g)]


@pytest.mark.parametrize("logN", [4, 6, 10, 12])
def test_eval_automorph_matches_coefficient_automorph(oracle_lib, logN):
    N = 1 << logN
    q = oracle_lib.gen_primes(50, 12, 2)[1]
    x = _rand(q, N, 11)
    for g in [5, pow(5, 7, 2 * N), 2 * N - 1]:
        coeff = oracle_lib.intt(x, logN, q)
        expect = oracle_lib.ntt(oracle_lib.automorph_coeff(coeff, logN, g, q), logN, q)
        assert np.array_equal(oracle_lib.automorph_eval(x, logN, g), expect)


def test_eval_automorph_composes(oracle_lib):
    logN = 8
    N = 1 << logN
    q = oracle_lib.gen_primes(50, 12, 1)[0]
    x = _rand(q, N, 5)
    g, h = pow(5, 3, 2 * N), 2 * N - 1
    lhs = oracle_lib.automorph_eval(oracle_lib.automorph_eval(x, logN, h), logN, g)
    rhs = oracle_lib.automorph_eval(x, logN, g * h % (2 * N))
    assert np.array_equal(lhs, rhs)
    assert np.array_equal(oracle_lib.automorph_eval(x, logN, 1), x)
