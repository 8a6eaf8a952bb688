"""Oracle pins for the NTT (Sec. 2.3, "Polynomial Representation").

* the fast transform against the O(N^2) definition evaluated in Python;
* iNTT(NTT(a) * NTT(b)) against the schoolbook negacyclic product;
* round trips at the full ring sizes of the configurations.
"""
import numpy as np
import pytest

from tests.crt import negacyclic_mul


def brv(x, bits):
    return int(format(x, f"0{bits}b")[::-1], 2) if bits else 0


def _rand(q, N, seed):
    rng = np.random.default_rng(seed)
    return np.array([int(rng.integers(0, 1 << 62)) % q for _ in range(N)], dtype=np.uint64)


@pytest.mark.parametrize("logN", [1, 2, 3, 4, 5, 6])
def test_ntt_matches_definition(oracle_lib, logN):
    N = 1 << logN
    for q in oracle_lib.gen_primes(50, 12, 3):
        a = _rand(q, N, logN + q % 97)
        psi = oracle_lib.min_psi(q, logN)
        expect = [sum(int(a[i]) * pow(psi, (2 * brv(j, logN) + 1) * i, q) for i in range(N)) % q for j in range(N)]
        assert [int(x) for x in oracle_lib.ntt(a, logN, q)] == expect
        assert [int(x) for x in oracle_lib.ntt_naive(a, logN, q)] == expect


@pytest.mark.parametrize("logN", [4, 7, 8])
def test_ntt_product_is_negacyclic_convolution(oracle_lib, logN):
    N = 1 << logN
    q = oracle_lib.gen_primes(54, 16, 1)[0]
    a, b = _rand(q, N, 1), _rand(q, N, 2)
    ah, bh = oracle_lib.ntt(a, logN, q), oracle_lib.ntt(b, logN, q)
    prod_h = np.array([int(x) * int(y) % q for x, y in zip(ah, bh)], dtype=np.uint64)
    got = [int(x) for x in oracle_lib.intt(prod_h, logN, q)]
    expect = [c % q for c in negacyclic_mul(a, b)]
    assert got == expect


@pytest.mark.parametrize("bits,logN", [(50, 12), (54, 16)])
def test_ntt_round_trip_full_size(oracle_lib, bits, logN):
    N = 1 << logN
    q = oracle_lib.gen_primes(bits, logN, 2)[1]
    a = _rand(q, N, 3)
    ah = oracle_lib.ntt(a, logN, q)
    assert not np.array_equal(ah, a)
    assert np.array_equal(oracle_lib.intt(ah, logN, q), a)


def test_ntt_of_monomial_and_constant(oracle_lib):
    # NTT(1) is all ones; NTT(X) at slot j is psi^(2 brv(j)+1)
    logN, q = 10, oracle_lib.gen_primes(50, 12, 1)[0]
    N = 1 << logN
    one = np.zeros(N, dtype=np.uint64)
    one[0] = 1
    assert np.all(oracle_lib.ntt(one, logN, q) == 1)
    x = np.zeros(N, dtype=np.uint64)
    x[1] = 1
    psi = oracle_lib.min_psi(q, logN)
    got = oracle_lib.ntt(x, logN, q)
    for j in [0, 1, 2, 3, 511, 512, N - 1]:
        assert int(got[j]) == pow(psi, 2 * brv(j, logN) + 1, q)
