"""Oracle pins: prime chain and roots of unity (not GPU).

The configurations ask for the largest NTT-friendly primes (q = 1 mod 2N)
below 2^bits; the pins check that with an independent primality routine
(sympy) and by showing that no candidate was skipped.
"""
import pytest

sympy = pytest.importorskip("sympy")


@pytest.mark.parametrize("bits,logN,count", [(50, 12, 9), (54, 16, 32), (54, 15, 32), (40, 5, 12)])
def test_primes_are_the_largest_ntt_friendly(oracle_lib, bits, logN, count):
    ps = oracle_lib.gen_primes(bits, logN, count)
    twoN = 2 << logN
    assert len(ps) == count
    assert all(p < (1 << bits) for p in ps)
    assert all(p % twoN == 1 for p in ps)
    assert ps == sorted(ps, reverse=True) and len(set(ps)) == count
    assert all(sympy.isprime(p) for p in ps)
    # no skipped candidate: every 1 + m*2N between consecutive primes is composite
    m_top = ((1 << bits) - 2) // twoN
    m = m_top
    for p in ps:
        while 1 + m * twoN > p:
            assert not sympy.isprime(1 + m * twoN)
            m -= 1
        assert 1 + m * twoN == p
        m -= 1


def test_is_prime_small_and_carmichael(oracle_lib):
    for n in range(0, 2000):
        assert oracle_lib.is_prime(n) == sympy.isprime(n), n
    for n in [561, 1105, 1729, 2465, 2821, 6601, 3215031751, 2152302898747, 3474749660383]:
        assert not oracle_lib.is_prime(n)
    assert oracle_lib.is_prime((1 << 61) - 1)


@pytest.mark.parametrize("bits,logN,idx", [(50, 12, 0), (50, 12, 5), (54, 16, 0), (54, 16, 31), (40, 5, 3)])
def test_min_psi_is_smallest_primitive_2N_root(oracle_lib, bits, logN, idx):
    q = oracle_lib.gen_primes(bits, logN, idx + 1)[idx]
    N = 1 << logN
    psi = oracle_lib.min_psi(q, logN)
    assert pow(psi, N, q) == q - 1
    # independent: primitive root of Z_q^* from sympy, all N odd powers
    g = sympy.primitive_root(q)
    root = pow(g, (q - 1) // (2 * N), q)
    cands = set()
    cur, r2 = root, root * root % q
    for _ in range(N):
        cands.add(cur)
        cur = cur * r2 % q
    assert len(cands) == N
    assert psi == min(cands)
