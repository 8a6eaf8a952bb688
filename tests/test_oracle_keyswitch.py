"""Oracle pins for KeySwitch / Rotate / HRotate / PtMatVecMult by decryption.

A real ternary secret s and Gaussian errors (sigma 3.2, |e| <= 19) give keys
b_j = -a_j s + e_j + g_j s' (Eq. kskShape, Han-Ki gadget g_j = [P]_{q_i} on
digit j).  The key-switch error e = u*s + v - a*s' must satisfy

  |e|_inf <= beta*alpha*N*19*max_j(Q_j)/P + (h_s+1)/2 + (k-1)(h_s+1) + 1,

derived from: ModUp lifts digit j to a value < alpha*Q_j (FastBConv leaves
u*Q_j, u < alpha); the inner product adds sum_j d_j e_j; ModDown divides by P
with rounding error <= 1/2 per term and a FastBConv error eps in [0, k).
A dropped term, a wrong sign or a transposed operand gives errors of size Q.
"""
from math import prod

import numpy as np
import pytest

import synth
from tests.crt import automorph_int, centered, crt_columns, negacyclic_mul


def params(oracle_lib, logN, L, k, dnum, bits=50, prime_logN=12):
    return oracle_lib.Params(logN, L, k, dnum, primes=oracle_lib.gen_primes(bits, prime_logN, L + k))


def make_key(oracle_lib, P, s, sp_eval, tag):
    a = np.stack([synth.uniform_residues(P.primes, P.N, f"{tag}/a{j}") for j in range(P.dnum)])
    e = np.stack([synth.gaussian(P.N, f"{tag}/e{j}") for j in range(P.dnum)])
    return oracle_lib.keygen(P, a, s, sp_eval, e)


def ks_bound(P, ell, s):
    alpha, beta = P.alpha, P.beta(ell)
    Pp = prod(int(x) for x in P.primes[P.L:])
    qmax = max(prod(int(x) for x in P.primes[j * alpha:min((j + 1) * alpha, ell)]) for j in range(beta))
    hs = int(np.count_nonzero(s))
    return beta * alpha * P.N * 19 * qmax / Pp + (hs + 1) / 2 + (P.k - 1) * (hs + 1) + 1


def decrypt_int(oracle_lib, P, ell, s, a, b):
    res = oracle_lib.decrypt_residues(P, ell, s, a, b)
    qs = [int(x) for x in P.primes[:ell]]
    Q = prod(qs)
    return [centered(x, Q) for x in crt_columns(res, qs)]


def encrypt(oracle_lib, P, ell, s, tag, mbound=1000):
    m = synth.small_uniform(P.N, f"{tag}/m", mbound)
    e = synth.gaussian(P.N, f"{tag}/e")
    a = synth.uniform_residues(P.primes[:ell], P.N, f"{tag}/a")
    b = oracle_lib.encrypt(P, ell, s, m + e, a)
    return a, b, [int(x) for x in m + e]


CASES = [
    # logN, L, k, dnum, ell   (first: the single-KeySwitch configuration N=2^12, ell=6, k=3, dnum=2)
    (12, 6, 3, 2, 6),
    (6, 6, 3, 2, 5),
    (6, 7, 3, 3, 7),
    (6, 8, 4, 2, 3),
    (6, 6, 3, 2, 1),
]


@pytest.mark.parametrize("logN,L,k,dnum,ell", CASES)
def test_keyswitch_decrypts_within_bound(oracle_lib, logN, L, k, dnum, ell):
    P = params(oracle_lib, logN, L, k, dnum)
    s = synth.ternary(P.N, "pin/ks/s")
    s2 = synth.ternary(P.N, "pin/ks/s_prime")
    sp = oracle_lib.signed_to_eval(P, s2)
    key = make_key(oracle_lib, P, s, sp, "pin/ks/key")
    a = synth.uniform_residues(P.primes[:ell], P.N, "pin/ks/a")
    u, v = oracle_lib.keyswitch(P, ell, a, key)
    # e = u*s + v - a*s'
    qs = [int(x) for x in P.primes[:ell]]
    dec = oracle_lib.decrypt_residues(P, ell, s, u, v)
    a_sp = np.stack([oracle_lib.intt(np.array([int(x) * int(y) % q for x, y in zip(a[i], sp[i])], dtype=np.uint64),
                                     P.logN, q) for i, q in enumerate(qs)])
    Q = prod(qs)
    err = [centered(x - y, Q) for x, y in zip(crt_columns(dec, qs), crt_columns(a_sp, qs))]
    bound = ks_bound(P, ell, s)
    assert max(abs(x) for x in err) <= bound
    assert bound < Q / 4


@pytest.mark.parametrize("logN,L,k,dnum,ell,r", [(12, 6, 3, 2, 6, 1), (6, 6, 3, 2, 5, 3), (6, 7, 3, 3, 7, 2)])
def test_rotate_and_hrotate_decrypt(oracle_lib, logN, L, k, dnum, ell, r):
    P = params(oracle_lib, logN, L, k, dnum)
    twoN = 2 * P.N
    s = synth.ternary(P.N, "pin/rot/s")
    a, b, mprime = encrypt(oracle_lib, P, ell, s, "pin/rot/ct")
    gs = [pow(5, i + 1, twoN) for i in range(r - 1)] + [twoN - 1]  # rotations and a conjugation
    keys = [make_key(oracle_lib, P, s, oracle_lib.rot_secret(P, s, g), f"pin/rot/key{g}") for g in gs]
    bound = ks_bound(P, ell, s)
    outs = oracle_lib.hrotate(P, ell, a, b, gs, keys)
    for g, key, (oa, ob) in zip(gs, keys, outs):
        expect = automorph_int(mprime, g)
        got = decrypt_int(oracle_lib, P, ell, s, oa, ob)
        assert max(abs(x - y) for x, y in zip(got, expect)) <= bound
        ra, rb = oracle_lib.rotate(P, ell, a, b, g, key)
        got_r = decrypt_int(oracle_lib, P, ell, s, ra, rb)
        assert max(abs(x - y) for x, y in zip(got_r, expect)) <= bound
        # Algorithm 3 automorphs before ModUp, Algorithm 4 after: different bits, same message
        assert not (np.array_equal(ra, oa) and np.array_equal(rb, ob))


def test_relinearisation_key_switches_s_squared(oracle_lib):
    P = params(oracle_lib, 6, 6, 3, 2)
    ell = 6
    s = synth.ternary(P.N, "pin/relin/s")
    key = make_key(oracle_lib, P, s, oracle_lib.sq_secret(P, s), "pin/relin/key")
    a = synth.uniform_residues(P.primes[:ell], P.N, "pin/relin/a")
    u, v = oracle_lib.keyswitch(P, ell, a, key)
    # u*s + v ~ a*s^2: decrypting (u, v) and (a*s, 0) under s must agree up to the bound
    qs = [int(x) for x in P.primes[:ell]]
    Q = prod(qs)
    s_int = [int(x) for x in s]
    s2 = negacyclic_mul(s_int, s_int)
    a_coeff = crt_columns(np.stack([oracle_lib.intt(a[i], P.logN, q) for i, q in enumerate(qs)]), qs)
    a_s2 = negacyclic_mul(a_coeff, s2)
    dec = crt_columns(oracle_lib.decrypt_residues(P, ell, s, u, v), qs)
    err = [centered(x - y, Q) for x, y in zip(dec, a_s2)]
    assert max(abs(x) for x in err) <= ks_bound(P, ell, s)


@pytest.mark.parametrize("nb,ng,ell,rescale", [(2, 2, 6, False), (3, 1, 5, False), (2, 2, 6, True)])
def test_ptmatvec_decrypts(oracle_lib, nb, ng, ell, rescale):
    P = params(oracle_lib, 6, 6, 3, 2)
    twoN = 2 * P.N
    s = synth.ternary(P.N, "pin/pmv/s")
    a, b, mprime = encrypt(oracle_lib, P, ell, s, "pin/pmv/ct", mbound=100)
    stride = 1
    g_baby = [1] + [pow(5, i * stride, twoN) for i in range(1, nb)]
    g_giant = [1] + [pow(5, t * nb * stride, twoN) for t in range(1, ng)]
    key_b = [None] + [make_key(oracle_lib, P, s, oracle_lib.rot_secret(P, s, g), f"pin/pmv/kb{i}")
                      for i, g in enumerate(g_baby) if i > 0]
    key_g = [None] + [make_key(oracle_lib, P, s, oracle_lib.rot_secret(P, s, g), f"pin/pmv/kg{t}")
                      for t, g in enumerate(g_giant) if t > 0]
    rows = list(range(ell)) + list(range(P.L, P.L + P.k))
    Ms = [synth.small_uniform(P.N, f"pin/pmv/M{d}", 2) for d in range(nb * ng)]
    diags = [oracle_lib.signed_to_eval(P, M)[rows] for M in Ms]
    oa, ob = oracle_lib.ptmatvec(P, ell, a, b, nb, ng, g_baby, g_giant, key_b, key_g, diags, rescale_out=rescale)
    expect = [0] * P.N
    for t in range(ng):
        inner = [0] * P.N
        for i in range(nb):
            term = negacyclic_mul([int(x) for x in Ms[t * nb + i]], automorph_int(mprime, g_baby[i]))
            inner = [x + y for x, y in zip(inner, term)]
        rot = automorph_int(inner, g_giant[t]) if t > 0 else inner
        expect = [x + y for x, y in zip(expect, rot)]
    Bks = ks_bound(P, ell, s)
    hs = int(np.count_nonzero(s))
    per_giant = nb * P.N * 2 * (Bks) + (hs + 1) / 2 + (P.k - 1) * (hs + 1) + 1
    bound = ng * (per_giant + Bks)
    if rescale:
        ql = int(P.primes[ell - 1])
        got = decrypt_int(oracle_lib, P, ell - 1, s, oa, ob)
        # Rescale divides message and error by q_last (the rounding adds < 1 + h_s/2)
        assert max(abs(x - y / ql) for x, y in zip(got, expect)) <= bound / ql + 1 + (hs + 1) / 2
    else:
        got = decrypt_int(oracle_lib, P, ell, s, oa, ob)
        assert max(abs(x - y) for x, y in zip(got, expect)) <= bound


@pytest.mark.parametrize("logN,L,k,dnum,ell", [(6, 6, 3, 2, 6), (6, 7, 3, 3, 4), (6, 6, 3, 2, 2), (12, 6, 3, 2, 6)])
def test_mult_decrypts_to_rescaled_product(oracle_lib, logN, L, k, dnum, ell):
    """Algorithm 2: Dec(Mult(ct1, ct2)) = (m1 * m2 + e_ks) / q_{ell-1} up to the
    Rescale rounding, where m_i = Delta * x_i + e_i are the encrypted
    polynomials and * is the negacyclic product.  With a the rescaled
    ciphertext's rounding residues r_a, r_b (|r| <= q/2):
      |Dec(out) - m1*m2 / q_{ell-1}| <= ks_bound / q_{ell-1} + (h_s + 1) / 2."""
    P = params(oracle_lib, logN, L, k, dnum)
    s = synth.ternary(P.N, "pin/mult/s")
    rlk = make_key(oracle_lib, P, s, oracle_lib.sq_secret(P, s), "pin/mult/rlk")
    ql = int(P.primes[ell - 1])
    delta = 1 << (ql.bit_length() // 2 + 4)
    cts, ms = [], []
    for i in range(2):
        x = synth.small_uniform(P.N, f"pin/mult/x{i}", 8)
        m = delta * x + synth.gaussian(P.N, f"pin/mult/e{i}")
        a = synth.uniform_residues(P.primes[:ell], P.N, f"pin/mult/a{i}")
        cts.append((a, oracle_lib.encrypt(P, ell, s, m, a)))
        ms.append([int(v) for v in m])
    (a1, b1), (a2, b2) = cts
    oa, ob = oracle_lib.mult(P, ell, a1, b1, a2, b2, rlk)
    assert oa.shape == (ell - 1, P.N)
    got = decrypt_int(oracle_lib, P, ell - 1, s, oa, ob)
    prod_m = negacyclic_mul(ms[0], ms[1])
    hs = int(np.count_nonzero(s))
    bound = ks_bound(P, ell, s) / ql + (hs + 1) / 2
    err = max(abs(g * ql - t) for g, t in zip(got, prod_m)) / ql
    assert err <= bound
    assert max(abs(t) for t in prod_m) / ql > 100 * bound  # the check is not vacuous
    # both operand orders give the same bits (the tensor step is symmetric)
    oa2, ob2 = oracle_lib.mult(P, ell, a2, b2, a1, b1, rlk)
    np.testing.assert_array_equal(oa, oa2)
    np.testing.assert_array_equal(ob, ob2)


@pytest.mark.parametrize("logN,L,k,dnum,ell", [(6, 6, 3, 2, 6), (6, 7, 3, 3, 4), (6, 6, 3, 2, 2)])
def test_newmult_decrypts_to_rescaled_product(oracle_lib, logN, L, k, dnum, ell):
    """Algorithm 7: the lifted sum P*(m1*m2) + E is divided by P*q_{ell-1} in one
    merged ModDown, so |Dec(out) - m1*m2 / q_{ell-1}| <= E/(P q_{ell-1}) +
    (h_s + 1)/2 + (k + 1)(h_s + 1) + 1 (rounding of both polynomials, the fast
    conversion error over k+1 limbs), E the ModUp / inner-product noise."""
    P = params(oracle_lib, logN, L, k, dnum)
    s = synth.ternary(P.N, "pin/newmult/s")
    rlk = make_key(oracle_lib, P, s, oracle_lib.sq_secret(P, s), "pin/newmult/rlk")
    ql = int(P.primes[ell - 1])
    delta = 1 << (ql.bit_length() // 2 + 4)
    cts, ms = [], []
    for i in range(2):
        x = synth.small_uniform(P.N, f"pin/newmult/x{i}", 8)
        m = delta * x + synth.gaussian(P.N, f"pin/newmult/e{i}")
        a = synth.uniform_residues(P.primes[:ell], P.N, f"pin/newmult/a{i}")
        cts.append((a, oracle_lib.encrypt(P, ell, s, m, a)))
        ms.append([int(v) for v in m])
    (a1, b1), (a2, b2) = cts
    oa, ob = oracle_lib.newmult(P, ell, a1, b1, a2, b2, rlk)
    got = decrypt_int(oracle_lib, P, ell - 1, s, oa, ob)
    prod_m = negacyclic_mul(ms[0], ms[1])
    hs = int(np.count_nonzero(s))
    alpha, beta = P.alpha, P.beta(ell)
    Pp = prod(int(x) for x in P.primes[P.L:])
    qmax = max(prod(int(x) for x in P.primes[j * alpha:min((j + 1) * alpha, ell)]) for j in range(beta))
    bound = beta * alpha * P.N * 19 * qmax / (Pp * ql) + (hs + 1) / 2 + (P.k + 1) * (hs + 1) + 1
    err = max(abs(g * ql - t) for g, t in zip(got, prod_m)) / ql
    assert err <= bound
    assert max(abs(t) for t in prod_m) / ql > 100 * bound
    # the same product as Algorithm 2 up to the two methods' error terms, but other bits
    ra, rb = oracle_lib.mult(P, ell, a1, b1, a2, b2, rlk)
    assert not (np.array_equal(ra, oa) and np.array_equal(rb, ob))


@pytest.mark.parametrize("n,ell", [(3, 6), (2, 2)])
def test_newmult_sum_decrypts_to_the_inner_product(oracle_lib, n, ell):
    """The ModDown-hoisted encrypted inner product: one merged ModDown after the
    sum of the n lifted products, so Dec(out) ~ sum_i m1_i*m2_i / q_{ell-1}
    within n*E/(P q_{ell-1}) + (h_s+1)/2 + (k+1)(h_s+1) + 1; for n = 1 it is
    NewMult bit for bit."""
    P = params(oracle_lib, 6, 6, 3, 2)
    s = synth.ternary(P.N, "pin/nmsum/s")
    rlk = make_key(oracle_lib, P, s, oracle_lib.sq_secret(P, s), "pin/nmsum/rlk")
    ql = int(P.primes[ell - 1])
    delta = 1 << (ql.bit_length() // 2 + 4)
    cts1, cts2, ms1, ms2 = [], [], [], []
    for i in range(n):
        for cts, ms, tag in ((cts1, ms1, "x"), (cts2, ms2, "y")):
            m = delta * synth.small_uniform(P.N, f"pin/nmsum/{tag}{i}", 8) + synth.gaussian(P.N, f"pin/nmsum/e{tag}{i}")
            a = synth.uniform_residues(P.primes[:ell], P.N, f"pin/nmsum/a{tag}{i}")
            cts.append((a, oracle_lib.encrypt(P, ell, s, m, a)))
            ms.append([int(v) for v in m])
    oa, ob = oracle_lib.newmult_sum(P, ell, cts1, cts2, rlk)
    got = decrypt_int(oracle_lib, P, ell - 1, s, oa, ob)
    want = [0] * P.N
    for m1, m2 in zip(ms1, ms2):
        want = [w + v for w, v in zip(want, negacyclic_mul(m1, m2))]
    hs = int(np.count_nonzero(s))
    alpha, beta = P.alpha, P.beta(ell)
    Pp = prod(int(x) for x in P.primes[P.L:])
    qmax = max(prod(int(x) for x in P.primes[j * alpha:min((j + 1) * alpha, ell)]) for j in range(beta))
    bound = n * beta * alpha * P.N * 19 * qmax / (Pp * ql) + (hs + 1) / 2 + (P.k + 1) * (hs + 1) + 1
    assert max(abs(g * ql - t) for g, t in zip(got, want)) / ql <= bound
    assert max(abs(t) for t in want) / ql > 100 * bound
    one = oracle_lib.newmult_sum(P, ell, cts1[:1], cts2[:1], rlk)
    ref = oracle_lib.newmult(P, ell, *cts1[0], *cts2[0], rlk)
    np.testing.assert_array_equal(one[0], ref[0])
    np.testing.assert_array_equal(one[1], ref[1])
