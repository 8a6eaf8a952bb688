"""Oracle pins for the basis-change steps, by big-integer CRT (not GPU).

* ModUp (Algorithm 6): the coefficient-form output, CRT-reconstructed over
  C_ell U P, equals X_j + u*Q_j with one integer u in [0, alpha), X_j being
  the digit's own CRT value.
* ModDown by P: out = floor((X + floor(P/2)) / P) - eps, eps in [0, k).
* Rescale: exactly round(X / q_{ell-1}) mod Q_{ell-1}.
* PModUp: ModDown(PModUp(y)) == y.
"""
from math import prod

import numpy as np
import pytest

import synth
from tests.crt import crt_columns


def make_params(oracle_lib, logN=5, L=6, k=3, dnum=2, bits=50, prime_logN=12):
    primes = oracle_lib.gen_primes(bits, prime_logN, L + k)
    return oracle_lib.Params(logN, L, k, dnum, primes=primes)


@pytest.mark.parametrize("L,k,dnum,ell", [(6, 3, 2, 6), (6, 3, 2, 5), (6, 3, 2, 4), (7, 3, 3, 7), (8, 4, 2, 3)])
def test_modup_crt(oracle_lib, L, k, dnum, ell):
    P = make_params(oracle_lib, L=L, k=k, dnum=dnum)
    ext = P.ext_primes(ell)
    a = synth.uniform_residues(P.primes[:ell], P.N, "pin/modup/a")
    a_coeff = np.stack([oracle_lib.intt(a[i], P.logN, int(P.primes[i])) for i in range(ell)])
    for j in range(P.beta(ell)):
        lo, hi = j * P.alpha, min((j + 1) * P.alpha, ell)
        dig_mod = [int(x) for x in P.primes[lo:hi]]
        Qj = prod(dig_mod)
        out = oracle_lib.modup(P, ell, j, a)
        assert np.array_equal(out[lo:hi], a[lo:hi])  # digit limbs are copied
        Xout = crt_columns(oracle_lib.ntt_limbs(P, ell, out, inverse=True), ext)
        Xj = crt_columns(a_coeff[lo:hi], dig_mod)
        us = set()
        for xo, xj in zip(Xout, Xj):
            assert (xo - xj) % Qj == 0
            u = (xo - xj) // Qj
            assert 0 <= u < hi - lo
            us.add(u)
        if hi - lo > 1:
            assert len(us) > 1  # the approximate conversion really leaves u*Q_j terms


@pytest.mark.parametrize("L,k,dnum,ell", [(6, 3, 2, 6), (6, 3, 2, 2), (7, 4, 3, 5)])
def test_moddown_crt(oracle_lib, L, k, dnum, ell):
    P = make_params(oracle_lib, L=L, k=k, dnum=dnum)
    ext = P.ext_primes(ell)
    x = synth.uniform_residues(ext, P.N, "pin/moddown/x")
    out = oracle_lib.moddown(P, ell, x)
    X = crt_columns(oracle_lib.ntt_limbs(P, ell, x, inverse=True), ext)
    qs = [int(v) for v in P.primes[:ell]]
    Q = prod(qs)
    Pp = prod(int(v) for v in P.primes[P.L:])
    Y = crt_columns(np.stack([oracle_lib.intt(out[i], P.logN, qs[i]) for i in range(ell)]), qs)
    for xv, yv in zip(X, Y):
        eps = ((xv + Pp // 2) // Pp - yv) % Q
        assert 0 <= eps < P.k


@pytest.mark.parametrize("L,k,dnum,ell", [(6, 3, 2, 6), (6, 3, 2, 2), (7, 3, 3, 4)])
def test_moddown_merged_crt(oracle_lib, L, k, dnum, ell):
    """The merged ModDown of NewMult divides by D = P * q_{ell-1}: per
    coefficient, out = round(X / D) - eps (mod Q_{ell-1}) with eps in [0, k+1)
    (the fast conversion over the k+1 limbs of D), X the CRT value of the
    input over C_ell U P."""
    P = make_params(oracle_lib, L=L, k=k, dnum=dnum)
    ext = P.ext_primes(ell)
    x = synth.uniform_residues(ext, P.N, "pin/mdmerged/x")
    out = oracle_lib.moddown_merged(P, ell, x)
    assert out.shape == (ell - 1, P.N)
    X = crt_columns(oracle_lib.ntt_limbs(P, ell, x, inverse=True), ext)
    qs = [int(v) for v in P.primes[:ell]]
    D = prod(int(v) for v in P.primes[P.L:]) * qs[-1]
    Qd = prod(qs[:-1])
    Y = crt_columns(np.stack([oracle_lib.intt(out[i], P.logN, qs[i]) for i in range(ell - 1)]), qs[:-1])
    seen = set()
    for xv, yv in zip(X, Y):
        eps = ((xv + D // 2) // D - yv) % Qd
        assert 0 <= eps <= P.k
        seen.add(eps)
    assert len(seen) > 1  # the conversion error really occurs (not a vacuous bound)


@pytest.mark.parametrize("ell", [2, 3, 6])
def test_rescale_exact(oracle_lib, ell):
    P = make_params(oracle_lib)
    qs = [int(v) for v in P.primes[:ell]]
    x = synth.uniform_residues(qs, P.N, "pin/rescale/x")
    out = oracle_lib.rescale(P, ell, x)
    X = crt_columns(np.stack([oracle_lib.intt(x[i], P.logN, qs[i]) for i in range(ell)]), qs)
    Y = crt_columns(np.stack([oracle_lib.intt(out[i], P.logN, qs[i]) for i in range(ell - 1)]), qs[:-1])
    ql, Qd = qs[-1], prod(qs[:-1])
    for xv, yv in zip(X, Y):
        # q is odd, so round(X/ql) has no ties: floor((X + (ql-1)/2) / ql)
        assert yv == ((xv + ql // 2) // ql) % Qd


def test_pmodup_then_moddown_returns_input_up_to_constant(oracle_lib):
    """ModDown(PModUp(y)) = y - u_H: the P-limbs of P*y are 0, so after the
    rounding constant floor(P/2) is added every coefficient carries the same
    P-residues and the fast base conversion leaves the same u_H in [0, k) on
    every coefficient and limb."""
    P = make_params(oracle_lib)
    for ell in (1, 4, 6):
        y = synth.uniform_residues(P.primes[:ell], P.N, "pin/pmodup/y")
        lifted = oracle_lib.pmodup(P, ell, y)
        assert np.all(lifted[ell:] == 0)
        qs = [int(v) for v in P.primes[:ell]]
        for t, q in enumerate(qs):
            assert np.array_equal(lifted[t], np.array([int(v) * (prod(int(p) for p in P.primes[P.L:]) % q) % q
                                                       for v in y[t]], dtype=np.uint64))
        out = oracle_lib.moddown(P, ell, lifted)
        Q = prod(qs)
        Y0 = crt_columns(np.stack([oracle_lib.intt(y[i], P.logN, qs[i]) for i in range(ell)]), qs)
        Y1 = crt_columns(np.stack([oracle_lib.intt(out[i], P.logN, qs[i]) for i in range(ell)]), qs)
        diffs = {(y0 - y1) % Q for y0, y1 in zip(Y0, Y1)}
        assert len(diffs) == 1 and 0 <= diffs.pop() < P.k
