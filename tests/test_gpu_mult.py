"""Mult with relinearisation and Rescale (Algorithm 2) and NewMult (Algorithm 7,
the merged ModDown) through the C ABI: single and batched, bit-exact against
the oracle (tolerance 0)."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg1(oracle_lib):
    return Setup(oracle_lib, 12, 6, 3, 2, 50)


@pytest.fixture(scope="module")
def cfg_odd(oracle_lib):
    return Setup(oracle_lib, 11, 7, 3, 3, 50)


def _pair(S, ell, tag):
    a1, b1 = S.ct(ell, f"{tag}/1")
    a2, b2 = S.ct(ell, f"{tag}/2")
    return a1, b1, a2, b2


@pytest.mark.parametrize("new", [False, True])
@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_mult_parity(request, which, new):
    S = request.getfixturevalue(which)
    P = S.P
    key = S.key(0, f"gpu/mult/{which}/rlk")[0]
    dk = dev(key)
    ref = S.o.newmult if new else S.o.mult
    for ell in sorted({P.L, P.alpha + 1, 2}):
        a1, b1, a2, b2 = _pair(S, ell, f"gpu/mult/{which}/{ell}")
        oa, ob = S.ctx.mult(dev(a1), dev(b1), dev(a2), dev(b2), ell, dk, new=new)
        ra, rb = ref(P, ell, a1, b1, a2, b2, key)
        np.testing.assert_array_equal(host(oa), ra, err_msg=f"ell={ell}")
        np.testing.assert_array_equal(host(ob), rb, err_msg=f"ell={ell}")


@pytest.mark.parametrize("new", [False, True])
def test_mult_batch_uneven_levels(cfg_odd, new):
    """Batched products at levels 2..7 with two keys: each entry equals the
    single call and the oracle."""
    S = cfg_odd
    P = S.P
    keys = [S.key(0, "gpu/multb/rlk0")[0], S.key(0, "gpu/multb/rlk1")[0]]
    dkeys = [dev(k) for k in keys]
    levels = [7, 2, 5, 3, 7, 4, 6, 2]
    cts = [_pair(S, ell, f"gpu/multb/{i}") for i, ell in enumerate(levels)]
    d1 = [(dev(c[0]), dev(c[1])) for c in cts]
    d2 = [(dev(c[2]), dev(c[3])) for c in cts]
    outs = S.ctx.mult_batch(d1, d2, levels, [dkeys[i % 2] for i in range(len(levels))], new=new)
    ref = S.o.newmult if new else S.o.mult
    for i, ell in enumerate(levels):
        sa, sb = S.ctx.mult(*d1[i], *d2[i], ell, dkeys[i % 2], new=new)
        np.testing.assert_array_equal(host(outs[i][0]), host(sa))
        np.testing.assert_array_equal(host(outs[i][1]), host(sb))
        ra, rb = ref(P, ell, *cts[i], keys[i % 2])
        np.testing.assert_array_equal(host(outs[i][0]), ra, err_msg=f"entry {i}")
        np.testing.assert_array_equal(host(outs[i][1]), rb, err_msg=f"entry {i}")


@pytest.mark.parametrize("new", [False, True])
def test_mult_wide_primes(oracle_lib, new):
    """58-bit primes: the entries run with the single-operation launches."""
    S = Setup(oracle_lib, 11, 4, 2, 2, 58)
    key = S.key(0, "gpu/multw/rlk")[0]
    ref = S.o.newmult if new else S.o.mult
    for ell in (4, 2):
        cts = _pair(S, ell, f"gpu/multw/{ell}")
        oa, ob = S.ctx.mult(*[dev(x) for x in cts], ell, dev(key), new=new)
        ra, rb = ref(S.P, ell, *cts, key)
        np.testing.assert_array_equal(host(oa), ra)
        np.testing.assert_array_equal(host(ob), rb)


def test_mult_rejects_level_one(cfg1):
    ckks = _gpu()
    a1, b1, a2, b2 = _pair(cfg1, 1, "gpu/mult/l1")
    key = dev(cfg1.key(0, "gpu/mult/l1/rlk")[0])
    with pytest.raises(ckks.CkksError):
        cfg1.ctx.mult(dev(a1), dev(b1), dev(a2), dev(b2), 1, key, oa=cfg1.ctx.empty(1), ob=cfg1.ctx.empty(1),
                      ws=cfg1.ctx.workspace(3, 1))


def test_mult_headline_shape(oracle_lib):
    """N=2^16, ell=24, k=8, dnum=3, 54-bit primes (one full oracle run each)."""
    S = Setup(oracle_lib, 16, 24, 8, 3, 54)
    key = S.key(0, "gpu/B/relin")[0]
    cts = _pair(S, 24, "gpu/B/mult")
    dk, dc = dev(key), [dev(x) for x in cts]
    for new, ref in ((False, S.o.mult), (True, S.o.newmult)):
        oa, ob = S.ctx.mult(*dc, 24, dk, new=new)
        ra, rb = ref(S.P, 24, *cts, key)
        np.testing.assert_array_equal(host(oa), ra)
        np.testing.assert_array_equal(host(ob), rb)


@pytest.mark.parametrize("n,ell", [(5, 7), (1, 4), (3, 2)])
def test_newmult_sum_parity(cfg_odd, n, ell):
    """Sum of n NewMult products with one merged ModDown against the oracle."""
    S = cfg_odd
    key = S.key(0, "gpu/nmsum/rlk")[0]
    pairs = [_pair(S, ell, f"gpu/nmsum/{n}/{ell}/{i}") for i in range(n)]
    c1 = [(dev(p[0]), dev(p[1])) for p in pairs]
    c2 = [(dev(p[2]), dev(p[3])) for p in pairs]
    oa, ob = S.ctx.newmult_sum(c1, c2, ell, dev(key))
    ra, rb = S.o.newmult_sum(S.P, ell, [(p[0], p[1]) for p in pairs], [(p[2], p[3]) for p in pairs], key)
    np.testing.assert_array_equal(host(oa), ra)
    np.testing.assert_array_equal(host(ob), rb)
