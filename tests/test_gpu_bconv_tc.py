"""The two paths of the fast basis conversion (Algorithm 6 and the table "CKKS
Subroutines"): on the tensor cores (tcgen05 f16 MMA on byte pieces of the
residues, exact f32 sums, one reduction per output) and on the integer units
(32-bit split multiply-adds).  Both must give the oracle's residues bit for bit
(tolerance 0) in every operation that converts: ModUp, ModDown, Rescale, the
merged ModDown of NewMult and the batched KeySwitch."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (logN, L, k, dnum, bits): tensor-core K groups 6, 6, 8 (54-bit primes, the
# widest of the integer path too), 18 (alpha = 16 sources, the largest
# supported), 16 with more than 32 targets (alpha = 14: ModUp converts to up to
# 34 limbs and ModDown to 40, in two chunks of uneven size), and N = 2^10
# (8 tiles of 128 coefficients, fewer than the CTAs a launch could use), and the
# longest chain (L = 64) with alpha = 16 sources: conversions to 56 and 64 limbs
SHAPES = [(12, 6, 3, 2, 50), (11, 7, 3, 3, 50), (11, 10, 5, 2, 54), (11, 32, 8, 2, 50), (11, 40, 8, 3, 50),
          (10, 5, 2, 2, 50), (10, 64, 8, 4, 50)]


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "n%d_L%d_k%d_d%d_b%d" % s)
def S(request, oracle_lib):
    return Setup(oracle_lib, *request.param)


def _both(ctx, fn):
    """fn() on the tensor cores, then on the integer units (host copies)."""
    try:
        assert ctx.bconv_tensor_cores(True)
        a = fn()
        ctx.bconv_tensor_cores(False)
        b = fn()
    finally:
        ctx.bconv_tensor_cores(True)
    return a, b


def _h(x):
    return [host(t) for t in x] if isinstance(x, (tuple, list)) else host(x)


def test_modup_moddown_rescale(S):
    P, ctx = S.P, S.ctx
    for ell in sorted({P.L, P.L - 1, P.alpha + 1, 2}):
        a = synth.uniform_residues(P.primes[:ell], P.N, f"gpu/tc/modup/{ell}")
        da = dev(a)
        for j in range(P.beta(ell)):
            tc, sp = _both(ctx, lambda: host(ctx.modup(da, ell, j)))
            np.testing.assert_array_equal(tc, sp, err_msg=f"modup ell={ell} j={j}")
            np.testing.assert_array_equal(tc, S.o.modup(P, ell, j, a), err_msg=f"modup ell={ell} j={j}")
        x = synth.uniform_residues(P.ext_primes(ell), P.N, f"gpu/tc/moddown/{ell}")
        dx = dev(x)
        tc, sp = _both(ctx, lambda: host(ctx.moddown(dx, ell)))
        np.testing.assert_array_equal(tc, sp, err_msg=f"moddown ell={ell}")
        np.testing.assert_array_equal(tc, S.o.moddown(P, ell, x), err_msg=f"moddown ell={ell}")
        y = synth.uniform_residues(P.primes[:ell], P.N, f"gpu/tc/rescale/{ell}")
        dy = dev(y)
        tc, sp = _both(ctx, lambda: host(ctx.rescale(dy, ell)))
        np.testing.assert_array_equal(tc, sp, err_msg=f"rescale ell={ell}")
        np.testing.assert_array_equal(tc, S.o.rescale(P, ell, y), err_msg=f"rescale ell={ell}")
    assert ctx.poll_status()


def test_newmult_merged_moddown(S):
    P, ctx = S.P, S.ctx
    key = S.key(0, "gpu/tc/relin")[0]
    dkey = dev(key)
    ell = P.L
    a1, b1 = S.ct(ell, "gpu/tc/m1")
    a2, b2 = S.ct(ell, "gpu/tc/m2")
    d = [dev(v) for v in (a1, b1, a2, b2)]
    tc, sp = _both(ctx, lambda: _h(ctx.mult(*d, ell, dkey, new=True)))
    ra, rb = S.o.newmult(P, ell, a1, b1, a2, b2, key)
    for got in (tc, sp):
        np.testing.assert_array_equal(got[0], ra)
        np.testing.assert_array_equal(got[1], rb)


def test_batched_keyswitch(S):
    P, ctx = S.P, S.ctx
    key = S.key(0, "gpu/tc/bks")[0]
    dkey = dev(key)
    levels = synth.uniform_ints(6, 1, P.L, f"gpu/tc/bks/{P.logN}/{P.L}")
    a = [S.ct(ell, f"gpu/tc/bks/{i}")[0] for i, ell in enumerate(levels)]
    da = [dev(x) for x in a]
    tc, sp = _both(ctx, lambda: [_h(o) for o in ctx.keyswitch_batch(da, None, levels, None, [dkey] * len(levels))])
    for i, ell in enumerate(levels):
        np.testing.assert_array_equal(tc[i][0], sp[i][0], err_msg=f"entry {i}")
        np.testing.assert_array_equal(tc[i][1], sp[i][1], err_msg=f"entry {i}")
    i = levels.index(max(levels))
    ru, rv = S.o.keyswitch(P, levels[i], a[i], key)
    np.testing.assert_array_equal(tc[i][0], ru)
    np.testing.assert_array_equal(tc[i][1], rv)


def test_availability(oracle_lib):
    ckks = _gpu()
    wide = oracle_lib.gen_primes(58, 11, 6)
    ctx = ckks.Context(11, wide[:4], wide[4:], 2)
    assert not ctx.bconv_tensor_cores(True)  # 58-bit primes: integer path only
    many = oracle_lib.gen_primes(50, 11, 40)
    ctx = ckks.Context(11, many[:34], many[34:], 2)
    assert not ctx.bconv_tensor_cores(True)  # alpha = 17 sources


@pytest.fixture(scope="module")
def cfgB(oracle_lib):
    return Setup(oracle_lib, 16, 24, 8, 3, 54)


@pytest.mark.parametrize("r", [1, 2, 1 << 14])
def test_headline_shape(cfgB, r):
    """HRotate by 5^r (r = 1, 2 and 2^14, the largest rotation of N/2 slots)
    at N=2^16, ell=24, k=8, dnum=3: both conversion paths equal the oracle."""
    S = cfgB
    P, ctx = S.P, S.ctx
    g = pow(5, r, 2 << 16)
    key = S.key(g, "gpu/tc/B/key%d" % r)[0]
    a, b = S.ct(P.L, "gpu/tc/B/ct")
    da, db, dk = dev(a), dev(b), dev(key)
    tc, sp = _both(ctx, lambda: _h(ctx.hrotate(da, db, P.L, [g], [dk])[0]))
    np.testing.assert_array_equal(tc[0], sp[0])
    np.testing.assert_array_equal(tc[1], sp[1])
    (ra, rb), = S.o.hrotate(P, P.L, a, b, [g], [key])
    np.testing.assert_array_equal(tc[0], ra)
    np.testing.assert_array_equal(tc[1], rb)
    assert ctx.poll_status()


@pytest.mark.parametrize("hint", [8, 64])
def test_concurrency_hint_headline(cfgB, hint):
    """ckks_concurrency_hint sizes the tensor-core conversion for a 1/hint share
    of the SMs (hint 64: one or two CTAs per group walking all 512 tiles): an
    HRotate, a ModUp of every digit and a ModDown at N=2^16, ell=24 equal the
    oracle, and a batch of four KeySwitches equals the same batch at hint 1."""
    S = cfgB
    P, ctx = S.P, S.ctx
    g = 5
    key = S.key(g, "gpu/tc/B/key1")[0]
    a, b = S.ct(P.L, "gpu/tc/B/ct")
    da, db, dk = dev(a), dev(b), dev(key)
    levels = [24, 9, 17, 24]
    xs = [dev(S.ct(ell, f"gpu/tc/B/hint/{i}")[0]) for i, ell in enumerate(levels)]
    ref = [_h(o) for o in ctx.keyswitch_batch(xs, None, levels, None, [dk] * 4)]
    x = dev(S.ct(P.L, "gpu/tc/B/hint/x")[0])
    ctx.concurrency_hint(hint)
    try:
        oa, ob = _h(ctx.hrotate(da, db, P.L, [g], [dk])[0])
        (ra, rb), = S.o.hrotate(P, P.L, a, b, [g], [key])
        np.testing.assert_array_equal(oa, ra)
        np.testing.assert_array_equal(ob, rb)
        for j in range(P.beta(P.L)):
            np.testing.assert_array_equal(host(ctx.modup(da, P.L, j)), S.o.modup(P, P.L, j, a))
        ext = synth.uniform_residues(P.ext_primes(P.L), P.N, "gpu/tc/B/hint/ext")
        np.testing.assert_array_equal(host(ctx.moddown(dev(ext), P.L)), S.o.moddown(P, P.L, ext))
        got = [_h(o) for o in ctx.keyswitch_batch(xs, None, levels, None, [dk] * 4)]
        for (ga, gb), (wa, wb) in zip(got, ref):
            np.testing.assert_array_equal(ga, wa)
            np.testing.assert_array_equal(gb, wb)
        assert ctx.poll_status()
    finally:
        ctx.concurrency_hint(1)


@pytest.fixture(scope="module")
def cfg1(oracle_lib):
    return Setup(oracle_lib, 12, 6, 3, 2, 50)


def test_bounded_wait_runs_out_and_is_reported(cfg1):
    """The device-side wait of the tensor-core conversion is bounded: the
    self-test waits on a barrier nothing arrives on, gives up after 20 ms and
    records it; ckks_poll_status reports CKKS_ETIMEOUT once, and the context
    keeps working (a KeySwitch afterwards still equals the oracle)."""
    import time

    ckks = _gpu()
    S = cfg1
    P, ctx = S.P, S.ctx
    assert ctx.poll_status()
    t0 = time.perf_counter()
    ctx.selftest_bounded_wait(20000)
    torch.cuda.synchronize()
    waited = time.perf_counter() - t0
    assert 0.015 < waited < 5.0
    with pytest.raises(ckks.CkksError) as err:
        ctx.poll_status()
    assert err.value.code == ckks.CKKS_ETIMEOUT
    assert ctx.poll_status()  # reported once, then cleared
    with pytest.raises(ckks.CkksError):
        ctx.selftest_bounded_wait(0)
    key = S.key(0, "gpu/tc/after-timeout")[0]
    a, _ = S.ct(P.L, "gpu/tc/after-timeout/ct")
    u, v = ctx.keyswitch(dev(a), P.L, dev(key))
    ru, rv = S.o.keyswitch(P, P.L, a, key)
    np.testing.assert_array_equal(host(u), ru)
    np.testing.assert_array_equal(host(v), rv)
