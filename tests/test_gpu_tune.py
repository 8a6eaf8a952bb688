"""The NTT autotuner: every tile shape and radix split it can pick gives the
same bits (the transform is the same arithmetic in another CTA shape, or with
one stage moved between the two passes), and tuning keeps one of the timed
shapes per pass and launch size and one of the timed splits per direction and
launch size."""
import itertools

import numpy as np
import pytest

from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg14(oracle_lib):
    return Setup(oracle_lib, 14, 6, 3, 3, 54)


def test_every_tile_shape_gives_the_oracle_bits(cfg14):
    S = cfg14
    P = S.P
    g = 5
    key = S.key(g, "gpu/tune/key")[0]
    a, b = S.ct(P.L, "gpu/tune/ct")
    (ra, rb), = S.o.hrotate(P, P.L, a, b, [g], [key])
    da, db, dk = dev(a), dev(b), dev(key)
    x = S.ct(P.L, "gpu/tune/ntt")[0]
    want = np.stack([S.o.ntt(x[t], P.logN, int(P.primes[t])) for t in range(P.L)])
    shapes = [list(c) + [0, 0, 0, 0] for c in itertools.product(range(3), repeat=4)]
    splits = [[0, 0, 0, 0, f, f, i, i] for f, i in itertools.product((-1, 0, 1), repeat=2)]
    for choice in shapes + splits:
        S.ctx.tune_set(choice)
        (oa, ob), = S.ctx.hrotate(da, db, P.L, [g], [dk])
        np.testing.assert_array_equal(host(oa), ra, err_msg=f"shape {choice}")
        np.testing.assert_array_equal(host(ob), rb, err_msg=f"shape {choice}")
        d = dev(x)
        S.ctx.ntt(d, P.L)
        np.testing.assert_array_equal(host(d), want, err_msg=f"shape {choice}")
        S.ctx.intt(d, P.L)
        np.testing.assert_array_equal(host(d), x, err_msg=f"shape {choice}")
    S.ctx.tune_set([0] * 8)


@pytest.mark.parametrize("split", [[-1, -1, -1, -1], [1, 1, 1, 1], [-1, 1, 1, -1]])
def test_radix_splits_headline(oracle_lib, split):
    """N=2^16, ell=24, k=8, dnum=3, 54-bit primes: an HRotate (whose ModUp
    transforms 72 limbs in one launch, the large size class) equals the oracle
    with each radix split, and a batch of four KeySwitches (inverse transforms
    of 79 limbs) equals the same batch with the default split."""
    S = Setup(oracle_lib, 16, 24, 8, 3, 54)
    P, ctx = S.P, S.ctx
    g = 5
    key = S.key(g, "gpu/tune/B/key")[0]
    a, b = S.ct(P.L, "gpu/tune/B/ct")
    (ra, rb), = S.o.hrotate(P, P.L, a, b, [g], [key])
    da, db, dk = dev(a), dev(b), dev(key)
    levels = [24, 7, 24, 24]
    xs = [dev(S.ct(ell, f"gpu/tune/B/b{i}")[0]) for i, ell in enumerate(levels)]
    ctx.tune_set([0] * 8)
    ref = ctx.keyswitch_batch(xs, None, levels, None, [dk] * 4)
    ctx.tune_set([0, 0, 0, 0] + split)
    try:
        (oa, ob), = ctx.hrotate(da, db, P.L, [g], [dk])
        np.testing.assert_array_equal(host(oa), ra)
        np.testing.assert_array_equal(host(ob), rb)
        got = ctx.keyswitch_batch(xs, None, levels, None, [dk] * 4)
        for (ga, gb), (wa, wb) in zip(got, ref):
            assert torch.equal(ga, wa) and torch.equal(gb, wb)
        x = a[:3]
        d = dev(x)
        ctx.ntt(d, 3)
        for t in range(3):
            np.testing.assert_array_equal(host(d)[t], S.o.ntt(x[t], P.logN, int(P.primes[t])))
        assert ctx.poll_status()
    finally:
        ctx.tune_set([0] * 8)


def test_autotune_picks_a_timed_shape(cfg14):
    ckks = _gpu()
    choice, times = cfg14.ctx.autotune(limbs=64)
    assert len(choice) == 8 and len(times) == 24
    assert all(0 <= c <= 2 for c in choice[:4]) and all(-1 <= c <= 1 for c in choice[4:])
    # the fastest shape, unless it beats the default by less than the tuner's
    # margin (0.5% for a width, 3% for a split); times are in the order
    # [default, half, double] and [split -1, 0, +1]
    for i, c in enumerate(choice[:4]):
        row = times[i * 3:(i + 1) * 3]
        assert all(t > 0 for t in row)
        fastest = min(range(3), key=lambda o: row[o])
        assert c == (fastest if row[fastest] < row[0] * 0.995 else 0)
    for i, c in enumerate(choice[4:]):
        row = times[12 + i * 3:12 + (i + 1) * 3]
        assert all(t > 0 for t in row)
        fastest = min(range(3), key=lambda o: row[o])
        assert c + 1 == (fastest if row[fastest] < row[1] * 0.97 else 1)
    with pytest.raises(ckks.CkksError):
        cfg14.ctx.tune_set([0, 3, 0, 0, 0, 0, 0, 0])
    with pytest.raises(ckks.CkksError):
        cfg14.ctx.tune_set([0, 0, 0, 0, 0, 2, 0, 0])
    with pytest.raises(ckks.CkksError):
        cfg14.ctx.tune_set([0, 0, 0, 0])
    cfg14.ctx.tune_set([0] * 8)


def test_autotune_cache_round_trip(cfg14, tmp_path):
    cache = str(tmp_path / "tune.json")
    ch1, _ = cfg14.ctx.autotune(limbs=32, cache=cache)
    cfg14.ctx.tune_set([0] * 8)
    ch2, _ = cfg14.ctx.autotune(limbs=32, cache=cache)  # from the cache, no timing
    assert ch1 == ch2
    cfg14.ctx.tune_set([0] * 8)


def test_poll_status_and_allocation_failure(cfg14):
    ckks = _gpu()
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert cfg14.ctx.poll_status(st) is True
    # a budget no GPU has: the server's arena allocation fails cleanly
    with pytest.raises(ckks.CkksError):
        ckks.Server([cfg14.ctx], 1 << 50, max_batch=4, streams=1)
    assert cfg14.ctx.poll_status(st) is True  # the context is still usable
