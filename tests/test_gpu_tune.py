"""The NTT autotuner: every tile shape it can pick gives the same bits (the
transform is the same arithmetic in another CTA shape), and tuning keeps one
of the timed shapes per pass and launch size."""
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
    for choice in itertools.product(range(3), repeat=4):
        S.ctx.tune_set(list(choice))
        (oa, ob), = S.ctx.hrotate(da, db, P.L, [g], [dk])
        np.testing.assert_array_equal(host(oa), ra, err_msg=f"shape {choice}")
        np.testing.assert_array_equal(host(ob), rb, err_msg=f"shape {choice}")
        d = dev(x)
        S.ctx.ntt(d, P.L)
        for t in range(P.L):
            np.testing.assert_array_equal(host(d)[t], S.o.ntt(x[t], P.logN, int(P.primes[t])))
    S.ctx.tune_set([0, 0, 0, 0])


def test_autotune_picks_a_timed_shape(cfg14):
    ckks = _gpu()
    choice, times = cfg14.ctx.autotune(limbs=64)
    assert len(choice) == 4 and all(0 <= c <= 2 for c in choice)
    for i, c in enumerate(choice):
        row = times[i * 3:(i + 1) * 3]
        assert all(t > 0 for t in row)
        assert row[c] == min(row)
    with pytest.raises(ckks.CkksError):
        cfg14.ctx.tune_set([0, 3, 0, 0])
    cfg14.ctx.tune_set([0, 0, 0, 0])


def test_autotune_cache_round_trip(cfg14, tmp_path):
    cache = str(tmp_path / "tune.json")
    ch1, _ = cfg14.ctx.autotune(limbs=32, cache=cache)
    cfg14.ctx.tune_set([0, 0, 0, 0])
    ch2, _ = cfg14.ctx.autotune(limbs=32, cache=cache)  # from the cache, no timing
    assert ch1 == ch2
    cfg14.ctx.tune_set([0, 0, 0, 0])


def test_poll_status_and_allocation_failure(cfg14):
    ckks = _gpu()
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    assert cfg14.ctx.poll_status(st) is True
    # a budget no GPU has: the server's arena allocation fails cleanly
    with pytest.raises(ckks.CkksError):
        ckks.Server([cfg14.ctx], 1 << 50, max_batch=4, streams=1)
    assert cfg14.ctx.poll_status(st) is True  # the context is still usable
