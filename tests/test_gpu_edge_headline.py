"""Edge-value inputs through ModUp, ModDown, KeySwitch and HRotate at the
headline shape (N=2^16, ell=24, k=8, dnum=3, 54-bit primes), on both basis
conversion paths (tensor cores and integer units), against the oracle bit for
bit (tolerance 0).

The GPU path's lazy arithmetic is tightest here, with the widest primes:
  * the tensor-core conversion sums byte products y_ij * m_tijc, largest when
    every byte of the scaled source y_i = [x_i (Q_j/q_i)^-1]_{q_i} is 0xFF
    (Algorithm 6, step 2; the ModDown conversion of Sec. 2.4 likewise);
  * with primes this large its outputs go unreduced (below 8t) into the lazy
    forward NTT, whose values then grow towards 76p;
  * all-0, all-(q-1) and single-spike limbs are the transforms' extremes.
The inputs are built so that these cases occur: in coefficient form, every
scaled source of every digit equal to the largest residue whose low 48 bits
are all ones (or q-1, or 0 at every other coefficient), then transformed to
evaluation form by the oracle's NTT.
"""
import numpy as np
import pytest

from tests.test_gpu_parity import Setup, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _both(ctx, fn):
    """fn() on the tensor cores, then on the integer units."""
    try:
        assert ctx.bconv_tensor_cores(True)
        a = fn()
        ctx.bconv_tensor_cores(False)
        b = fn()
    finally:
        ctx.bconv_tensor_cores(True)
    return a, b


@pytest.fixture(scope="module")
def B(oracle_lib):
    return Setup(oracle_lib, 16, 24, 8, 3, 54)


def _all_ones_low48(q):
    """The largest residue below q whose low 48 bits are all set."""
    v = ((q >> 48) << 48) - 1
    assert 0 < v < q and (v & ((1 << 48) - 1)) == (1 << 48) - 1
    return v


def _scaled_source_input(o, logN, primes, groups, pattern):
    """Evaluation-form limbs whose coefficient form x_i makes every scaled source
    y_i = [x_i * (Q_g / q_i)^-1]_{q_i} take `pattern`, where Q_g is the product of
    the primes of the group holding limb i (a ModUp digit, or the special primes
    for ModDown, with `offset` = [H]_{q_i} to undo the rounding addend)."""
    N = 1 << logN
    primes = [int(q) for q in primes]
    out = np.zeros((len(primes), N), dtype=np.uint64)
    for g, offset in groups:
        Qg = 1
        for i in g:
            Qg *= primes[i]
        for i in g:
            q = primes[i]
            qhat = (Qg // q) % q
            x = np.empty(N, dtype=np.uint64)
            if pattern == "max":
                x[:] = (_all_ones_low48(q) * qhat - offset[i]) % q
            elif pattern == "qm1":
                x[:] = ((q - 1) * qhat - offset[i]) % q
            else:  # "alternate": max at even coefficients, 0 at odd ones
                x[0::2] = (_all_ones_low48(q) * qhat - offset[i]) % q
                x[1::2] = (-offset[i]) % q
            out[i] = o.ntt(x, logN, q)
    return out


def _eval_edges(primes, N):
    """Limb t: all 0 (t % 3 == 0), all q-1 (t % 3 == 1), or q-1 at one coefficient (t % 3 == 2)."""
    x = np.zeros((len(primes), N), dtype=np.uint64)
    for t, q in enumerate(primes):
        if t % 3 == 1:
            x[t][:] = int(q) - 1
        elif t % 3 == 2:
            x[t][(977 * t) % N] = int(q) - 1
    return x


def _digits(P, ell):
    return [list(range(j * P.alpha, min((j + 1) * P.alpha, ell))) for j in range(P.beta(ell))]


@pytest.mark.parametrize("pattern", ["max", "qm1", "alternate", "eval_edges"])
def test_modup_moddown_edges_headline(B, pattern):
    P, ctx, o = B.P, B.ctx, B.o
    ell = P.L
    chain = P.primes[:ell]
    zero = {i: 0 for i in range(ell + P.k)}
    if pattern == "eval_edges":
        a = _eval_edges(chain, P.N)
    else:
        a = _scaled_source_input(o, P.logN, chain, [(g, zero) for g in _digits(P, ell)], pattern)
    da = dev(a)
    for j in range(P.beta(ell)):
        tc, sp = _both(ctx, lambda: host(ctx.modup(da, ell, j)))
        want = o.modup(P, ell, j, a)
        np.testing.assert_array_equal(tc, want, err_msg=f"modup tensor cores, digit {j}")
        np.testing.assert_array_equal(sp, want, err_msg=f"modup integer units, digit {j}")
    ext = P.ext_primes(ell)
    if pattern == "eval_edges":
        x = _eval_edges(ext, P.N)
    else:
        # the special limbs carry the extreme scaled sources (after the +H of
        # the rounding), the chain limbs the pattern's own residues
        Pprod = 1
        for p in ext[ell:]:
            Pprod *= int(p)
        H = Pprod // 2
        offs = {i: H % int(ext[i]) for i in range(len(ext))}
        x = _scaled_source_input(o, P.logN, ext, [(list(range(ell, ell + P.k)), offs)], pattern)
        x[:ell] = _scaled_source_input(o, P.logN, ext, [(list(range(ell)), zero)], pattern)[:ell]
    dx = dev(x)
    tc, sp = _both(ctx, lambda: host(ctx.moddown(dx, ell)))
    want = o.moddown(P, ell, x)
    np.testing.assert_array_equal(tc, want, err_msg="moddown tensor cores")
    np.testing.assert_array_equal(sp, want, err_msg="moddown integer units")


@pytest.mark.parametrize("pattern", ["max", "eval_edges"])
def test_keyswitch_hrotate_edges_headline(B, pattern):
    P, ctx, o = B.P, B.ctx, B.o
    ell = P.L
    chain = P.primes[:ell]
    if pattern == "eval_edges":
        a = _eval_edges(chain, P.N)
    else:
        a = _scaled_source_input(o, P.logN, chain, [(g, {i: 0 for i in range(ell)}) for g in _digits(P, ell)],
                                 pattern)
    b = _eval_edges(chain, P.N)[::-1].copy()
    key = B.key(5, "gpu/edge/B/key5")[0]
    da, db, dk = dev(a), dev(b), dev(key)
    tc, sp = _both(ctx, lambda: [host(t) for t in ctx.keyswitch(da, ell, dk)])
    ru, rv = o.keyswitch(P, ell, a, key)
    for got, path in ((tc, "tensor cores"), (sp, "integer units")):
        np.testing.assert_array_equal(got[0], ru, err_msg=f"keyswitch u, {path}")
        np.testing.assert_array_equal(got[1], rv, err_msg=f"keyswitch v, {path}")
    tc, sp = _both(ctx, lambda: [host(t) for t in ctx.hrotate(da, db, ell, [5], [dk])[0]])
    ((ra, rb),) = o.hrotate(P, ell, a, b, [5], [key])
    for got, path in ((tc, "tensor cores"), (sp, "integer units")):
        np.testing.assert_array_equal(got[0], ra, err_msg=f"hrotate a, {path}")
        np.testing.assert_array_equal(got[1], rb, err_msg=f"hrotate b, {path}")
    assert ctx.poll_status()
