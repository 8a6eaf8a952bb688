"""The fused key-switching dataflow (ckks_fuse_select): ModUp's last forward
NTT pass, KSKInnerProd and ModDown's first inverse pass of the special limbs
in one kernel (Sec. 4.2 beta-limb caching, Sec. 4.4 re-ordering).  KeySwitch,
Rotate (Alg. 3) and HRotate (Alg. 4) through it must give the oracle's
residues bit for bit (tolerance 0) at every ring degree it serves, with
partial last digits, compressed keys, edge-value inputs and many calls
overlapping on streams."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

# (logN, L, k, dnum, bits): the single-KeySwitch configuration, a partial last
# digit (alpha = 3), beta = 4 digits, N = 2^15 and 2^17 with 54-bit primes
SHAPES = [(12, 6, 3, 2, 50), (11, 7, 3, 3, 50), (13, 8, 2, 4, 50), (15, 9, 3, 3, 54), (17, 4, 2, 2, 54),
          (10, 5, 2, 2, 50)]


@pytest.fixture(scope="module", params=SHAPES, ids=lambda s: "n%d_L%d_k%d_d%d_b%d" % s)
def S(request, oracle_lib):
    S = Setup(oracle_lib, *request.param)
    assert S.ctx.fuse_modup(True)
    yield S
    S.ctx.fuse_modup(False)


def test_keyswitch_rotate_hrotate_fused(S):
    P, ctx, o = S.P, S.ctx, S.o
    g = 5
    relin = S.key(0, "gpu/fused/relin")[0]
    rot = S.key(g, "gpu/fused/rot5")[0]
    for ell in sorted({P.L, P.L - 1, P.alpha + 1, 1}):
        if ell < 1:
            continue
        a, b = S.ct(ell, f"gpu/fused/ct{ell}")
        da, db = dev(a), dev(b)
        u, v = ctx.keyswitch(da, ell, dev(relin))
        ru, rv = o.keyswitch(P, ell, a, relin)
        np.testing.assert_array_equal(host(u), ru, err_msg=f"keyswitch u ell={ell}")
        np.testing.assert_array_equal(host(v), rv, err_msg=f"keyswitch v ell={ell}")
        ((ha, hb),) = ctx.hrotate(da, db, ell, [g], [dev(rot)])
        ((ra, rb),) = o.hrotate(P, ell, a, b, [g], [rot])
        np.testing.assert_array_equal(host(ha), ra, err_msg=f"hrotate a ell={ell}")
        np.testing.assert_array_equal(host(hb), rb, err_msg=f"hrotate b ell={ell}")
        oa, ob = ctx.rotate(da, db, ell, g, dev(rot))
        ra, rb = o.rotate(P, ell, a, b, g, rot)
        np.testing.assert_array_equal(host(oa), ra, err_msg=f"rotate a ell={ell}")
        np.testing.assert_array_equal(host(ob), rb, err_msg=f"rotate b ell={ell}")
    assert ctx.poll_status()


def test_fused_compressed_key(S):
    """A compressed key (rows b_j only, a_j regenerated from the seed inside the
    fused kernel) gives the bits of the same key stored in full."""
    P, ctx = S.P, S.ctx
    seed = 0x2112063960ABCDEF
    s = synth.ternary(P.N, "gpu/fused/comp/s")
    e = np.stack([synth.gaussian(P.N, f"gpu/fused/comp/e{j}") for j in range(P.dnum)])
    kb = ctx.keygen_ksk_seeded(dev(s), dev(e), seed, 5)
    full = ctx.ksk_expand(kb, seed)
    ctx.register_compressed_key(kb, seed)
    try:
        a, b = S.ct(P.L, "gpu/fused/comp/ct")
        da, db = dev(a), dev(b)
        ((ca, cb),) = ctx.hrotate(da, db, P.L, [5], [kb])
        ((fa, fb),) = ctx.hrotate(da, db, P.L, [5], [full])
        np.testing.assert_array_equal(host(ca), host(fa))
        np.testing.assert_array_equal(host(cb), host(fb))
    finally:
        ctx.unregister_compressed_key(kb)


@pytest.fixture(scope="module")
def B(oracle_lib):
    B = Setup(oracle_lib, 16, 24, 8, 3, 54)
    assert B.ctx.fuse_modup(True)
    yield B
    B.ctx.fuse_modup(False)


@pytest.mark.parametrize("r", [1, 1 << 14])
def test_fused_headline_hrotate(B, r):
    P, ctx = B.P, B.ctx
    g = pow(5, r, 2 * P.N)
    key = B.key(g, "gpu/fused/B/key%d" % r)[0]
    a, b = B.ct(P.L, "gpu/fused/B/ct")
    ((oa, ob),) = ctx.hrotate(dev(a), dev(b), P.L, [g], [dev(key)])
    ((ra, rb),) = B.o.hrotate(P, P.L, a, b, [g], [key])
    np.testing.assert_array_equal(host(oa), ra)
    np.testing.assert_array_equal(host(ob), rb)


def test_fused_headline_edges_both_conversions(B):
    """Maximal scaled sources and all-0 / all-(q-1) / spike limbs (see
    test_gpu_edge_headline) through the fused KeySwitch on both conversion paths."""
    from tests.test_gpu_edge_headline import _both, _digits, _eval_edges, _scaled_source_input

    P, ctx, o = B.P, B.ctx, B.o
    ell = P.L
    chain = P.primes[:ell]
    key = B.key(0, "gpu/fused/B/relin")[0]
    dk = dev(key)
    for a in (_scaled_source_input(o, P.logN, chain, [(g, {i: 0 for i in range(ell)}) for g in _digits(P, ell)],
                                   "max"), _eval_edges(chain, P.N)):
        da = dev(a)
        tc, sp = _both(ctx, lambda: [host(t) for t in ctx.keyswitch(da, ell, dk)])
        ru, rv = o.keyswitch(P, ell, a, key)
        for got in (tc, sp):
            np.testing.assert_array_equal(got[0], ru)
            np.testing.assert_array_equal(got[1], rv)


def test_fused_concurrent_streams_equal_one_at_a_time():
    """Sixteen fused HRotates on 8 streams, repeated, equal the same HRotates run
    one at a time (tolerance 0)."""
    import bench
    from paper_2112_06396_gb300 import ckks

    L = bench.L
    primes = ckks.ckks_gen_primes(bench.BITS, bench.LOGN, L + bench.K_SP)
    ctx = ckks.Context(bench.LOGN, primes[:L], primes[L:], bench.DNUM)
    assert ctx.fuse_modup(True)
    items = bench.make_workload(ctx, 16, 0, torch)
    one = bench.Lanes(ctx, 1, torch, ckks)
    ref = []
    for it in items:
        ctx.hrotate(it["a"], it["b"], L, [it["g"]], [it["key"]], outs=[(it["oa"], it["ob"])], ws=one.ws[0])
        torch.cuda.synchronize()
        ref.append((it["oa"].clone(), it["ob"].clone()))
    ctx.fuse_modup(False)
    for c, it in enumerate(items):  # the unfused path gives the same bits
        ctx.hrotate(it["a"], it["b"], L, [it["g"]], [it["key"]], outs=[(it["oa"], it["ob"])], ws=one.ws[0])
        torch.cuda.synchronize()
        assert torch.equal(it["oa"], ref[c][0]) and torch.equal(it["ob"], ref[c][1]), c
    ctx.fuse_modup(True)
    lanes = bench.Lanes(ctx, bench.STREAMS, torch, ckks)
    bad = []
    for s in range(8):
        for it in items:
            it["oa"].zero_()
            it["ob"].zero_()
        bench.step(ctx, items, lanes)
        torch.cuda.synchronize()
        bad += [(s, c) for c, it in enumerate(items)
                if not (torch.equal(it["oa"], ref[c][0]) and torch.equal(it["ob"], ref[c][1]))]
    assert not bad, bad[:10]
    assert ctx.poll_status()
