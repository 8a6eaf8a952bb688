"""Parity of the CUDA path (through the C ABI) with the CPU oracle.

Exact modular arithmetic: every comparison is bit-exact (tolerance 0).
Sizes: the single-KeySwitch configuration (N=2^12, ell=6, k=3, dnum=2, 50-bit
primes), extra shapes with partial last digits, every supported ring degree
for the transforms, and the headline shape (N=2^16, ell=24, k=8, dnum=3,
54-bit primes) for HRotate.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06396_gb300 import ckks

    return ckks


def dev(x):
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def host(t):
    torch.cuda.synchronize()
    return t.cpu().numpy()


class Setup:
    def __init__(self, oracle_lib, logN, L, k, dnum, bits):
        ckks = _gpu()
        primes = oracle_lib.gen_primes(bits, logN, L + k)
        self.P = oracle_lib.Params(logN, L, k, dnum, primes=primes)
        self.ctx = ckks.Context(logN, primes[:L], primes[L:], dnum)
        assert self.ctx.q + self.ctx.p == primes
        self.o = oracle_lib
        self.s = synth.ternary(self.P.N, f"gpu/{logN}/s")

    def key(self, g, tag):
        P, o = self.P, self.o
        a = np.stack([synth.uniform_residues(P.primes, P.N, f"{tag}/a{j}") for j in range(P.dnum)])
        e = np.stack([synth.gaussian(P.N, f"{tag}/e{j}") for j in range(P.dnum)])
        sp = o.sq_secret(P, self.s) if g == 0 else o.rot_secret(P, self.s, g)
        return o.keygen(P, a, self.s, sp, e), a, e

    def ct(self, ell, tag):
        P = self.P
        a = synth.uniform_residues(P.primes[:ell], P.N, f"{tag}/a")
        b = synth.uniform_residues(P.primes[:ell], P.N, f"{tag}/b")
        return a, b


@pytest.fixture(scope="module")
def cfg1(oracle_lib):
    return Setup(oracle_lib, 12, 6, 3, 2, 50)


@pytest.fixture(scope="module")
def cfg_odd(oracle_lib):
    # alpha = 3 with a partial last digit at most levels
    return Setup(oracle_lib, 11, 7, 3, 3, 50)


# ------------------------------------------------------------------ transforms
@pytest.mark.parametrize("logN", [10, 11, 12, 13, 14, 15, 16, 17])
def test_ntt_intt_parity_all_sizes(oracle_lib, logN):
    ckks = _gpu()
    L, k = 3, 2
    primes = oracle_lib.gen_primes(54 if logN >= 15 else 50, logN, L + k)
    ctx = ckks.Context(logN, primes[:L], primes[L:], 1)
    ell = 2
    ext = primes[:ell] + primes[L:]
    x = synth.uniform_residues(ext, 1 << logN, f"gpu/ntt/{logN}")
    d = dev(x)
    ctx.ntt(d, ell)
    got = host(d)
    for t, q in enumerate(ext):
        np.testing.assert_array_equal(got[t], oracle_lib.ntt(x[t], logN, q))
    ctx.intt(d, ell)
    np.testing.assert_array_equal(host(d), x)
    # inverse on its own against the oracle's inverse
    d2 = dev(x)
    ctx.intt(d2, ell, 1, 2)
    got2 = host(d2)
    np.testing.assert_array_equal(got2[0], x[0])
    for t in (1, 2):
        np.testing.assert_array_equal(got2[t], oracle_lib.intt(x[t], logN, ext[t]))


def test_ntt_edge_values(cfg1):
    """All-zero, all q-1 and single-spike limbs."""
    P = cfg1.P
    ell = 2
    ext = cfg1.P.ext_primes(ell)
    x = np.zeros((ell + P.k, P.N), dtype=np.uint64)
    for t, q in enumerate(ext):
        if t % 3 == 1:
            x[t][:] = q - 1
        elif t % 3 == 2:
            x[t][P.N - 1] = q - 1
    d = dev(x)
    cfg1.ctx.ntt(d, ell)
    got = host(d)
    for t, q in enumerate(ext):
        np.testing.assert_array_equal(got[t], cfg1.o.ntt(x[t], P.logN, q))


@pytest.mark.parametrize("g_exp", [1, 5, 1000, -1])
def test_automorph_parity(cfg1, g_exp):
    P = cfg1.P
    twoN = 2 * P.N
    g = twoN - 1 if g_exp == -1 else pow(5, g_exp, twoN)
    x = synth.uniform_residues(P.primes[:4], P.N, "gpu/auto")
    got = host(cfg1.ctx.automorph(dev(x), g))
    np.testing.assert_array_equal(got, cfg1.o.automorph_eval(x, P.logN, g))


# ------------------------------------------------------------------ basis conversion
@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_modup_parity(request, which):
    S = request.getfixturevalue(which)
    P = S.P
    for ell in sorted({P.L, P.L - 1, 1, P.alpha + 1}):
        if ell < 1:
            continue
        a = synth.uniform_residues(P.primes[:ell], P.N, f"gpu/modup/{ell}")
        da = dev(a)
        for j in range(P.beta(ell)):
            got = host(S.ctx.modup(da, ell, j))
            np.testing.assert_array_equal(got, S.o.modup(P, ell, j, a), err_msg=f"ell={ell} j={j}")


@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_moddown_and_pmodup_parity(request, which):
    S = request.getfixturevalue(which)
    P = S.P
    for ell in sorted({P.L, 2, 1}):
        x = synth.uniform_residues(P.ext_primes(ell), P.N, f"gpu/moddown/{ell}")
        got = host(S.ctx.moddown(dev(x), ell))
        np.testing.assert_array_equal(got, S.o.moddown(P, ell, x))
        y = x[:ell].copy()
        np.testing.assert_array_equal(host(S.ctx.pmodup(dev(y), ell)), S.o.pmodup(P, ell, y))


def test_rescale_parity(cfg1):
    P = cfg1.P
    for ell in range(2, P.L + 1):
        x = synth.uniform_residues(P.primes[:ell], P.N, f"gpu/rescale/{ell}")
        got = host(cfg1.ctx.rescale(dev(x), ell))
        np.testing.assert_array_equal(got, cfg1.o.rescale(P, ell, x))


def test_inner_prod_parity(cfg1):
    P = cfg1.P
    ell = P.L - 1
    key, _, _ = cfg1.key(5, "gpu/inner/key")
    digits = np.stack([cfg1.o.modup(P, ell, j, synth.uniform_residues(P.primes[:ell], P.N, "gpu/inner/a"))
                       for j in range(P.beta(ell))])
    u, v = cfg1.ctx.ksk_inner_prod(dev(digits), ell, dev(key))
    ou, ov = cfg1.o.ksk_inner_prod(P, ell, digits, key)
    np.testing.assert_array_equal(host(u), ou)
    np.testing.assert_array_equal(host(v), ov)


# ------------------------------------------------------------------ composed operations
@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_keyswitch_parity(request, which):
    S = request.getfixturevalue(which)
    P = S.P
    key, _, _ = S.key(0, f"gpu/ks/{which}")
    dkey = dev(key)
    for ell in sorted({P.L, P.alpha, 1}):
        a, _ = S.ct(ell, f"gpu/ks/{ell}")
        u, v = S.ctx.keyswitch(dev(a), ell, dkey)
        ou, ov = S.o.keyswitch(P, ell, a, key)
        np.testing.assert_array_equal(host(u), ou, err_msg=f"ell={ell}")
        np.testing.assert_array_equal(host(v), ov, err_msg=f"ell={ell}")


def test_rotate_parity(cfg1):
    P = cfg1.P
    g = pow(5, 3, 2 * P.N)
    key, _, _ = cfg1.key(g, "gpu/rot/key")
    ell = P.L
    a, b = cfg1.ct(ell, "gpu/rot/ct")
    oa, ob = cfg1.ctx.rotate(dev(a), dev(b), ell, g, dev(key))
    ra, rb = cfg1.o.rotate(P, ell, a, b, g, key)
    np.testing.assert_array_equal(host(oa), ra)
    np.testing.assert_array_equal(host(ob), rb)


@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_hrotate_parity(request, which):
    S = request.getfixturevalue(which)
    P = S.P
    twoN = 2 * P.N
    gs = [pow(5, 1, twoN), pow(5, 17, twoN), twoN - 1]
    keys = [S.key(g, f"gpu/hr/{which}/{g}")[0] for g in gs]
    ell = P.L - 1
    a, b = S.ct(ell, f"gpu/hr/{which}")
    outs = S.ctx.hrotate(dev(a), dev(b), ell, gs, [dev(k) for k in keys])
    ref = S.o.hrotate(P, ell, a, b, gs, keys)
    for (ga, gb), (ra, rb) in zip(outs, ref):
        np.testing.assert_array_equal(host(ga), ra)
        np.testing.assert_array_equal(host(gb), rb)


@pytest.mark.parametrize("nb,ng,rescale", [(3, 2, True), (4, 1, False), (1, 2, True)])
def test_ptmatvec_parity(cfg1, nb, ng, rescale):
    P = cfg1.P
    twoN = 2 * P.N
    stride = 4
    g_baby = [1] + [pow(5, i * stride, twoN) for i in range(1, nb)]
    g_giant = [1] + [pow(5, t * nb * stride, twoN) for t in range(1, ng)]
    kb = [None] + [cfg1.key(g, f"gpu/pmv/kb{g}")[0] for g in g_baby[1:]]
    kg = [None] + [cfg1.key(g, f"gpu/pmv/kg{g}")[0] for g in g_giant[1:]]
    ell = P.L
    a, b = cfg1.ct(ell, "gpu/pmv/ct")
    diags = [synth.uniform_residues(P.ext_primes(ell), P.N, f"gpu/pmv/M{d}") for d in range(nb * ng)]
    oa, ob = cfg1.ctx.ptmatvecmult(dev(a), dev(b), ell, nb, ng, g_baby, g_giant,
                                   [None if k is None else dev(k) for k in kb],
                                   [None if k is None else dev(k) for k in kg],
                                   [dev(d) for d in diags], rescale=rescale)
    ra, rb = cfg1.o.ptmatvec(P, ell, a, b, nb, ng, g_baby, g_giant, kb, kg, diags, rescale_out=rescale)
    np.testing.assert_array_equal(host(oa), ra)
    np.testing.assert_array_equal(host(ob), rb)


@pytest.mark.parametrize("g", [0, 5, -1])
def test_keygen_parity(cfg1, g):
    P = cfg1.P
    g = 2 * P.N - 1 if g == -1 else g
    ref, a, e = cfg1.key(g, f"gpu/keygen/{g}")
    key = cfg1.ctx.keygen_ksk(dev(cfg1.s), dev(e), dev(a), g)
    np.testing.assert_array_equal(host(key), ref)


def test_invalid_arguments_rejected(cfg1):
    ckks = _gpu()
    P = cfg1.P
    x = dev(np.zeros((P.L + P.k, P.N), dtype=np.uint64))
    with pytest.raises(ckks.CkksError):
        cfg1.ctx.ntt(x, P.L + 1)           # level above L
    with pytest.raises(ckks.CkksError):
        cfg1.ctx.automorph(x, 4)           # even Galois element
    with pytest.raises(ckks.CkksError):
        cfg1.ctx.rescale(x[:1], 1)         # rescale needs ell >= 2
    with pytest.raises(ckks.CkksError):
        cfg1.ctx.modup(x, 2, 5)            # digit out of range
    with pytest.raises(ckks.CkksError):
        ckks.Context(12, [97], [193], 1)   # primes not = 1 mod 2N


# ------------------------------------------------------------------ headline shape
@pytest.fixture(scope="module")
def cfgB(oracle_lib):
    return Setup(oracle_lib, 16, 24, 8, 3, 54)


def test_hrotate_parity_headline_shape(cfgB):
    """HRotate by 5^1 at N=2^16, ell=24, k=8, dnum=3 (full oracle run)."""
    S = cfgB
    P = S.P
    g = 5
    key, _, _ = S.key(g, "gpu/B/key5")
    a, b = S.ct(P.L, "gpu/B/ct")
    outs = S.ctx.hrotate(dev(a), dev(b), P.L, [g], [dev(key)])
    (ra, rb), = S.o.hrotate(P, P.L, a, b, [g], [key])
    np.testing.assert_array_equal(host(outs[0][0]), ra)
    np.testing.assert_array_equal(host(outs[0][1]), rb)


def test_keyswitch_repeatable_headline_shape(cfgB):
    """Two launches on the same inputs give identical bits (no races)."""
    S = cfgB
    P = S.P
    key = S.key(0, "gpu/B/relin")[0]
    a, _ = S.ct(P.L, "gpu/B/ct2")
    dk, da = dev(key), dev(a)
    u1, v1 = S.ctx.keyswitch(da, P.L, dk)
    u2, v2 = S.ctx.keyswitch(da, P.L, dk)
    np.testing.assert_array_equal(host(u1), host(u2))
    np.testing.assert_array_equal(host(v1), host(v2))
    # sampled limbs against the oracle
    ou, ov = S.o.keyswitch(P, P.L, a, key)
    np.testing.assert_array_equal(host(u1), ou)
    np.testing.assert_array_equal(host(v1), ov)


# ------------------------------------------------------------------ other ring degrees of the configurations
def test_serving_ring_degree_n15(oracle_lib):
    """N=2^15 (the serving loop's second ring degree), 54-bit primes: batched
    KeySwitch / HRotate entries and Mult against the oracle."""
    S = Setup(oracle_lib, 15, 9, 3, 3, 54)
    P = S.P
    key = S.key(0, "gpu/n15/relin")[0]
    rot = S.key(5, "gpu/n15/rot5")[0]
    dk, dr = dev(key), dev(rot)
    levels = [9, 4, 6]
    cts = [S.ct(ell, f"gpu/n15/{i}") for i, ell in enumerate(levels)]
    outs = S.ctx.keyswitch_batch([dev(a) for a, _ in cts], [None, dev(cts[1][1]), None], levels, [1, 5, 1],
                                 [dk, dr, dk])
    for i, ell in enumerate(levels):
        a, b = cts[i]
        if i == 1:
            ((ra, rb),) = S.o.hrotate(P, ell, a, b, [5], [rot])
        else:
            ra, rb = S.o.keyswitch(P, ell, a, key)
        np.testing.assert_array_equal(host(outs[i][0]), ra)
        np.testing.assert_array_equal(host(outs[i][1]), rb)
    a2, b2 = S.ct(6, "gpu/n15/m2")
    ma, mb = S.ctx.mult(dev(cts[2][0]), dev(cts[2][1]), dev(a2), dev(b2), 6, dk)
    ra, rb = S.o.mult(P, 6, cts[2][0], cts[2][1], a2, b2, key)
    np.testing.assert_array_equal(host(ma), ra)
    np.testing.assert_array_equal(host(mb), rb)


def test_keyswitch_ring_degree_n17(oracle_lib):
    """N=2^17 (the paper's bootstrapping ring degree), 54-bit primes, small level."""
    S = Setup(oracle_lib, 17, 4, 2, 2, 54)
    key = S.key(0, "gpu/n17/relin")[0]
    a, _ = S.ct(4, "gpu/n17/ct")
    u, v = S.ctx.keyswitch(dev(a), 4, dev(key))
    ru, rv = S.o.keyswitch(S.P, 4, a, key)
    np.testing.assert_array_equal(host(u), ru)
    np.testing.assert_array_equal(host(v), rv)


def test_ptmatvec_headline_shape(cfgB):
    """PtMatVecMult (2 baby x 2 giant steps, rescaled) at N=2^16, ell=24, k=8, dnum=3."""
    S = cfgB
    P = S.P
    twoN = 2 * P.N
    g_baby, g_giant = [1, 5], [1, pow(5, 2, twoN)]
    kb = [None, S.key(5, "gpu/B/pmv/kb")[0]]
    kg = [None, S.key(g_giant[1], "gpu/B/pmv/kg")[0]]
    a, b = S.ct(P.L, "gpu/B/pmv/ct")
    diags = [synth.uniform_residues(P.ext_primes(P.L), P.N, f"gpu/B/pmv/M{d}") for d in range(4)]
    oa, ob = S.ctx.ptmatvecmult(dev(a), dev(b), P.L, 2, 2, g_baby, g_giant, [None, dev(kb[1])], [None, dev(kg[1])],
                                [dev(d) for d in diags], rescale=True)
    ra, rb = S.o.ptmatvec(P, P.L, a, b, 2, 2, g_baby, g_giant, kb, kg, diags, rescale_out=True)
    np.testing.assert_array_equal(host(oa), ra)
    np.testing.assert_array_equal(host(ob), rb)
