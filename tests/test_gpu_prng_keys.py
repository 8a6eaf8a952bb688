"""Compressed key-switching keys (Sec. 5.3) through the C ABI: the GPU key
generator, the expansion of a compressed key, and key switching that
regenerates the uniform key half on chip must give the bits of the oracle's
full key and of key switching with that full key (tolerance 0)."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def cfg(oracle_lib):
    return Setup(oracle_lib, 11, 7, 3, 3, 50)


def _seeded_key(S, g, seed, tag):
    P = S.P
    e = np.stack([synth.gaussian(P.N, f"{tag}/e{j}") for j in range(P.dnum)])
    key_b = S.ctx.keygen_ksk_seeded(dev(S.s), dev(e), seed, g)
    sp = S.o.sq_secret(P, S.s) if g == 0 else S.o.rot_secret(P, S.s, g)
    ref = S.o.keygen(P, S.o.prng_key_a(P, seed), S.s, sp, e)
    return key_b, ref


@pytest.mark.parametrize("g", [0, 5])
def test_seeded_keygen_and_expand_match_oracle(cfg, g):
    seed = synth.stream_seed(f"gpu/prng/seed{g}")
    key_b, ref = _seeded_key(cfg, g, seed, f"gpu/prng/key{g}")
    np.testing.assert_array_equal(host(key_b), ref[:, 1])
    full = cfg.ctx.ksk_expand(key_b, seed)
    np.testing.assert_array_equal(host(full), ref)


def test_batch_with_compressed_keys_equals_full_keys(cfg):
    P = cfg.P
    g = 25
    seeds = [synth.stream_seed("gpu/prng/b/relin"), synth.stream_seed("gpu/prng/b/rot")]
    kr, ref_r = _seeded_key(cfg, 0, seeds[0], "gpu/prng/b/relin")
    kg, ref_g = _seeded_key(cfg, g, seeds[1], "gpu/prng/b/rot")
    full_r, full_g = cfg.ctx.ksk_expand(kr, seeds[0]), cfg.ctx.ksk_expand(kg, seeds[1])
    levels = [7, 3, 5, 1, 6, 2, 7, 4]
    a, b, gal, kb, kf, sd = [], [], [], [], [], []
    for i, ell in enumerate(levels):
        ai, bi = cfg.ct(ell, f"gpu/prng/b/{i}")
        rot = i % 2 == 1
        a.append(dev(ai))
        b.append(dev(bi) if rot else None)
        gal.append(g if rot else 1)
        kb.append(kg if rot else kr)
        kf.append(full_g if rot else full_r)
        sd.append(seeds[1] if rot else seeds[0])
    got = cfg.ctx.keyswitch_batch(a, b, levels, gal, kb, seeds=sd)
    want = cfg.ctx.keyswitch_batch(a, b, levels, gal, kf)
    for (ga, gb), (wa, wb) in zip(got, want):
        np.testing.assert_array_equal(host(ga), host(wa))
        np.testing.assert_array_equal(host(gb), host(wb))
    # and against the oracle for two entries
    for i in (0, 1):
        ell = levels[i]
        ai = host(a[i])
        if b[i] is None:
            ru, rv = cfg.o.keyswitch(P, ell, ai, ref_r)
        else:
            ((ru, rv),) = cfg.o.hrotate(P, ell, ai, host(b[i]), [g], [ref_g])
        np.testing.assert_array_equal(host(got[i][0]), ru)
        np.testing.assert_array_equal(host(got[i][1]), rv)


def test_server_with_compressed_keys(cfg):
    ckks = _gpu()
    from paper_2112_06396_gb300 import serving

    seed = synth.stream_seed("gpu/prng/srv")
    kb, _ = _seeded_key(cfg, 0, seed, "gpu/prng/srv")
    full = cfg.ctx.ksk_expand(kb, seed)
    srv = ckks.Server([cfg.ctx], 1 << 30, max_batch=8, streams=2)
    h = srv.add_key(0, kb, seed=seed)
    st = srv.stats()
    assert st["mem_keys"] == kb.numel() * 8  # half of a full key
    reqs = []
    for i, ell in enumerate([7, 2, 5, 3, 6, 4]):
        a1, b1 = cfg.ct(ell, f"gpu/prng/srv/{i}/1")
        a2, b2 = cfg.ct(ell, f"gpu/prng/srv/{i}/2")
        reqs.append({"t_ms": 0.01 * i, "op": "newmult" if i % 2 else "mult", "ctx": 0, "level": ell, "a": dev(a1),
                     "b": dev(b1), "a2": dev(a2), "b2": dev(b2), "key": h, "oa": cfg.ctx.empty(ell - 1),
                     "ob": cfg.ctx.empty(ell - 1)})
    serving.replay(srv, reqs)
    for r in reqs:
        oa, ob = cfg.ctx.mult(r["a"], r["b"], r["a2"], r["b2"], r["level"], full, new=r["op"] == "newmult")
        np.testing.assert_array_equal(host(r["oa"]), host(oa))
        np.testing.assert_array_equal(host(r["ob"]), host(ob))
    srv.close()


def test_compressed_keys_headline_shape(oracle_lib):
    """N=2^16, ell=24, k=8, dnum=3: 8 KeySwitches with one compressed key equal
    the same batch with the expanded key."""
    S = Setup(oracle_lib, 16, 24, 8, 3, 54)
    seed = synth.stream_seed("gpu/prng/B")
    e = np.stack([synth.gaussian(S.P.N, f"gpu/prng/B/e{j}") for j in range(3)])
    kb = S.ctx.keygen_ksk_seeded(dev(S.s), dev(e), seed, 0)
    full = S.ctx.ksk_expand(kb, seed)
    levels = [24, 17, 9, 4, 24, 12, 20, 8]
    a = [dev(S.ct(ell, f"gpu/prng/B/{i}")[0]) for i, ell in enumerate(levels)]
    got = S.ctx.keyswitch_batch(a, None, levels, None, [kb] * 8, seeds=[seed] * 8)
    want = S.ctx.keyswitch_batch(a, None, levels, None, [full] * 8)
    for (ga, gb), (wa, wb) in zip(got, want):
        assert torch.equal(ga, wa) and torch.equal(gb, wb)
    # the expansion's first digit row against the oracle's generator on a sample
    a0 = host(full[0, 0])
    for l in (0, 23, 24, 31):
        for n in (0, 1, 4097, S.P.N - 1):
            assert int(a0[l, n]) == S.o.prng_key_a_element(S.P, seed, 0, l, n)


def test_registered_compressed_keys_in_every_call(cfg):
    """A compressed key registered with its context works in the single calls
    (KeySwitch, Rotate, HRotate, PtMatVecMult with compressed baby and giant
    keys) with the bits of the expanded key."""
    S = cfg
    P, ctx = S.P, S.ctx
    twoN = 2 * P.N
    ell = P.L
    a, b = S.ct(ell, "gpu/prng/reg/ct")
    da, db = dev(a), dev(b)
    relin_seed = synth.stream_seed("gpu/prng/reg/relin")
    kr, _ = _seeded_key(S, 0, relin_seed, "gpu/prng/reg/relin")
    ctx.register_compressed_key(kr, relin_seed)
    full_r = ctx.ksk_expand(kr, relin_seed)
    u1, v1 = ctx.keyswitch(da, ell, kr)
    u2, v2 = ctx.keyswitch(da, ell, full_r)
    assert torch.equal(u1, u2) and torch.equal(v1, v2)
    nb, ng = 3, 2
    g_baby = [1] + [pow(5, i, twoN) for i in range(1, nb)]
    g_giant = [1] + [pow(5, nb, twoN)]
    comp, full = {}, {}
    for g in g_baby[1:] + g_giant[1:]:
        sd = synth.stream_seed(f"gpu/prng/reg/{g}")
        kb, _ = _seeded_key(S, g, sd, f"gpu/prng/reg/{g}")
        ctx.register_compressed_key(kb, sd)
        comp[g], full[g] = kb, ctx.ksk_expand(kb, sd)
    g = g_baby[1]
    (ra, rb), = ctx.hrotate(da, db, ell, [g], [comp[g]])
    (fa, fb), = ctx.hrotate(da, db, ell, [g], [full[g]])
    assert torch.equal(ra, fa) and torch.equal(rb, fb)
    ra, rb = ctx.rotate(da, db, ell, g, comp[g])
    fa, fb = ctx.rotate(da, db, ell, g, full[g])
    assert torch.equal(ra, fa) and torch.equal(rb, fb)
    diags = [dev(synth.uniform_residues(P.ext_primes(ell), P.N, f"gpu/prng/reg/M{d}")) for d in range(nb * ng)]
    kbc = [None] + [comp[g] for g in g_baby[1:]]
    kgc = [None] + [comp[g] for g in g_giant[1:]]
    kbf = [None] + [full[g] for g in g_baby[1:]]
    kgf = [None] + [full[g] for g in g_giant[1:]]
    ca, cb = ctx.ptmatvecmult(da, db, ell, nb, ng, g_baby, g_giant, kbc, kgc, diags, rescale=True)
    pa, pb = ctx.ptmatvecmult(da, db, ell, nb, ng, g_baby, g_giant, kbf, kgf, diags, rescale=True)
    assert torch.equal(ca, pa) and torch.equal(cb, pb)
    for k in [kr] + list(comp.values()):
        ctx.unregister_compressed_key(k)


def test_registered_compressed_key_wide_primes(oracle_lib):
    """58-bit primes (single-operation launches): a registered compressed key
    gives the bits of its expansion, and those of the oracle."""
    S = Setup(oracle_lib, 11, 4, 2, 2, 58)
    seed = synth.stream_seed("gpu/prng/wide")
    kb, ref = _seeded_key(S, 0, seed, "gpu/prng/wide")
    S.ctx.register_compressed_key(kb, seed)
    for ell in (4, 1):
        a, _ = S.ct(ell, f"gpu/prng/wide/{ell}")
        u, v = S.ctx.keyswitch(dev(a), ell, kb)
        ru, rv = S.o.keyswitch(S.P, ell, a, ref)
        np.testing.assert_array_equal(host(u), ru)
        np.testing.assert_array_equal(host(v), rv)
    S.ctx.unregister_compressed_key(kb)


@pytest.mark.parametrize("shape", [(16, 7, 3, 3, 54), (12, 12, 2, 6, 50)], ids=["n16_dnum3", "n12_dnum6"])
def test_batch_runs_of_shared_compressed_keys(oracle_lib, shape):
    """A batch whose entries come in runs sharing one key (compressed keys
    registered with the context, and full keys, in one call): consecutive
    entries with one compressed key are served by one CTA per tile and prime,
    the key half generated once per group (at N=2^16 the launch is large
    enough for groups as long as the runs).  Runs of 1 to 5 entries, uneven
    levels (so a group's entries own different chain primes and digit counts;
    one run starts with an entry at level 1), KeySwitch and HRotate entries in
    one run, dnum 3 (digits held in registers) and 6 (digits looped, groups of
    one): every entry equals the same batch with expanded keys, and the oracle
    on a sample.  The batch runs as one part on one stream."""
    S = Setup(oracle_lib, *shape)
    P, ctx = S.P, S.ctx
    ctx.batch_streams(1)
    g = 25
    sr, sg = synth.stream_seed("gpu/prng/runs/relin"), synth.stream_seed("gpu/prng/runs/rot")
    kr, ref_r = _seeded_key(S, 0, sr, "gpu/prng/runs/relin")
    kg, ref_g = _seeded_key(S, g, sg, "gpu/prng/runs/rot")
    full_r, full_g = ctx.ksk_expand(kr, sr), ctx.ksk_expand(kg, sg)
    ctx.register_compressed_key(kr, sr)
    ctx.register_compressed_key(kg, sg)
    try:
        L = P.L
        # (key, expanded key, oracle key, rotation?) per entry, in runs
        plan = ([(kg, full_g, ref_g, True)] * 3 + [(full_r, full_r, ref_r, False)] * 2 +
                [(kr, full_r, ref_r, False)] * 5 + [(kg, full_g, ref_g, True)] + [(full_g, full_g, ref_g, True)])
        levels = [1, L, 2, L, 3, 1, L - 1, 2, L, max(1, L // 2), L, 4]
        a, b, gal, keys, fulls = [], [], [], [], []
        for i, ((k, f, _, rot), ell) in enumerate(zip(plan, levels)):
            ai, bi = S.ct(ell, f"gpu/prng/runs/{i}")
            a.append(dev(ai))
            b.append(dev(bi) if rot else None)
            gal.append(g if rot else 1)
            keys.append(k)
            fulls.append(f)
        got = ctx.keyswitch_batch(a, b, levels, gal, keys)
        want = ctx.keyswitch_batch(a, b, levels, gal, fulls)
        for i, ((ga, gb), (wa, wb)) in enumerate(zip(got, want)):
            assert torch.equal(ga, wa) and torch.equal(gb, wb), i
        for i in (1, 6, 8):
            ell, ref = levels[i], plan[i][2]
            ai = host(a[i])
            if b[i] is None:
                ru, rv = S.o.keyswitch(P, ell, ai, ref)
            else:
                ((ru, rv),) = S.o.hrotate(P, ell, ai, host(b[i]), [g], [ref])
            np.testing.assert_array_equal(host(got[i][0]), ru)
            np.testing.assert_array_equal(host(got[i][1]), rv)
        # single KeySwitch calls with the full and the compressed key
        ru, rv = S.o.keyswitch(P, L, host(a[3]), ref_r)
        for k in (full_r, kr):
            u, v = ctx.keyswitch(a[3], L, k)
            np.testing.assert_array_equal(host(u), ru)
            np.testing.assert_array_equal(host(v), rv)
        assert ctx.poll_status()
    finally:
        ctx.unregister_compressed_key(kr)
        ctx.unregister_compressed_key(kg)
        ctx.batch_streams(2)
