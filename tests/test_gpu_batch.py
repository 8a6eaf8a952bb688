"""Batched key switching through the C ABI: many ciphertexts at uneven levels,
each with its own key and Galois element, one launch per pipeline step.

Every entry of a batch must carry the bits of the single-ciphertext call
(KeySwitch, or HRotate with one rotation, Algorithm 4) and of the oracle.
Exact modular arithmetic: tolerance 0.
"""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _entries(S, levels, rot_every, tag):
    """Inputs of a mixed batch: entry i is an HRotate when i % rot_every == 1
    (Galois elements 5, 5^7, 2N-1 in turn), else a KeySwitch.  Keys are
    shared between entries of the same Galois element."""
    P = S.P
    twoN = 2 * P.N
    gs_cycle = [5, pow(5, 7, twoN), twoN - 1]
    keys = {}
    a, b, g, kh = [], [], [], []
    for i, ell in enumerate(levels):
        ai, bi = S.ct(ell, f"{tag}/ct{i}")
        rot = rot_every > 0 and i % rot_every == 1
        gi = gs_cycle[(i // max(rot_every, 1)) % 3] if rot else 0
        if gi not in keys:
            keys[gi] = S.key(gi, f"{tag}/key{gi}")[0]
        a.append(ai)
        b.append(bi if rot else None)
        g.append(gi if rot else 1)
        kh.append(gi)
    return a, b, g, kh, keys


def _run_and_check(S, levels, rot_every, tag, oracle_every=1):
    P, ctx = S.P, S.ctx
    a, b, g, kh, keys = _entries(S, levels, rot_every, tag)
    dkeys = {gi: dev(k) for gi, k in keys.items()}
    da = [dev(x) for x in a]
    db = [None if x is None else dev(x) for x in b]
    outs = ctx.keyswitch_batch(da, db, levels, g, [dkeys[gi] for gi in kh])
    for i, ell in enumerate(levels):
        if db[i] is None:
            su, sv = ctx.keyswitch(da[i], ell, dkeys[kh[i]])
        else:
            ((su, sv),) = ctx.hrotate(da[i], db[i], ell, [g[i]], [dkeys[kh[i]]])
        np.testing.assert_array_equal(host(outs[i][0]), host(su), err_msg=f"entry {i} ell={ell}")
        np.testing.assert_array_equal(host(outs[i][1]), host(sv), err_msg=f"entry {i} ell={ell}")
        if i % oracle_every == 0:
            if b[i] is None:
                ru, rv = S.o.keyswitch(P, ell, a[i], keys[kh[i]])
            else:
                ((ru, rv),) = S.o.hrotate(P, ell, a[i], b[i], [g[i]], [keys[kh[i]]])
            np.testing.assert_array_equal(host(outs[i][0]), ru, err_msg=f"oracle entry {i}")
            np.testing.assert_array_equal(host(outs[i][1]), rv, err_msg=f"oracle entry {i}")
    return outs


@pytest.fixture(scope="module")
def cfg1(oracle_lib):
    return Setup(oracle_lib, 12, 6, 3, 2, 50)


@pytest.fixture(scope="module")
def cfg_odd(oracle_lib):
    return Setup(oracle_lib, 11, 7, 3, 3, 50)


def test_batch_mixed_levels_keyswitch_and_hrotate(cfg1):
    """Every level 1..L, KeySwitch and HRotate entries interleaved."""
    _run_and_check(cfg1, [6, 1, 3, 5, 2, 6, 4, 1, 3, 6], 2, "gpu/batch/c1")


def test_batch_partial_digits(cfg_odd):
    """alpha = 3, L = 7: last digits of 1 or 2 limbs at most levels."""
    _run_and_check(cfg_odd, [7, 5, 1, 4, 2, 6, 3, 7], 3, "gpu/batch/odd")


def test_batch_more_than_64_entries(oracle_lib):
    """70 entries: two internal batches, the second of 6."""
    S = Setup(oracle_lib, 10, 4, 2, 2, 50)
    levels = synth.uniform_ints(70, 1, 4, "gpu/batch/70/levels")
    _run_and_check(S, levels, 4, "gpu/batch/70", oracle_every=9)


def test_batch_wide_primes_run_one_by_one(oracle_lib):
    """58-bit primes: no split conversion, entries run one after another."""
    S = Setup(oracle_lib, 11, 4, 2, 2, 58)
    _run_and_check(S, [4, 2, 3, 1], 2, "gpu/batch/wide")


def test_batch_edge_arguments(cfg1):
    ckks = _gpu()
    ctx, P = cfg1.ctx, cfg1.P
    assert ctx.keyswitch_batch([], None, [], None, []) == []
    a, _ = cfg1.ct(2, "gpu/batch/edge")
    key = dev(cfg1.key(0, "gpu/batch/edge/key")[0])
    da = dev(a)
    with pytest.raises(ckks.CkksError):
        ctx.keyswitch_batch([da], None, [P.L + 1], None, [key])      # level above L
    with pytest.raises(ckks.CkksError):
        ctx.keyswitch_batch([da], None, [0], None, [key])            # level 0
    with pytest.raises(ckks.CkksError):
        ctx.keyswitch_batch([da], [da], [2], [4], [key])             # even Galois element
    # the Galois element of a KeySwitch entry is ignored
    (u, v), = ctx.keyswitch_batch([da], [None], [2], [4], [key])
    su, sv = ctx.keyswitch(da, 2, key)
    np.testing.assert_array_equal(host(u), host(su))
    np.testing.assert_array_equal(host(v), host(sv))


@pytest.fixture(scope="module")
def cfgB(oracle_lib):
    return Setup(oracle_lib, 16, 24, 8, 3, 54)


def test_batch_64_uneven_levels_headline_shape(cfgB):
    """64 KeySwitches at levels uniform in {4..24}, N=2^16, k=8, dnum=3, one
    shared key: every entry against the single call, the lowest- and
    highest-level entries against the oracle."""
    S = cfgB
    P, ctx = S.P, S.ctx
    levels = synth.uniform_ints(64, 4, 24, "batch/levels")
    key = S.key(0, "gpu/B/relin")[0]
    dkey = dev(key)
    a = [S.ct(ell, f"gpu/B/batch/ct{i}")[0] for i, ell in enumerate(levels)]
    da = [dev(x) for x in a]
    outs = ctx.keyswitch_batch(da, None, levels, None, [dkey] * 64)
    ws = S.ctx.workspace(3, P.L)
    for i, ell in enumerate(levels):
        su, sv = ctx.keyswitch(da[i], ell, dkey, ws=ws)
        np.testing.assert_array_equal(host(outs[i][0]), host(su), err_msg=f"entry {i} ell={ell}")
        np.testing.assert_array_equal(host(outs[i][1]), host(sv), err_msg=f"entry {i} ell={ell}")
    for i in (levels.index(min(levels)), levels.index(max(levels))):
        ru, rv = S.o.keyswitch(P, levels[i], a[i], key)
        np.testing.assert_array_equal(host(outs[i][0]), ru)
        np.testing.assert_array_equal(host(outs[i][1]), rv)
    # a second run over the same workspace gives the same bits
    outs2 = ctx.keyswitch_batch(da, None, levels, None, [dkey] * 64)
    for (u1, v1), (u2, v2) in zip(outs, outs2):
        assert torch.equal(u1, u2) and torch.equal(v1, v2)


def test_batch_captured_in_a_cuda_graph(cfg1):
    """The batched call launches only kernels on the caller's stream (no
    allocation, no synchronisation), so it can be captured once in a CUDA graph
    and replayed; the replay gives the same bits as the direct call."""
    S = cfg1
    levels = [6, 2, 5, 3, 6, 1]
    key = dev(S.key(0, "gpu/graph/key")[0])
    a = [dev(S.ct(ell, f"gpu/graph/{i}")[0]) for i, ell in enumerate(levels)]
    want = S.ctx.keyswitch_batch(a, None, levels, None, [key] * len(levels))
    outs = [(S.ctx.empty(ell), S.ctx.empty(ell)) for ell in levels]
    ws = S.ctx.batch_workspace(levels)
    st = torch.cuda.Stream()
    torch.cuda.synchronize()
    with torch.cuda.stream(st):
        S.ctx.keyswitch_batch(a, None, levels, None, [key] * len(levels), outs=outs, ws=ws, stream=st)  # warm-up
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=st):
        S.ctx.keyswitch_batch(a, None, levels, None, [key] * len(levels), outs=outs, ws=ws, stream=st)
    for o in outs:
        o[0].zero_()
        o[1].zero_()
    g.replay()
    torch.cuda.synchronize()
    for (ga, gb), (wa, wb) in zip(outs, want):
        assert torch.equal(ga, wa) and torch.equal(gb, wb)


def test_batch_split_over_streams(cfg1):
    """ckks_batch_streams: a batch of 16 KeySwitch / HRotate entries at uneven
    levels cut over 1 to 4 streams gives the same bits every time, equal to the
    oracle on sampled entries, and a split batch captured in a CUDA graph (the
    fork and join of the streams become graph edges) replays to the same bits."""
    S = cfg1
    P, ctx = S.P, S.ctx
    levels = [6, 2, 5, 3, 6, 1, 4, 6, 2, 5, 3, 6, 1, 4, 5, 6]
    g = 5
    relin = S.key(0, "gpu/split/relin")[0]
    rot = S.key(g, "gpu/split/rot")[0]
    cts = [S.ct(ell, f"gpu/split/{i}") for i, ell in enumerate(levels)]
    da = [dev(a) for a, _ in cts]
    db = [dev(b) if i % 3 == 1 else None for i, (_, b) in enumerate(cts)]
    gal = [g if i % 3 == 1 else 1 for i in range(len(levels))]
    keys = [dev(rot) if i % 3 == 1 else dev(relin) for i in range(len(levels))]
    results = []
    try:
        for nst in (1, 2, 3, 4):
            ctx.batch_streams(nst)
            outs = ctx.keyswitch_batch(da, db, levels, gal, keys)
            results.append([(host(u), host(v)) for u, v in outs])
        for r in results[1:]:
            for i, ((u0, v0), (u, v)) in enumerate(zip(results[0], r)):
                np.testing.assert_array_equal(u, u0, err_msg=f"entry {i}")
                np.testing.assert_array_equal(v, v0, err_msg=f"entry {i}")
        for i in (0, 1, 5, 13):
            a, b = cts[i]
            if i % 3 == 1:
                ((ra, rb),) = S.o.hrotate(P, levels[i], a, b, [g], [rot])
            else:
                ra, rb = S.o.keyswitch(P, levels[i], a, relin)
            np.testing.assert_array_equal(results[0][i][0], ra, err_msg=f"entry {i} vs oracle")
            np.testing.assert_array_equal(results[0][i][1], rb, err_msg=f"entry {i} vs oracle")
        ctx.batch_streams(4)
        outs = [(ctx.empty(ell), ctx.empty(ell)) for ell in levels]
        ws = ctx.batch_workspace(levels)
        st = torch.cuda.Stream()
        torch.cuda.synchronize()
        with torch.cuda.stream(st):
            ctx.keyswitch_batch(da, db, levels, gal, keys, outs=outs, ws=ws, stream=st)  # warm-up
        torch.cuda.synchronize()
        graph = torch.cuda.CUDAGraph()
        with torch.cuda.graph(graph, stream=st):
            ctx.keyswitch_batch(da, db, levels, gal, keys, outs=outs, ws=ws, stream=st)
        for o in outs:
            o[0].zero_()
            o[1].zero_()
        graph.replay()
        torch.cuda.synchronize()
        for i, (u, v) in enumerate(outs):
            np.testing.assert_array_equal(host(u), results[0][i][0], err_msg=f"graph entry {i}")
            np.testing.assert_array_equal(host(v), results[0][i][1], err_msg=f"graph entry {i}")
    finally:
        ctx.batch_streams(2)


@pytest.mark.parametrize("which", ["cfg1", "cfg_odd"])
def test_hrotate_batch_hoisted_rotations(request, which):
    """Several ciphertexts at uneven levels, each rotated by several Galois
    elements with one ModUp per ciphertext: every output equals ckks_hrotate of
    that ciphertext with the same rotations, and the oracle."""
    S = request.getfixturevalue(which)
    P = S.P
    twoN = 2 * P.N
    gs = [5, pow(5, 3, twoN), twoN - 1, pow(5, 9, twoN)]
    keys = {g: S.key(g, f"gpu/hrb/{which}/{g}")[0] for g in gs}
    dkeys = {g: dev(k) for g, k in keys.items()}
    levels = [P.L, 2, P.L - 1, 1]
    nrots = [3, 1, 4, 2]
    cts, rots = [], []
    for c, (ell, r) in enumerate(zip(levels, nrots)):
        a, b = S.ct(ell, f"gpu/hrb/{which}/{c}")
        cts.append((a, b))
        rots.append([gs[(c + j) % len(gs)] for j in range(r)])
    dcts = [(dev(a), dev(b)) for a, b in cts]
    outs = S.ctx.hrotate_batch(dcts, levels, [[(g, dkeys[g]) for g in r] for r in rots])
    for c, ell in enumerate(levels):
        single = S.ctx.hrotate(*dcts[c], ell, rots[c], [dkeys[g] for g in rots[c]])
        ref = S.o.hrotate(P, ell, *cts[c], rots[c], [keys[g] for g in rots[c]])
        for (ga, gb), (sa, sb), (ra, rb) in zip(outs[c], single, ref):
            np.testing.assert_array_equal(host(ga), host(sa))
            np.testing.assert_array_equal(host(gb), host(sb))
            np.testing.assert_array_equal(host(ga), ra)
            np.testing.assert_array_equal(host(gb), rb)


def test_hrotate_batch_many_rotations_headline_shape(cfgB):
    """Two ciphertexts at N=2^16, ell=24 and 20, 40 rotations each (80 rotation
    entries: two launches of the inner-product and ModDown steps): equal to
    the single hoisted calls."""
    S = cfgB
    P = S.P
    twoN = 2 * P.N
    gs = [pow(5, i + 1, twoN) for i in range(4)]
    keys = {g: dev(S.key(g, f"gpu/hrbB/{g}")[0]) for g in gs}
    levels = [24, 20]
    dcts = [tuple(dev(x) for x in S.ct(ell, f"gpu/hrbB/{c}")) for c, ell in enumerate(levels)]
    rots = [[gs[j % 4] for j in range(40)] for _ in levels]
    outs = S.ctx.hrotate_batch(dcts, levels, [[(g, keys[g]) for g in r] for r in rots])
    for c, ell in enumerate(levels):
        single = S.ctx.hrotate(*dcts[c], ell, rots[c][:4], [keys[g] for g in rots[c][:4]])
        for j in range(40):
            sa, sb = single[j % 4]
            assert torch.equal(outs[c][j][0], sa) and torch.equal(outs[c][j][1], sb)
