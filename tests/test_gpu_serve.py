"""The serving loop through the C ABI: requests of two ring degrees, mixed
operations (HRotate, KeySwitch, Mult + relinearisation + Rescale, NewMult) and mixed
levels arrive while others run; every result must carry the bits of the oracle's
result for that request (HRotate = Algorithm 4, Mult = Algorithm 2, NewMult =
Algorithm 7, KeySwitch = Algorithms 2-4's key switch) and of the same request run
alone through the single-ciphertext calls (tolerance 0, exact modular arithmetic),
whatever batch it landed in and whatever ran beside it."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class Pool:
    """Contexts (by default N = 2^11 and 2^12, L = 6, k = 2, dnum = 3), a
    relinearisation key and two rotation keys each, generated by the oracle."""

    def __init__(self, oracle_lib, shapes=((11, 6, 2, 3, 50), (12, 6, 2, 3, 50)), tag="gpu/serve"):
        self.S = [Setup(oracle_lib, *sh) for sh in shapes]
        self.o = oracle_lib
        self.gs = [5, 25]
        self.keys = []
        self.okeys = []
        for c, S in enumerate(self.S):
            ok = {g: S.key(g, f"{tag}/{c}/key{g}")[0] for g in [0] + self.gs}
            self.okeys.append(ok)
            self.keys.append({g: dev(k) for g, k in ok.items()})

    def requests(self, n, tag, gap_ms=0.02, min_level=2):
        ops = synth.uniform_ints(n, 0, 3, f"{tag}/op")
        ctxs = synth.uniform_ints(n, 0, len(self.S) - 1, f"{tag}/ctx")
        lv = synth.uniform_ints(n, min_level, min(S.P.L for S in self.S), f"{tag}/level")
        gaps = synth.exponential_gaps(n, gap_ms, f"{tag}/gaps")
        t = np.cumsum(gaps)
        reqs = []
        for i in range(n):
            c, ell = ctxs[i], lv[i]
            S = self.S[c]
            a, b = S.ct(ell, f"{tag}/{i}/1")
            r = {"t_ms": float(t[i]), "ctx": c, "level": ell, "a": dev(a), "b": dev(b)}
            if ops[i] == 0:
                g = self.gs[i % 2]
                r.update(op="hrotate", galois=g, kkey=g, oa=S.ctx.empty(ell), ob=S.ctx.empty(ell))
            elif ops[i] in (1, 3):
                a2, b2 = S.ct(ell, f"{tag}/{i}/2")
                r.update(op="mult" if ops[i] == 1 else "newmult", a2=dev(a2), b2=dev(b2), galois=1, kkey=0,
                         oa=S.ctx.empty(ell - 1), ob=S.ctx.empty(ell - 1))
            else:
                r.update(op="keyswitch", galois=1, kkey=0, oa=S.ctx.empty(ell), ob=S.ctx.empty(ell))
            r["host"] = (a, b) if ops[i] in (0, 2) else (a, b, a2, b2)
            reqs.append(r)
        return reqs

    def oracle(self, r):
        """The oracle's result for request r (host arrays)."""
        S, o = self.S[r["ctx"]], self.o
        key = self.okeys[r["ctx"]][r["kkey"]]
        ell = r["level"]
        if r["op"] == "hrotate":
            a, b = r["host"]
            ((oa, ob),) = o.hrotate(S.P, ell, a, b, [r["galois"]], [key])
        elif r["op"] == "mult":
            oa, ob = o.mult(S.P, ell, *r["host"], key)
        elif r["op"] == "newmult":
            oa, ob = o.newmult(S.P, ell, *r["host"], key)
        else:
            oa, ob = o.keyswitch(S.P, ell, r["host"][0], key)
        return oa, ob

    def alone(self, r):
        ctx = self.S[r["ctx"]].ctx
        key = self.keys[r["ctx"]][r["kkey"]]
        ell = r["level"]
        if r["op"] == "hrotate":
            ((oa, ob),) = ctx.hrotate(r["a"], r["b"], ell, [r["galois"]], [key])
        elif r["op"] in ("mult", "newmult"):
            oa, ob = ctx.mult(r["a"], r["b"], r["a2"], r["b2"], ell, key, new=r["op"] == "newmult")
        else:
            oa, ob = ctx.keyswitch(r["a"], ell, key)
        return host(oa), host(ob)


@pytest.fixture(scope="module")
def pool(oracle_lib):
    return Pool(oracle_lib)


def _server(pool, budget, max_batch, streams):
    ckks = _gpu()
    srv = ckks.Server([S.ctx for S in pool.S], budget, max_batch=max_batch, streams=streams)
    handles = [{g: srv.add_key(c, k) for g, k in pool.keys[c].items()} for c in range(2)]
    return srv, handles


@pytest.mark.parametrize("max_batch,streams", [(16, 3), (1, 1)])
def test_results_same_alone_and_in_the_mix(pool, max_batch, streams):
    from paper_2112_06396_gb300 import serving

    srv, handles = _server(pool, 1 << 30, max_batch, streams)
    reqs = pool.requests(48, f"gpu/serve/mix{max_batch}")
    for r in reqs:
        r["key"] = handles[r["ctx"]][r["kkey"]]
    results, stats = serving.replay(srv, reqs)
    assert len(results) == len(reqs)
    st = srv.stats()
    assert st["pending"] == 0 and st["in_flight"] == 0 and st["mem_in_flight"] == 0
    assert st["requests_launched"] == len(reqs)
    if max_batch > 1:
        assert st["batches"] < len(reqs)  # requests really were batched
    for i, r in enumerate(reqs):
        ga, gb = host(r["oa"]), host(r["ob"])
        what = f"request {i} ({r['op']}, ctx {r['ctx']}, ell {r['level']})"
        oa, ob = pool.oracle(r)
        np.testing.assert_array_equal(ga, oa, err_msg=f"{what} vs oracle")
        np.testing.assert_array_equal(gb, ob, err_msg=f"{what} vs oracle")
        ra, rb = pool.alone(r)
        np.testing.assert_array_equal(ga, ra, err_msg=f"{what} vs alone")
        np.testing.assert_array_equal(gb, rb, err_msg=f"{what} vs alone")
    assert {r["op"] for r in reqs} == {"hrotate", "mult", "newmult", "keyswitch"}
    assert stats["p99_ms"] >= stats["p50_ms"] > 0
    srv.close()


def test_memory_admission_limits_what_runs(pool):
    """A budget that holds the keys and about one request at a time: everything
    still completes, with the same bits, and memory in flight stays within it."""
    ckks = _gpu()
    S1 = pool.S[1]
    key_bytes = sum(k.numel() * 8 for c in range(2) for k in pool.keys[c].values())
    ws = S1.ctx.workspace_bytes(ckks.OP_MULT, 6)
    budget = key_bytes + ws + 16 * 6 * S1.ctx.N * 8 + (1 << 16)
    srv, handles = _server(pool, budget, 16, 4)
    reqs = pool.requests(12, "gpu/serve/tight", gap_ms=0.0)
    for r in reqs:
        r["key"] = handles[r["ctx"]][r["kkey"]]
    seen_max = 0
    t0 = srv.now_ms()
    ids = []
    for r in reqs:
        if r["op"] in ("mult", "newmult"):
            ids.append(srv.submit_mult(r["ctx"], (r["a"], r["b"]), (r["a2"], r["b2"]), r["level"], r["key"], r["oa"],
                                       r["ob"], t0, new=r["op"] == "newmult"))
        elif r["op"] == "hrotate":
            ids.append(srv.submit_hrotate(r["ctx"], r["a"], r["b"], r["level"], r["galois"], r["key"], r["oa"],
                                          r["ob"], t0))
        else:
            ids.append(srv.submit_keyswitch(r["ctx"], r["a"], r["level"], r["key"], r["oa"], r["ob"], t0))
    done = []
    while len(done) < len(reqs):
        srv.step()
        st = srv.stats()
        seen_max = max(seen_max, st["mem_keys"] + st["mem_in_flight"])
        assert st["mem_keys"] + st["mem_in_flight"] <= budget
        done += srv.poll()
    assert sorted(d[0] for d in done) == sorted(ids)
    assert seen_max > key_bytes
    for r in reqs:
        oa, ob = pool.oracle(r)
        np.testing.assert_array_equal(host(r["oa"]), oa)
        np.testing.assert_array_equal(host(r["ob"]), ob)
        ra, rb = pool.alone(r)
        np.testing.assert_array_equal(host(r["oa"]), ra)
        np.testing.assert_array_equal(host(r["ob"]), rb)
    srv.close()


def test_serving_config_shapes_against_the_oracle(oracle_lib):
    """The serving configuration's shapes: N = 2^16 and 2^15, L = 24, k = 8,
    dnum = 3, 54-bit primes, levels uniform in {3..24}, a mixed served run: every
    request equals its single call, and one request of each operation at
    N = 2^16 (the largest level first) and one at N = 2^15 equal the oracle."""
    from paper_2112_06396_gb300 import serving

    big = Pool(oracle_lib, shapes=((16, 24, 8, 3, 54), (15, 24, 8, 3, 54)), tag="gpu/serve16")
    srv, handles = _server(big, 1 << 34, 16, 3)
    reqs = big.requests(24, "gpu/serve16/mix", min_level=3)
    for r in reqs:
        r["key"] = handles[r["ctx"]][r["kkey"]]
    results, stats = serving.replay(srv, reqs)
    assert len(results) == len(reqs)
    assert srv.stats()["batches"] < len(reqs)
    checked = {}
    for i in sorted(range(len(reqs)), key=lambda i: (reqs[i]["ctx"], -reqs[i]["level"])):
        r = reqs[i]
        ga, gb = host(r["oa"]), host(r["ob"])
        ra, rb = big.alone(r)
        np.testing.assert_array_equal(ga, ra, err_msg=f"request {i} vs alone")
        np.testing.assert_array_equal(gb, rb, err_msg=f"request {i} vs alone")
        tag = r["op"] if r["ctx"] == 0 else "n15"
        if checked.get(tag, 0) < 1:
            oa, ob = big.oracle(r)
            np.testing.assert_array_equal(ga, oa, err_msg=f"request {i} ({r['op']}, ell {r['level']}) vs oracle")
            np.testing.assert_array_equal(gb, ob, err_msg=f"request {i} vs oracle")
            checked[tag] = 1
    assert len(checked) >= 4, checked
    srv.close()


def test_timeout_in_a_served_batch_fails_only_that_batch(pool):
    """The serving loop reads its lane's status word when a batch completes: the
    test hook runs the bounded-wait self-test (an mbarrier nothing arrives on,
    20 ms) in front of the next batch, and every request of that batch must come
    back with CKKS_ETIMEOUT; the requests of the next batch must come back valid
    and equal to the oracle.  Nothing faults."""
    ckks = _gpu()
    srv, handles = _server(pool, 1 << 30, 16, 2)
    reqs = pool.requests(8, "gpu/serve/timeout", gap_ms=0.0)
    for r in reqs:
        r["key"] = handles[r["ctx"]][r["kkey"]]

    def submit(rs):
        ids = {}
        for r in rs:
            if r["op"] in ("mult", "newmult"):
                rid = srv.submit_mult(r["ctx"], (r["a"], r["b"]), (r["a2"], r["b2"]), r["level"], r["key"], r["oa"],
                                      r["ob"], new=r["op"] == "newmult")
            elif r["op"] == "hrotate":
                rid = srv.submit_hrotate(r["ctx"], r["a"], r["b"], r["level"], r["galois"], r["key"], r["oa"],
                                         r["ob"])
            else:
                rid = srv.submit_keyswitch(r["ctx"], r["a"], r["level"], r["key"], r["oa"], r["ob"])
            ids[rid] = r
        return ids

    def drain(n):
        out = []
        while len(out) < n:
            srv.step()
            out += srv.poll(with_status=True)
        return out

    first = reqs[0]
    srv.selftest_timeout(20000)
    ids = submit([first])
    got = drain(1)
    assert [(g[0], g[3]) for g in got] == [(next(iter(ids)), ckks.CKKS_ETIMEOUT)]
    ids = submit(reqs)
    got = drain(len(reqs))
    assert sorted(g[0] for g in got) == sorted(ids)
    assert all(g[3] == ckks.CKKS_OK for g in got)
    for r in reqs:
        oa, ob = pool.oracle(r)
        np.testing.assert_array_equal(host(r["oa"]), oa)
        np.testing.assert_array_equal(host(r["ob"]), ob)
    # the contexts' own status words were not touched by the served timeout
    torch.cuda.synchronize()
    for S in pool.S:
        assert S.ctx.poll_status() is True  # raises CkksError on CKKS_ETIMEOUT
    srv.close()


def test_submit_rejects_bad_requests(pool):
    ckks = _gpu()
    srv, handles = _server(pool, 1 << 30, 8, 2)
    S = pool.S[0]
    a, b = S.ct(3, "gpu/serve/bad")
    da, db = dev(a), dev(b)
    o = S.ctx.empty(3)
    with pytest.raises(ckks.CkksError):
        srv.submit_hrotate(0, da, db, 3, 5, handles[1][5], o, o)        # key of the other context
    with pytest.raises(ckks.CkksError):
        srv.submit_hrotate(0, da, db, 3, 4, handles[0][5], o, o)        # even Galois element
    with pytest.raises(ckks.CkksError):
        srv.submit_mult(0, (da, db), (da, db), 1, handles[0][0], o, o)  # Mult at level 1
    with pytest.raises(ckks.CkksError):
        srv.submit_keyswitch(2, da, 3, handles[0][0], o, o)             # no such context
    srv.close()
    tiny = ckks.Server([S.ctx], 1 << 19, max_batch=4, streams=1)
    with pytest.raises(ckks.CkksError):
        tiny.add_key(0, pool.keys[0][0])                                # the key alone exceeds the budget
    tiny.close()
