"""The serving loop through the C ABI: requests of two ring degrees, mixed
operations (HRotate, KeySwitch, Mult + relinearisation + Rescale, NewMult) and mixed
levels arrive while others run; every result must carry the bits of the same
request run alone (tolerance 0, exact modular arithmetic), whatever batch it
landed in and whatever ran beside it."""
import numpy as np
import pytest

import synth
from tests.test_gpu_parity import Setup, _gpu, dev, host

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


class Pool:
    """Two contexts (N = 2^11 and 2^12, L = 6, k = 2, dnum = 3), a relinearisation
    key and two rotation keys each."""

    def __init__(self, oracle_lib):
        self.S = [Setup(oracle_lib, 11, 6, 2, 3, 50), Setup(oracle_lib, 12, 6, 2, 3, 50)]
        self.gs = [5, 25]
        self.keys = []
        for c, S in enumerate(self.S):
            self.keys.append({g: dev(S.key(g, f"gpu/serve/{c}/key{g}")[0]) for g in [0] + self.gs})

    def requests(self, n, tag, gap_ms=0.02):
        ops = synth.uniform_ints(n, 0, 3, f"{tag}/op")
        ctxs = synth.uniform_ints(n, 0, 1, f"{tag}/ctx")
        lv = synth.uniform_ints(n, 2, 6, f"{tag}/level")
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
            reqs.append(r)
        return reqs

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
        ra, rb = pool.alone(r)
        np.testing.assert_array_equal(ga, ra, err_msg=f"request {i} ({r['op']}, ctx {r['ctx']}, ell {r['level']})")
        np.testing.assert_array_equal(gb, rb, err_msg=f"request {i}")
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
        ra, rb = pool.alone(r)
        np.testing.assert_array_equal(host(r["oa"]), ra)
        np.testing.assert_array_equal(host(r["ob"]), rb)
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
