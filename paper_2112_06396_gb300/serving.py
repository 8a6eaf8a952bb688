"""Open-loop load generation for the serving loop (ckks_server_*).

A request stream (arrival times, operation, context, level, inputs, key) is
submitted to a :class:`ckks.Server` at its arrival times while the caller's
thread keeps stepping the server; finished requests are polled as they
complete.  The server's native policy does the admission, batching and
overlap; this module only replays arrivals and collects latencies.
"""
from __future__ import annotations

import math
import statistics


def replay(server, requests, max_wall_s=600.0):
    """requests: list of dicts with keys t_ms (arrival offset), op ('hrotate',
    'mult', 'newmult' or 'keyswitch'), ctx, level, a, b (and a2, b2 for mult), galois,
    key (server handle), oa, ob; sorted by t_ms.  Returns (results, stats):
    results maps request index -> (latency_ms, done_ms); stats has the
    throughput over the run and p50 / p99 latencies."""
    t0 = server.now_ms()
    ids = {}
    results = {}
    i = 0
    n = len(requests)
    while len(results) < n:
        now = server.now_ms()
        if now - t0 > max_wall_s * 1e3:
            raise TimeoutError("serving replay exceeded its wall-clock limit")
        while i < n and requests[i]["t_ms"] <= now - t0:
            r = requests[i]
            arr = t0 + r["t_ms"]
            if r["op"] == "hrotate":
                rid = server.submit_hrotate(r["ctx"], r["a"], r["b"], r["level"], r["galois"], r["key"], r["oa"],
                                            r["ob"], arr)
            elif r["op"] in ("mult", "newmult"):
                rid = server.submit_mult(r["ctx"], (r["a"], r["b"]), (r["a2"], r["b2"]), r["level"], r["key"],
                                         r["oa"], r["ob"], arr, new=r["op"] == "newmult")
            else:
                rid = server.submit_keyswitch(r["ctx"], r["a"], r["level"], r["key"], r["oa"], r["ob"], arr)
            ids[rid] = i
            i += 1
        server.step()
        for rid, lat, done in server.poll():
            results[ids.pop(rid)] = (lat, done)
    lats = sorted(v[0] for v in results.values())
    first = t0 + min(r["t_ms"] for r in requests)
    last = max(v[1] for v in results.values())
    span = last - first
    return results, {
        "requests": n,
        "span_ms": span,
        "ops_per_s": n / (span / 1e3) if span > 0 else float("inf"),
        "p50_ms": statistics.median(lats),
        "p99_ms": lats[max(0, math.ceil(0.99 * n) - 1)],
        "mean_ms": statistics.fmean(lats),
        "max_ms": lats[-1],
    }
