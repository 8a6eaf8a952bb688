#!/usr/bin/env python
"""KeySwitch throughput on GB300 at N=2^16, ell=24, k=8, dnum=3.

One step = HRotate (Automorph by 5^r + KeySwitch, Algorithm 4 with r=1) of
each of C independent ciphertexts, each with its own rotation key, so the
step's working set (C x (24 MiB ciphertext + 96 MiB key + 24 MiB output))
is far larger than the 129 MB L2: inputs larger than L2, no flush needed.
Metric: KeySwitch ops/s (C per step).  Inputs are seeded synthetic residues
and keys generated on the GPU from a seeded ternary secret.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Under torchrun each rank runs its own C ciphertexts (weak scaling, no
collective on the data path); the time is the max over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

import synth  # noqa: E402
from paper_2112_06396_gb300 import traffic  # noqa: E402

LOGN, L, K_SP, DNUM, BITS = 16, 24, 8, 3, 54
METRIC = "KeySwitch ops/s at N=2^16, ell=24, dnum=3"
UNIT = "KeySwitch/s"
WORKLOAD = "HRotate(5^r)+KeySwitch N=2^16 ell=24 k=8 dnum=3 54-bit primes"
STREAMS = 8
BATCH_STREAMS = 2  # the library's default split of a batched call (ckks_batch_streams)


def load_peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        with open(path) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "sm_max_mhz": float(d.get("sm_max_mhz", 2070.0)), "src": "measured"}
    return {"hbm_gbs": 6800.0, "sm_max_mhz": 2070.0, "src": "fallback"}


# ------------------------------------------------------------------ clocks
class ClockSampler:
    """nvidia-smi samples of the SM clock and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = os.path.join("/tmp", f"bench_clocks_{os.getpid()}.csv")

    def start(self):
        try:
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits", "-i", str(self.gpu),
                 "-lms", "100"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.fh.close()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [p.strip() for p in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        smax = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": reasons, "samples": len(rows)}


# ------------------------------------------------------------------ workload
def make_workload(ctx, C, rank, torch):
    N = 1 << LOGN
    primes = ctx.q + ctx.p
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    s = synth.ternary(N, f"bench/r{rank}/s")
    ds = dev(s)
    items = []
    for c in range(C):
        g = pow(5, c + 1, 2 * N)
        a_key = np.stack([synth.uniform_residues(primes, N, f"bench/r{rank}/key{c}/a{j}") for j in range(DNUM)])
        e_key = np.stack([synth.gaussian(N, f"bench/r{rank}/key{c}/e{j}") for j in range(DNUM)])
        key = ctx.keygen_ksk(ds, dev(e_key), dev(a_key), g)
        a = dev(synth.uniform_residues(ctx.q, N, f"bench/r{rank}/ct{c}/a"))
        b = dev(synth.uniform_residues(ctx.q, N, f"bench/r{rank}/ct{c}/b"))
        items.append({"g": g, "key": key, "a": a, "b": b, "oa": ctx.empty(L), "ob": ctx.empty(L)})
    torch.cuda.synchronize()
    return items


class Lanes:
    """S CUDA streams, each with its own workspace: independent ciphertexts of a
    step are spread round-robin so their kernels overlap on the GPU."""

    def __init__(self, ctx, S, torch, ckks):
        self.torch = torch
        self.streams = [torch.cuda.Stream() for _ in range(S)]
        self.ws = [ctx.workspace(ckks.OP_HROTATE, L, 1) for _ in range(S)]

    def fork(self):
        ev = self.torch.cuda.current_stream().record_event()
        for s in self.streams:
            s.wait_event(ev)

    def join(self):
        cur = self.torch.cuda.current_stream()
        for s in self.streams:
            cur.wait_stream(s)


def step(ctx, items, lanes):
    lanes.fork()
    for i, it in enumerate(items):
        j = i % len(lanes.streams)
        ctx.hrotate(it["a"], it["b"], L, [it["g"]], [it["key"]], outs=[(it["oa"], it["ob"])], ws=lanes.ws[j],
                    stream=lanes.streams[j])
    lanes.join()


def _timed(torch, fn, reps=5, warm=2):
    for _ in range(warm):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(reps):
        fn()
    e1.record()
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / reps


def _keygen(ctx, torch, s, g, tag):
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    primes = ctx.q + ctx.p
    a_key = np.stack([synth.uniform_residues(primes, N, f"{tag}/a{j}") for j in range(ctx.dnum)])
    e_key = np.stack([synth.gaussian(N, f"{tag}/e{j}") for j in range(ctx.dnum)])
    return ctx.keygen_ksk(s, dev(e_key), dev(a_key), g)


def measure_small_keyswitch(ckks, torch, reps=50):
    """Single KeySwitch at N=2^12, ell=6, k=3, dnum=2, 50-bit primes: latency."""
    ctx = ckks.Context.from_bits(12, 6, 3, 2, 50)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    s = dev(synth.ternary(ctx.N, "bench/small/s"))
    key = _keygen(ctx, torch, s, 0, "bench/small/key")
    a = dev(synth.uniform_residues(ctx.q, ctx.N, "bench/small/a"))
    u, v = ctx.empty(6), ctx.empty(6)
    ws = ctx.workspace(ckks.OP_KEYSWITCH, 6)
    ms = _timed(torch, lambda: ctx.keyswitch(a, 6, key, u, v, ws), reps)
    out = {"shape": "KeySwitch N=2^12 ell=6 k=3 dnum=2 50-bit primes", "us_per_keyswitch": ms * 1e3,
           "keyswitch_per_s": 1e3 / ms,
           "compulsory_bytes": traffic.compulsory_keyswitch_bytes(ctx.N, 6, 3, 6, 2)}
    ctx.close()
    return out


def measure_batched(ctx, ckks, torch, reps=5):
    """64 KeySwitches at levels uniform in {4..24} sharing one key: one batched
    call (one launch per pipeline step) against one-at-a-time calls on one
    stream and the same calls spread over 4 streams."""
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    levels = synth.uniform_ints(64, 4, 24, "batch/levels")
    s = dev(synth.ternary(N, "bench/batch/s"))
    key = _keygen(ctx, torch, s, 0, "bench/batch/key")
    a = [dev(synth.uniform_residues(ctx.q[:ell], N, f"bench/batch/ct{i}")) for i, ell in enumerate(levels)]
    outs = [(ctx.empty(ell), ctx.empty(ell)) for ell in levels]
    ws = ctx.batch_workspace(levels)
    keys = [key] * len(levels)
    by_split = {}
    for nst in (1, 2, 3, 4):  # ckks_batch_streams: the batch cut over this many streams
        ctx.batch_streams(nst)
        t = _timed(torch, lambda: ctx.keyswitch_batch(a, None, levels, None, keys, outs=outs, ws=ws), reps)
        by_split[nst] = {"ms_per_batch": t, "keyswitch_per_s": len(levels) / t * 1e3}
    ctx.batch_streams(BATCH_STREAMS)
    t_batch = _timed(torch, lambda: ctx.keyswitch_batch(a, None, levels, None, keys, outs=outs, ws=ws), reps)
    ws1 = ctx.workspace(ckks.OP_KEYSWITCH, L)

    def serial():
        for i, ell in enumerate(levels):
            ctx.keyswitch(a[i], ell, key, outs[i][0], outs[i][1], ws1)

    t_serial = _timed(torch, serial, reps)
    streams = [torch.cuda.Stream() for _ in range(4)]
    ws4 = [ctx.workspace(ckks.OP_KEYSWITCH, L) for _ in range(4)]

    def four():
        ev = torch.cuda.current_stream().record_event()
        for st in streams:
            st.wait_event(ev)
        for i, ell in enumerate(levels):
            j = i % 4
            ctx.keyswitch(a[i], ell, key, outs[i][0], outs[i][1], ws4[j], stream=streams[j])
        for st in streams:
            torch.cuda.current_stream().wait_stream(st)

    t_four = _timed(torch, four, reps)
    # the batched call captured once in a CUDA graph and replayed
    gst = torch.cuda.Stream()
    with torch.cuda.stream(gst):
        ctx.keyswitch_batch(a, None, levels, None, keys, outs=outs, ws=ws, stream=gst)
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=gst):
        ctx.keyswitch_batch(a, None, levels, None, keys, outs=outs, ws=ws, stream=gst)
    t_graph = _timed(torch, graph.replay, reps)
    # the same batch with the key compressed (rows b only; a regenerated from a seed)
    seed = synth.stream_seed("bench/batch/seed")
    e_key = np.stack([synth.gaussian(N, f"bench/batch/key/e{j}") for j in range(DNUM)])
    key_b = ctx.keygen_ksk_seeded(s, dev(e_key), seed, 0)
    t_comp = _timed(torch, lambda: ctx.keyswitch_batch(a, None, levels, None, [key_b] * len(levels), outs=outs,
                                                       ws=ws, seeds=[seed] * len(levels)), reps)
    ctx.profile(True)
    ctx.profile_reset()
    ctx.keyswitch_batch(a, None, levels, None, keys, outs=outs, ws=ws)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    comp = traffic.compulsory_batch_keyswitch_bytes(N, levels, [0] * len(levels), K_SP, L, DNUM)
    n = len(levels)
    key_b_bytes = key_b.numel() * 8
    del a, outs, ws, ws1, ws4, graph, key_b
    torch.cuda.empty_cache()
    return {"shape": "64 KeySwitch, ell uniform in {4..24} (seeded), N=2^16, k=8, dnum=3, one shared key",
            "levels_sum": sum(levels),
            "batched": {"ms_per_batch": t_batch, "keyswitch_per_s": n / t_batch * 1e3,
                        "batch_streams": BATCH_STREAMS,
                        "launches": sum(v[1] for v in prof.values()),
                        "kernel_ms": {k: v[0] for k, v in prof.items() if v[1]}},
            "by_batch_streams": by_split,
            "graph_replay": {"ms_per_batch": t_graph, "keyswitch_per_s": n / t_graph * 1e3},
            "compressed_key": {"ms_per_batch": t_comp, "keyswitch_per_s": n / t_comp * 1e3,
                               "key_bytes": key_b_bytes},
            "serial_one_stream": {"ms_per_batch": t_serial, "keyswitch_per_s": n / t_serial * 1e3},
            "four_streams": {"ms_per_batch": t_four, "keyswitch_per_s": n / t_four * 1e3},
            "speedup_vs_serial": t_serial / t_batch,
            "compulsory_bytes": comp,
            "hbm_frac_of_measured": comp / (t_batch * 1e-3) / 1e9 / load_peaks()["hbm_gbs"]}


def measure_serving(ctx16, ckks, torch, n_req=400, rates=(2000, 4000, 8000, 16000), slo_ms=25.0):
    """Serving loop: Poisson arrivals of HRotate (r=1) and Mult + relinearisation
    + Rescale (50/50), N in {2^15, 2^16} (equiprobable), ell uniform in {3..24},
    dnum=3, one relinearisation and 4 rotation keys resident per ring degree.
    Continuous batching (up to 64 per batch, 4 streams) against serial
    launches (batch 1, one stream) at the same offered rates."""
    from paper_2112_06396_gb300 import serving

    primes = ctx16.q + ctx16.p  # = 1 mod 2^17, hence valid for N = 2^15 too
    ctx15 = ckks.Context(15, ctx16.q, ctx16.p, DNUM, device=ctx16.device.index)
    ctxs = [ctx15, ctx16]
    gs = [5, 25, 125, 625]
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx16.device)
    keys, cts = [], []
    for c, cx in enumerate(ctxs):
        s = dev(synth.ternary(cx.N, f"bench/serve/{c}/s"))
        keys.append({g: _keygen(cx, torch, s, g, f"bench/serve/{c}/key{g}") for g in [0] + gs})
        cts.append([dev(synth.uniform_residues(cx.q, cx.N, f"bench/serve/{c}/ct{j}")) for j in range(4)])
    ops = synth.uniform_ints(n_req, 0, 1, "bench/serve/op")
    which = synth.uniform_ints(n_req, 0, 1, "bench/serve/ctx")
    levels = synth.uniform_ints(n_req, 3, 24, "bench/serve/level")
    outs = [(ctxs[which[i]].empty(levels[i]), ctxs[which[i]].empty(levels[i])) for i in range(n_req)]
    key_bytes = sum(k.numel() * 8 for kk in keys for k in kk.values())
    budget = key_bytes + (24 << 30)

    def run(rate, max_batch, streams):
        srv = ckks.Server(ctxs, budget, max_batch=max_batch, streams=streams)
        hd = [{g: srv.add_key(c, k) for g, k in keys[c].items()} for c in range(2)]
        t = np.cumsum(synth.exponential_gaps(n_req, 1e3 / rate, f"bench/serve/gaps/{rate}"))
        reqs = []
        for i in range(n_req):
            c, ell = which[i], levels[i]
            a, b, a2, b2 = (x[:ell] for x in cts[c])
            oa, ob = outs[i]
            if ops[i] == 0:
                g = gs[i % len(gs)]
                reqs.append({"t_ms": float(t[i]), "op": "hrotate", "ctx": c, "level": ell, "a": a, "b": b,
                             "galois": g, "key": hd[c][g], "oa": oa, "ob": ob})
            else:
                reqs.append({"t_ms": float(t[i]), "op": "mult", "ctx": c, "level": ell, "a": a, "b": b, "a2": a2,
                             "b2": b2, "key": hd[c][0], "oa": oa[: ell - 1], "ob": ob[: ell - 1]})
        _, st = serving.replay(srv, reqs)
        stats = srv.stats()
        srv.close()
        st["batches"] = stats["batches"]
        return st

    run(4000, 64, 4)  # warm-up (kernel attributes, allocator)
    table = []
    for rate in rates:
        table.append({"offered_per_s": rate, "batched": run(rate, 64, 4), "serial": run(rate, 1, 1)})
    best = {}
    for mode in ("batched", "serial"):
        ok = [r[mode]["ops_per_s"] for r in table if r[mode]["p99_ms"] <= slo_ms]
        best[mode] = max(ok) if ok else None
    ctx15.close()
    del keys, cts, outs
    torch.cuda.empty_cache()
    return {"shape": "Poisson arrivals, 50% HRotate(r=1) / 50% Mult+Relin+Rescale, N in {2^15, 2^16}, "
                     "ell uniform in {3..24}, dnum=3, 5 keys resident per N; batched: up to 64 per batch on 4 "
                     "streams; serial: one request at a time",
            "requests_per_run": n_req, "p99_slo_ms": slo_ms, "by_rate": table,
            "max_ops_per_s_within_slo": best}


def measure_hoisted(ctx, ckks, torch, reps=5, n_ct=4, r=8):
    """Hoisted rotations (Algorithm 4 with r = 8): 4 ciphertexts at N=2^16, ell=24,
    each rotated by 5^1..5^8 with its own 8 keys: one batched call (ModUp once per
    ciphertext, every rotation's inner product and ModDown in one launch per
    step) against ckks_hrotate per ciphertext on 4 streams."""
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    s = dev(synth.ternary(N, "bench/hoist/s"))
    gs = [pow(5, j + 1, 2 * N) for j in range(r)]
    keys = [_keygen(ctx, torch, s, g, f"bench/hoist/k{j}") for j, g in enumerate(gs)]
    cts = [(dev(synth.uniform_residues(ctx.q, N, f"bench/hoist/a{c}")),
            dev(synth.uniform_residues(ctx.q, N, f"bench/hoist/b{c}"))) for c in range(n_ct)]
    rots = [[(g, k) for g, k in zip(gs, keys)] for _ in range(n_ct)]
    outs = [[(ctx.empty(L), ctx.empty(L)) for _ in range(r)] for _ in range(n_ct)]
    t_batch = _timed(torch, lambda: ctx.hrotate_batch(cts, [L] * n_ct, rots, outs=outs), reps)
    streams = [torch.cuda.Stream() for _ in range(4)]
    wss = [ctx.workspace(ckks.OP_HROTATE, L, r) for _ in range(4)]

    def four():
        ev = torch.cuda.current_stream().record_event()
        for st in streams:
            st.wait_event(ev)
        for c in range(n_ct):
            j = c % 4
            ctx.hrotate(cts[c][0], cts[c][1], L, gs, keys, outs=outs[c], ws=wss[j], stream=streams[j])
        for st in streams:
            torch.cuda.current_stream().wait_stream(st)

    t_four = _timed(torch, four, reps)
    nrot = n_ct * r
    comp = (2 * L * n_ct + nrot * 2 * L) * traffic.limb_bytes(N) + r * traffic.key_limbs(L, K_SP, L, DNUM) * \
        traffic.limb_bytes(N)
    del keys, cts, outs, wss
    torch.cuda.empty_cache()
    return {"shape": f"{n_ct} ciphertexts x {r} hoisted rotations (5^1..5^{r}), N=2^16, ell=24, k=8, dnum=3",
            "batched": {"ms": t_batch, "rotations_per_s": nrot / t_batch * 1e3},
            "single_calls_4_streams": {"ms": t_four, "rotations_per_s": nrot / t_four * 1e3},
            "compulsory_bytes": comp,
            "hbm_frac_of_measured": comp / (min(t_batch, t_four) * 1e-3) / 1e9 / load_peaks()["hbm_gbs"]}


def measure_steps(ctx, ckks, torch, reps=10):
    """Each step of the path on its own at N=2^16, ell=24, k=8, dnum=3, with its
    roofline: the transforms in butterflies/s (integer-issue bound), the data
    movers in GB/s of their compulsory bytes against the measured HBM copy rate."""
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    hbm = load_peaks()["hbm_gbs"]
    limb = traffic.limb_bytes(N)
    ext = L + K_SP
    x = dev(synth.uniform_residues(ctx.ext_primes(L) * 4, N, "bench/steps/x"))  # 128 limbs
    out = torch.empty_like(x)
    rows = {}
    t = _timed(torch, lambda: (ctx.ntt(x[:ext], L), ctx.intt(x[:ext], L)), reps)
    bf = 2 * ext * traffic.ntt_butterflies_per_limb(N)
    rows["ntt_intt"] = {"shape": f"forward + inverse of {ext} limbs", "us": t * 1e3, "gbutterfly_per_s": bf / t / 1e6}
    t = _timed(torch, lambda: ctx.automorph(x[:2 * L], 5, out=out[:2 * L]), reps)
    rows["automorph"] = {"shape": f"{2 * L} limbs (a ciphertext), g = 5", "us": t * 1e3,
                         "hbm_frac_of_measured": 2 * 2 * L * limb / (t * 1e-3) / 1e9 / hbm}
    a = x[:L]
    ws_m = ctx.workspace(ckks.OP_MODUP, L)
    dig = ctx.empty(ext)
    t = _timed(torch, lambda: ctx.modup(a, L, 0, out=dig, ws=ws_m), reps)
    rows["modup_one_digit"] = {"shape": f"digit 0 of {L} limbs -> {ext} limbs (8 iNTT, 24 new limbs, 24 NTT)",
                               "us": t * 1e3}
    digits = dev(synth.uniform_residues(ctx.ext_primes(L) * DNUM, N, "bench/steps/d"))
    s = dev(synth.ternary(N, "bench/steps/s"))
    key = _keygen(ctx, torch, s, 0, "bench/steps/key")
    u, v = ctx.empty(ext), ctx.empty(ext)
    t = _timed(torch, lambda: ctx.ksk_inner_prod(digits, L, key, u, v), reps)
    ip_bytes = (DNUM * ext + traffic.key_limbs(L, K_SP, L, DNUM) + 2 * ext) * limb
    rows["ksk_inner_prod"] = {"shape": f"beta=3 digits x {ext} positions, key {traffic.key_limbs(L, K_SP, L, DNUM)} limbs",
                              "us": t * 1e3, "hbm_frac_of_measured": ip_bytes / (t * 1e-3) / 1e9 / hbm}
    ws_d = ctx.workspace(ckks.OP_MODDOWN, L)
    md = ctx.empty(L)
    t = _timed(torch, lambda: ctx.moddown(u, L, out=md, ws=ws_d), reps)
    rows["moddown"] = {"shape": f"{ext} -> {L} limbs (8 iNTT, conversion, 24 NTT + scale)", "us": t * 1e3}

    # the basis conversion alone (measurement hook), on the tensor cores and on
    # the integer units, inside ModUp (8 -> 24 limbs) and ModDown (8 -> 24)
    def conv_us(fn):
        ctx.profile(True)
        ctx.profile_reset()
        for _ in range(reps):
            fn()
        torch.cuda.synchronize()
        ms, n, _ = ctx.profile_read()["bconv"]
        ctx.profile(False)
        return ms / max(n, 1) * 1e3

    conv = {}
    for name, on in (("tensor_cores", True), ("integer_units", False)):
        ctx.bconv_tensor_cores(on)
        conv[name] = {"modup_digit_us": conv_us(lambda: ctx.modup(a, L, 0, out=dig, ws=ws_m)),
                      "moddown_us": conv_us(lambda: ctx.moddown(u, L, out=md, ws=ws_d)),
                      "modup_one_digit_total_us": _timed(torch, lambda: ctx.modup(a, L, 0, out=dig, ws=ws_m), reps) * 1e3,
                      "moddown_total_us": _timed(torch, lambda: ctx.moddown(u, L, out=md, ws=ws_d), reps) * 1e3}
    ctx.bconv_tensor_cores(True)
    rows["basis_conversion"] = {"shape": "8 source limbs -> 24 target limbs of N=2^16 (one ModUp digit; the P "
                                         "limbs of one polynomial in ModDown)", **conv}
    del x, out, digits, key
    torch.cuda.empty_cache()
    return rows


def measure_rotation_sweep(ctx, items, lanes, torch, reps=10):
    """The headline step with every ciphertext rotated by 5^r, r in {1, 2, 2^14}
    (the Automorph gather pattern of the inner product depends on g).  The keys
    of the headline are reused: the arithmetic, hence the time, does not depend
    on them (these outputs are not checked; parity at each g is in the tests)."""
    out = {}
    twoN = 2 << LOGN
    for r in (1, 2, 1 << 14):
        g = pow(5, r, twoN)
        its = [dict(it, g=g) for it in items]
        ms = _timed(torch, lambda: step(ctx, its, lanes), reps)
        out[f"r={r}"] = {"galois": g, "ms_per_step": ms, "keyswitch_per_s": len(items) / ms * 1e3}
    return out


def measure_fused(ctx, ckks, items, lanes, torch, reps=10):
    """The fused key-switching dataflow (ckks_fuse_select: ModUp's last forward
    pass, KSKInnerProd and ModDown's first inverse pass in one kernel) against
    the default kernels: the headline step on the same streams, one HRotate
    alone, and the single KeySwitch at N=2^12."""
    one = Lanes(ctx, 1, torch, ckks)
    it0 = items[0]
    # on the current stream, the one _timed's events are recorded on
    alone = lambda: ctx.hrotate(it0["a"], it0["b"], L, [it0["g"]], [it0["key"]], outs=[(it0["oa"], it0["ob"])],
                                ws=one.ws[0])
    out = {}
    for on in (False, True):
        ctx.fuse_modup(on)
        ms_step = _timed(torch, lambda: step(ctx, items, lanes), reps)
        ctx.concurrency_hint(1)  # a call alone: grids sized for the whole GPU
        ms_one = _timed(torch, alone, 20)
        ctx.concurrency_hint(len(lanes.streams))
        out["fused" if on else "default"] = {"ms_per_step": ms_step, "keyswitch_per_s": len(items) / ms_step * 1e3,
                                              "hrotate_alone_us": ms_one * 1e3,
                                              "launches_per_hrotate": 9 if on else 11}
    ctx.fuse_modup(False)
    small = ckks.Context.from_bits(12, 6, 3, 2, 50)
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(small.device)
    s = dev(synth.ternary(small.N, "bench/small/s"))
    key = _keygen(small, torch, s, 0, "bench/small/key")
    a = dev(synth.uniform_residues(small.q, small.N, "bench/small/a"))
    u, v = small.empty(6), small.empty(6)
    ws = small.workspace(ckks.OP_KEYSWITCH, 6)
    for on in (False, True):
        small.fuse_modup(on)
        ms = _timed(torch, lambda: small.keyswitch(a, 6, key, u, v, ws), 50)
        out["fused" if on else "default"]["small_keyswitch_us"] = ms * 1e3
    small.close()
    return out


def measure_other_rows(ctx, ckks, torch, reps=5):
    """Rescale (Alg. 1's ModDown_{B,1}) of one ciphertext, and a CoeffToSlot-shaped
    PtMatVecMult: fftIter = 3 levels at ell = 24, 23, 22 (Alg. 8 with 8 baby x 4
    giant steps per level, rotation offsets (t*8 + i) * 32^level, 32 seeded
    diagonals over the extended basis per level, 7 baby + 3 giant rotation keys
    per level = 30 keys resident, Rescale after each level), all at N=2^16,
    timed with CUDA events outside the KeySwitch timed region."""
    N = 1 << LOGN
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    a = dev(synth.uniform_residues(ctx.q, N, "bench/rows/a"))
    b = dev(synth.uniform_residues(ctx.q, N, "bench/rows/b"))
    ws_r = ctx.workspace(ckks.OP_RESCALE, L)
    oa, ob = ctx.empty(L - 1), ctx.empty(L - 1)
    rescale_ms = _timed(torch, lambda: (ctx.rescale(a, L, oa, ws_r), ctx.rescale(b, L, ob, ws_r)), reps)

    nb, ng, radix_log = 8, 4, 5
    twoN = 2 * N
    s = dev(synth.ternary(N, "bench/rows/s"))
    levels = []
    for lv in range(3):
        ell = L - lv
        stride = 1 << (radix_log * lv)
        g_baby = [1] + [pow(5, i * stride, twoN) for i in range(1, nb)]
        g_giant = [1] + [pow(5, t * nb * stride, twoN) for t in range(1, ng)]
        kb = [None] + [_keygen(ctx, torch, s, g, f"bench/rows/l{lv}/kb{i}") for i, g in enumerate(g_baby) if i > 0]
        kg = [None] + [_keygen(ctx, torch, s, g, f"bench/rows/l{lv}/kg{t}") for t, g in enumerate(g_giant) if t > 0]
        diags = [dev(synth.uniform_residues(ctx.ext_primes(ell), N, f"bench/rows/l{lv}/M{d}"))
                 for d in range(nb * ng)]
        levels.append((ell, g_baby, g_giant, kb, kg, diags))
    ws_p = ctx.workspace(ckks.OP_PTMATVEC, L, ng)
    bufs = [(a, b)] + [(ctx.empty(L - 1 - i), ctx.empty(L - 1 - i)) for i in range(3)]

    def level(i):
        ell, g_baby, g_giant, kb, kg, diags = levels[i]
        ia, ib = bufs[i]
        pa, pb = bufs[i + 1]
        ctx.ptmatvecmult(ia, ib, ell, nb, ng, g_baby, g_giant, kb, kg, diags, True, pa, pb, ws_p)

    per_level = [_timed(torch, lambda i=i: level(i), reps) for i in range(3)]
    c2s_ms = _timed(torch, lambda: [level(i) for i in range(3)], reps)
    # where the time of the first level goes (measurement hook, one stream)
    ctx.profile(True)
    ctx.profile_reset()
    level(0)
    torch.cuda.synchronize()
    prof_l0 = {k: {"ms": v[0], "launches": v[1]} for k, v in ctx.profile_read().items() if v[1]}
    ctx.profile(False)
    # the same three levels with every rotation key compressed (Sec. 5.3): rows b_j
    # only, a_j regenerated from a seed inside the kernels
    full_levels = levels
    levels = []
    comp_key_bytes = 0
    for lv, (ell, g_baby, g_giant, kb, kg, diags) in enumerate(full_levels):
        def ckey(g, tag):
            nonlocal comp_key_bytes
            sd = synth.stream_seed(f"bench/rows/l{lv}/{tag}/seed")
            e_key = np.stack([synth.gaussian(N, f"bench/rows/l{lv}/{tag}/e{j}") for j in range(DNUM)])
            kbc = ctx.keygen_ksk_seeded(s, dev(e_key), sd, g)
            ctx.register_compressed_key(kbc, sd)
            comp_key_bytes += kbc.numel() * 8
            return kbc
        kbc = [None] + [ckey(g, f"kb{i}") for i, g in enumerate(g_baby) if i > 0]
        kgc = [None] + [ckey(g, f"kg{t}") for t, g in enumerate(g_giant) if t > 0]
        levels.append((ell, g_baby, g_giant, kbc, kgc, diags))
    per_level_c = [_timed(torch, lambda i=i: level(i), reps) for i in range(3)]
    c2s_ms_c = _timed(torch, lambda: [level(i) for i in range(3)], reps)
    for (_e, _gb, _gg, kbc, kgc, _d) in levels:
        for k in kbc[1:] + kgc[1:]:
            ctx.unregister_compressed_key(k)
    del full_levels
    comp = []
    for i, (ell, *_rest) in enumerate(levels):
        comp.append((2 * ell + (nb - 1 + ng - 1) * traffic.key_limbs(ell, K_SP, L, DNUM) + nb * ng * (ell + K_SP)
                     + 2 * (ell - 1)) * traffic.limb_bytes(N))
    hbm = load_peaks()["hbm_gbs"]
    del levels, bufs
    torch.cuda.empty_cache()
    return {
        "rescale": {"ms_per_ciphertext": rescale_ms, "ciphertexts_per_s": 1e3 / rescale_ms,
                    "shape": "2 polys, ell 24 -> 23"},
        "ptmatvecmult": {"shape": "CoeffToSlot-shaped: 3 levels at ell 24, 23, 22; 8 baby x 4 giant steps, "
                                  "stride 32^level, 32 diagonals and 10 keys per level (30 keys), rescaled",
                         "ms_per_level": per_level, "ms_coeff_to_slot": c2s_ms,
                         "level0_kernels": prof_l0,
                         "coeff_to_slot_per_s": 1e3 / c2s_ms,
                         "compressed_keys": {"ms_per_level": per_level_c, "ms_coeff_to_slot": c2s_ms_c,
                                             "coeff_to_slot_per_s": 1e3 / c2s_ms_c,
                                             "resident_key_bytes": comp_key_bytes},
                         "compulsory_bytes_per_level": comp,
                         "hbm_frac_of_measured_per_level": [c / (t * 1e-3) / 1e9 / hbm for c, t in zip(comp, per_level)]},
    }


def ntt_source_hash():
    h = hashlib.sha256()
    for f in ("ntt.cu", "common.cuh", "batch.cuh"):
        with open(os.path.join(ROOT, "paper_2112_06396_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def ncu_traffic_per_limb():
    """DRAM bytes per limb-transform of the NTT kernels from the committed ncu
    summary, if it was taken on the current kernel source (else None)."""
    path = os.path.join(ROOT, "profiles", "ntt_traffic.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        d = json.load(f)
    if d.get("source_hash") != ntt_source_hash():
        return None
    return float(d["dram_bytes_per_limb_transform"])


# ------------------------------------------------------------------ multi-rank helpers
def max_over_ranks(value, dist, device="cpu"):
    """The slowest rank's time (the whole job ends with it); no-op on one rank."""
    if dist is None:
        return value
    import torch

    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def job_throughput(world, per_rank_units_per_step, steps, ms):
    """Units per second of the whole job: every rank processes its own units
    (weak scaling), the time is the max over ranks."""
    return world * per_rank_units_per_step * steps / (ms / 1e3)


# ------------------------------------------------------------------ oracle (CPU) legs
def _oracle_inputs():
    """The oracle's HRotate (r=1) inputs at the bench configuration."""
    import oracle

    N = 1 << LOGN
    primes = oracle.gen_primes(BITS, LOGN, L + K_SP)
    P = oracle.Params(LOGN, L, K_SP, DNUM, primes=primes)
    g = 5
    s = synth.ternary(N, "bench/r0/s")
    a_key = np.stack([synth.uniform_residues(primes, N, f"bench/r0/key0/a{j}") for j in range(DNUM)])
    e_key = np.stack([synth.gaussian(N, f"bench/r0/key0/e{j}") for j in range(DNUM)])
    key = oracle.keygen(P, a_key, s, oracle.rot_secret(P, s, g), e_key)
    a = synth.uniform_residues(primes[:L], N, "bench/r0/ct0/a")
    b = synth.uniform_residues(primes[:L], N, "bench/r0/ct0/b")
    return P, a, b, g, key


def _oracle_worker(job):
    """One process of the all-cores oracle timing: build the inputs, then for
    every round wait for the other processes and run one HRotate; returns the
    (start, end) of each round on the host's monotonic clock."""
    import oracle

    barrier, rounds = job
    P, a, b, g, key = _oracle_inputs()
    out = []
    for _ in range(rounds):
        barrier.wait()
        t0 = time.perf_counter()
        oracle.hrotate(P, L, a, b, [g], [key])
        out.append((t0, time.perf_counter()))
    return out


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def cpu_model():
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for ln in out.splitlines():
            if ln.startswith("Model name:"):
                return ln.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    import platform

    return platform.machine()


def oracle_rounds(procs, rounds):
    """`rounds` rounds of `procs` concurrent oracle HRotates, one process per
    host core (spawned: no process is forked from one that has initialised
    CUDA).  Returns the span of each round (first start to last end) and every
    process's own HRotate time."""
    import multiprocessing as mp

    mpc = mp.get_context("spawn")
    with mpc.Manager() as man:
        barrier = man.Barrier(procs)
        with mpc.Pool(procs) as pool:
            res = pool.map(_oracle_worker, [(barrier, rounds)] * procs)
    spans = [max(r[k][1] for r in res) - min(r[k][0] for r in res) for k in range(rounds)]
    singles = [r[k][1] - r[k][0] for r in res for k in range(rounds)]
    return spans, singles


ORACLE_TASKS = ["config1_keyswitch", "config3_keyswitch_l4", "config3_keyswitch_l14", "config3_keyswitch_l24",
                "config4_ptmatvec_l24_8x1", "config5_hrotate_n15_l24", "config5_mult_n15_l24"]


def _oracle_side_task(name):
    """One single-thread oracle timing of a side configuration (spawned process).
    Keys are uniform residues: the arithmetic, hence the time, does not depend
    on them.  Returns (name, seconds, description)."""
    import oracle

    def setup(logN, ell_max, k, dnum, bits):
        primes = oracle.gen_primes(bits, logN, ell_max + k)
        return oracle.Params(logN, ell_max, k, dnum, primes=primes), primes

    def ukey(P, primes, tag):
        return np.stack([np.stack([synth.uniform_residues(primes, P.N, f"{tag}/{j}/{r}") for r in range(2)])
                         for j in range(P.dnum)])

    def timed(fn):
        t0 = time.perf_counter()
        fn()
        return time.perf_counter() - t0

    if name == "config1_keyswitch":
        P, pr = setup(12, 6, 3, 2, 50)
        key, a = ukey(P, pr, "ot/c1/k"), synth.uniform_residues(pr[:6], P.N, "ot/c1/a")
        return name, timed(lambda: oracle.keyswitch(P, 6, a, key)), "KeySwitch N=2^12 ell=6 k=3 dnum=2"
    if name.startswith("config3_keyswitch_l"):
        ell = int(name.rsplit("_l", 1)[1])
        P, pr = setup(LOGN, L, K_SP, DNUM, BITS)
        key, a = ukey(P, pr, "ot/c3/k"), synth.uniform_residues(pr[:ell], P.N, f"ot/c3/a{ell}")
        return name, timed(lambda: oracle.keyswitch(P, ell, a, key)), f"KeySwitch N=2^16 ell={ell} k=8 dnum=3"
    if name == "config4_ptmatvec_l24_8x1":
        P, pr = setup(LOGN, L, K_SP, DNUM, BITS)
        nb, ng, twoN = 8, 1, 2 << LOGN
        gb = [1] + [pow(5, i, twoN) for i in range(1, nb)]
        kb = [None] + [ukey(P, pr, f"ot/c4/kb{i}") for i in range(1, nb)]
        ext = [int(x) for x in pr[:L]] + [int(x) for x in pr[L:]]
        diags = [synth.uniform_residues(ext, P.N, f"ot/c4/d{i}") for i in range(nb * ng)]
        a, b = synth.uniform_residues(pr[:L], P.N, "ot/c4/a"), synth.uniform_residues(pr[:L], P.N, "ot/c4/b")
        sec = timed(lambda: oracle.ptmatvec(P, L, a, b, nb, ng, gb, [1], kb, [None], diags, True))
        return name, sec, "PtMatVecMult N=2^16 ell=24: 8 baby steps x 1 giant step (a quarter of one level), rescaled"
    if name.startswith("config5_"):
        P, pr = setup(15, L, K_SP, DNUM, BITS)
        key = ukey(P, pr, "ot/c5/k")
        a, b = synth.uniform_residues(pr[:L], P.N, "ot/c5/a"), synth.uniform_residues(pr[:L], P.N, "ot/c5/b")
        if "hrotate" in name:
            return name, timed(lambda: oracle.hrotate(P, L, a, b, [5], [key])), "HRotate(r=1) N=2^15 ell=24"
        a2, b2 = synth.uniform_residues(pr[:L], P.N, "ot/c5/a2"), synth.uniform_residues(pr[:L], P.N, "ot/c5/b2")
        return name, timed(lambda: oracle.mult(P, L, a, b, a2, b2, key)), "Mult+Relin+Rescale N=2^15 ell=24"
    raise ValueError(name)


def oracle_side_rows(procs):
    """Single-thread oracle times of the side configurations, run side by side
    on the host cores (spawned processes)."""
    import multiprocessing as mp

    with mp.get_context("spawn").Pool(min(procs, len(ORACLE_TASKS))) as pool:
        res = pool.map(_oracle_side_task, ORACLE_TASKS)
    return {n: {"seconds": sec, "ops_per_s": 1.0 / sec, "what": what} for n, sec, what in res}


def oracle_baseline(procs, rounds):
    """The cpu_baseline object: the oracle as it stands on every host core."""
    spans, singles = oracle_rounds(procs, rounds)
    span = statistics.mean(spans)
    return {"value": procs / span, "unit": UNIT, "cores": procs, "kind": "oracle",
            "sample": (f"{procs} concurrent oracle HRotate(r=1) runs at N=2^16, ell=24, k=8, dnum=3, one process "
                       f"per host core, {rounds} round(s)"),
            "single_thread_s": statistics.median(singles), "single_thread_value": 1.0 / statistics.median(singles),
            "nproc": host_cores(), "cpu_model": cpu_model()}


def base_config(C):
    return {"workload": WORKLOAD, "ciphertexts_per_step": C, "streams": STREAMS, "rotations_per_ciphertext": 1, "N": 1 << LOGN,
            "ell": L, "k": K_SP, "dnum": DNUM, "prime_bits": BITS, "keys": "one rotation key per ciphertext",
            "l2": "inputs larger than L2 (per-step working set > 1 GB), no flush"}


def run_reference(args, rank, world):
    if rank != 0:
        return 0
    W = min(args.warmup, 1)
    K = max(1, min(args.steps, 2))
    procs = args.oracle_procs or host_cores()
    spans, singles = oracle_rounds(procs, W + K)
    t = statistics.mean(spans[W:])
    value = procs / t
    sample = (f"per step {procs} concurrent oracle HRotate(r=1) runs (one process per host core) at N=2^16, "
              f"ell=24, k=8, dnum=3 ({K} timed steps, {W} warm-up, capped so the run ends in minutes)")
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": K,
            "warmup": W, "ms_per_step": t * 1e3, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "u64", "data": "synthetic", "config": base_config(procs),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": procs, "kind": "oracle", "sample": sample,
                             "single_thread_s": statistics.median(singles[W * procs:]), "nproc": host_cores(),
                             "cpu_model": cpu_model()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------------ GPU arm
def run_gpu(args, rank, world, local_rank):
    import torch

    from paper_2112_06396_gb300 import ckks

    torch.cuda.set_device(local_rank)
    dist = None
    if world > 1:
        import torch.distributed as dist

        dist.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    primes = ckks.ckks_gen_primes(BITS, LOGN, L + K_SP)
    ctx = ckks.Context(LOGN, primes[:L], primes[L:], DNUM, device=local_rank)
    tune_choice, tune_times = [0] * 8, []
    if args.fuse:
        ctx.fuse_modup(True)
    if not args.no_tune:
        tune_choice, tune_times = ctx.autotune(limbs=128)  # NTT tile shapes and radix splits for this GPU (ckks_autotune)
    # the step keeps `streams` HRotates running at once (ckks_concurrency_hint)
    ctx.concurrency_hint(args.streams)
    torch.cuda.synchronize()
    C = args.batch
    items = make_workload(ctx, C, rank, torch)
    lanes = Lanes(ctx, args.streams, torch, ckks)
    N = 1 << LOGN

    def barrier():
        if dist is not None:
            dist.barrier()

    for _ in range(args.warmup):
        step(ctx, items, lanes)
    torch.cuda.synchronize()

    # ---- timed region
    clocks = ClockSampler(local_rank)
    barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.25)  # let the sampler take its first reading
    t_wall0 = time.perf_counter()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(args.steps):
        step(ctx, items, lanes)
    e1.record()
    torch.cuda.synchronize()
    t_wall = time.perf_counter() - t_wall0
    barrier()
    clk = clocks.stop()
    ms = max_over_ranks(e0.elapsed_time(e1), dist, "cuda")
    ms_per_step = ms / args.steps
    value = job_throughput(world, C, args.steps, ms)

    # ---- per-kernel-class device time on the launch stream (measurement hook),
    # one stream so that every bracketed launch runs alone
    lane1 = Lanes(ctx, 1, torch, ckks)
    # one stream, every launch sized for the GPU alone (concurrency hint 1): the
    # kernel classes' shares of a step, with no launch stretched by a grid sized
    # for concurrent work
    ctx.concurrency_hint(1)
    ctx.profile(True)
    ctx.profile_reset()
    prof_steps = max(1, min(args.steps, 10))
    for _ in range(prof_steps):
        step(ctx, items, lane1)
    torch.cuda.synchronize()
    prof = ctx.profile_read()
    ctx.profile(False)
    ctx.concurrency_hint(args.streams)
    launches_per_step = sum(v[1] for v in prof.values()) / prof_steps
    by_class = {k: {"ms_per_step": v[0] / prof_steps, "launches_per_step": v[1] / prof_steps} for k, v in prof.items()}

    # ---- measured ceiling of the butterfly (register-only, every SM)
    ctx.butterfly_peak(rounds=2000)  # warm-up
    bps, bms, nbf = ctx.butterfly_peak(rounds=40000)
    bfly_peak = {"gbfly_s": bps / 1e9, "ms": bms, "butterflies": nbf,
                 "per_sm_per_clock_at_max": bps / (torch.cuda.get_device_properties(local_rank).multi_processor_count
                                                   * load_peaks()["sm_max_mhz"] * 1e6),
                 "kernel": "ckks_butterfly_peak: 16 words/thread in registers, 4 lazy CT stages per round, "
                           "32 warps/SM"}

    # ---- end to end through the public API with host buffers
    pin_in = [(torch.empty((L, N), dtype=torch.uint64).pin_memory(), torch.empty((L, N), dtype=torch.uint64).pin_memory())
              for _ in range(C)]
    pin_out = [(torch.empty((L, N), dtype=torch.uint64).pin_memory(), torch.empty((L, N), dtype=torch.uint64).pin_memory())
               for _ in range(C)]
    for (ha, hb), it in zip(pin_in, items):
        ha.copy_(it["a"].cpu())
        hb.copy_(it["b"].cpu())
    # sets of device inputs and outputs (--e2e-sets), taken in turn by the
    # steps, so that a step's host-to-device copies overlap the previous steps'
    # compute and device-to-host copies; every reuse of a buffer waits (by
    # event) for the last read of it: the HRotate that read an input set, the
    # copy back that read an output set
    NB = max(1, args.e2e_sets)
    dev_in = [[(ctx.empty(L), ctx.empty(L)) for _ in range(C)] for _ in range(NB)]
    dev_out = [[(ctx.empty(L), ctx.empty(L)) for _ in range(C)] for _ in range(NB)]
    in_free = [[None] * C for _ in range(NB)]
    out_free = [[None] * C for _ in range(NB)]

    # copies run on their own streams, in ciphertext order, so the copy engines
    # stream continuously: ciphertext i's HRotate waits only for its own inputs,
    # and its outputs leave as soon as it is done
    h2d, d2h = torch.cuda.Stream(), torch.cuda.Stream()

    # compute streams of the end-to-end run (--e2e-streams; the device-only
    # run's 8 by default)
    lanes_e = Lanes(ctx, args.e2e_streams, torch, ckks)
    ctx.concurrency_hint(args.e2e_streams)

    def e2e_step(s):
        b = s % NB
        lanes = lanes_e
        loaded, done = [], []
        with torch.cuda.stream(h2d):
            for i, ((ha, hb), (da, db)) in enumerate(zip(pin_in, dev_in[b])):
                if in_free[b][i] is not None:
                    h2d.wait_event(in_free[b][i])
                da.copy_(ha, non_blocking=True)
                db.copy_(hb, non_blocking=True)
                loaded.append(h2d.record_event())
        for i, ((da, db), (oa, ob), it) in enumerate(zip(dev_in[b], dev_out[b], items)):
            j = i % len(lanes.streams)
            st = lanes.streams[j]
            st.wait_event(loaded[i])
            if out_free[b][i] is not None:
                st.wait_event(out_free[b][i])
            ctx.hrotate(da, db, L, [it["g"]], [it["key"]], outs=[(oa, ob)], ws=lanes.ws[j], stream=st)
            done.append(st.record_event())
            in_free[b][i] = done[i]
        with torch.cuda.stream(d2h):
            for i, ((ha, hb), (oa, ob)) in enumerate(zip(pin_out, dev_out[b])):
                d2h.wait_event(done[i])
                ha.copy_(oa, non_blocking=True)
                hb.copy_(ob, non_blocking=True)
                out_free[b][i] = d2h.record_event()

    def e2e_run(steps, s0):
        cur = torch.cuda.current_stream()
        ev0 = cur.record_event()
        h2d.wait_event(ev0)
        d2h.wait_event(ev0)
        lanes_e.fork()
        for s in range(steps):
            e2e_step(s0 + s)
        cur.wait_stream(d2h)
        lanes_e.join()

    # the same K steps as the device-only region; the pipeline's fill and drain
    # (one step's copies in, one step's copies out) are inside the timed region
    e2e_steps = max(1, args.steps)
    e2e_run(NB, 0)
    torch.cuda.synchronize()
    barrier()
    f0, f1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    f0.record()
    e2e_run(e2e_steps, 0)
    f1.record()
    torch.cuda.synchronize()
    e2e_ms = max_over_ranks(f0.elapsed_time(f1), dist, "cuda")
    # the step's result is read back on the host: check it matches the device-only run
    ok = all(torch.equal(oa, it["oa"].cpu()) for (oa, _), it in zip(pin_out, items))
    bytes_io = C * 2 * L * N * 8

    if rank == 0:
        peaks = load_peaks()
        # dominant kernel class: NTT (forward + inverse passes)
        ntt_ms = prof["ntt_fwd"][0] + prof["ntt_inv"][0]
        ntt_launch = prof["ntt_fwd"][1] + prof["ntt_inv"][1]
        limb_transforms = (prof["ntt_fwd"][2] + prof["ntt_inv"][2]) / 2  # two passes per transform
        avg_launch_ms = ntt_ms / ntt_launch
        bfly_per_launch = limb_transforms * traffic.ntt_butterflies_per_limb(N) / ntt_launch
        bytes_per_launch = limb_transforms * traffic.ntt_bytes_per_limb(N) / ntt_launch
        achieved_gbfly = bfly_per_launch / (avg_launch_ms * 1e-3) / 1e9
        # ALU peak from unit counts and clock: 152 SMs x 64 32-bit IMAD/clk x f_max,
        # 10 IMADs per Shoup modular multiply (4 for the high word of x*w', 3 for
        # the low word of x*w, 3 for the low word of q*p), one per butterfly.
        peak_gbfly = 152 * 64 * peaks["sm_max_mhz"] * 1e6 / 10 / 1e9
        tr = ncu_traffic_per_limb()
        hbm_achieved = bytes_per_launch / (avg_launch_ms * 1e-3) / 1e9
        # The same kernel class in the timed (multi-stream) regime: its share of
        # the kernel time times the measured step time, against the butterflies
        # of one step.  This time per step is never above ms_per_step.
        share = ntt_ms / sum(v[0] for v in prof.values())
        ntt_ms_in_step = share * ms_per_step
        bfly_per_step = limb_transforms / prof_steps * traffic.ntt_butterflies_per_limb(N)
        achieved_in_step = bfly_per_step / (ntt_ms_in_step * 1e-3) / 1e9
        ks_bytes = traffic.compulsory_hrotate_bytes(N, L, K_SP, L, DNUM, 1)
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "u64", "data": "synthetic (seeded residues; keys from a seeded ternary secret)",
            "config": {**base_config(C), "parallelism": f"replicas x{world}", "fused_dataflow": bool(args.fuse),
                       "concurrency_hint": args.streams,
                       "ntt_tile_shapes": {"choice": tune_choice, "ms": [round(t, 4) for t in tune_times],
                                           "legend": "[column pass <=48 limbs, column pass larger, block pass <=48, "
                                                     "block pass larger]: 0 default width, 1 half, 2 double; then "
                                                     "radix split [forward <=48, forward larger, inverse <=48, "
                                                     "inverse larger]: block pass floor(logN/2)+split stages"}},
            "clocks": clk, "gpu_launches": int(round(launches_per_step * args.steps)),
            "wall_s_timed": t_wall,
            "hbm": {"compulsory_bytes_per_keyswitch": ks_bytes,
                    "achieved_gbs": ks_bytes * value / world / 1e9,
                    "frac_of_8tbs": ks_bytes * value / world / 8e12,
                    "frac_of_measured": ks_bytes * value / world / 1e9 / peaks["hbm_gbs"]},
            "roofline": {"kernel": "ntt (forward+inverse passes)", "bound": "alu", "achieved": achieved_gbfly,
                         "peak": peak_gbfly, "unit": "Gbutterfly/s", "frac": achieved_gbfly / peak_gbfly,
                         "peak_how": "152 SMs x 64 IMAD/clk x sm_max_mhz / 10 IMAD per butterfly",
                         "measured_peak": bfly_peak["gbfly_s"],
                         "frac_of_measured_peak": achieved_gbfly / bfly_peak["gbfly_s"],
                         "measured_peak_how": bfly_peak,
                         "in_step": {"ntt_ms_per_step": ntt_ms_in_step, "ms_per_step": ms_per_step,
                                     "butterflies_per_step": bfly_per_step, "achieved": achieved_in_step,
                                     "frac": achieved_in_step / peak_gbfly,
                                     "frac_of_measured_peak": achieved_in_step / bfly_peak["gbfly_s"],
                                     "how": "share of kernel time (one-stream hook, launches sized for the GPU "
                                            "alone) x ms_per_step of the timed multi-stream region"},
                         "traffic": None if tr is None else tr * limb_transforms / ntt_launch,
                         "algorithmic_bytes_per_launch": bytes_per_launch, "hbm_gbs_achieved": hbm_achieved,
                         "hbm_frac_of_measured": hbm_achieved / peaks["hbm_gbs"], "peak_src": peaks["src"],
                         "avg_launch_us": avg_launch_ms * 1e3,
                         "share_of_kernel_time": share},
            "kernels": by_class,
            "e2e": {"value": job_throughput(world, C, e2e_steps, e2e_ms), "unit": UNIT, "compute_streams": args.e2e_streams,
                    "buffer_sets": NB, "concurrency_hint": args.e2e_streams,
                    "steps": e2e_steps, "h2d_bytes_per_step": bytes_io,
                    "d2h_bytes_per_step": bytes_io, "matches_device_result": ok},
        }
        if not args.no_rows:
            ctx.concurrency_hint(args.streams)  # the headline step again
            sweep = measure_rotation_sweep(ctx, items, lanes, torch)
            fused = measure_fused(ctx, ckks, items, lanes, torch)
            del items, lanes, lane1, lanes_e, dev_in, dev_out
            torch.cuda.empty_cache()
            ctx.concurrency_hint(1)  # the other rows: calls alone or batched calls
            line["other_rows"] = measure_other_rows(ctx, ckks, torch)
            line["other_rows"]["rotation_sweep"] = sweep
            line["other_rows"]["fused_dataflow"] = fused
            line["other_rows"]["batched_keyswitch"] = measure_batched(ctx, ckks, torch)
            line["other_rows"]["small_keyswitch"] = measure_small_keyswitch(ckks, torch)
            line["other_rows"]["hoisted_rotations"] = measure_hoisted(ctx, ckks, torch)
            line["other_rows"]["steps"] = measure_steps(ctx, ckks, torch)
            line["other_rows"]["serving"] = measure_serving(ctx, ckks, torch)
        if world == 1 and not args.no_cpu_baseline:
            line["cpu_baseline"] = oracle_baseline(args.oracle_procs or host_cores(), 1)
            if not args.no_rows:
                line["other_rows"]["oracle_single_thread"] = oracle_side_rows(args.oracle_procs or host_cores())
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.barrier()
        dist.destroy_process_group()
    return 0


def run_profile_batch(args):
    """A small case for ncu: `--profile-batch n` batched KeySwitches at levels
    uniform in {4..24} (the first n of the 64-entry workload), one shared key
    (compressed, rows b only, with `--profile-compressed`), `--warmup` +
    `--steps` calls; nothing is printed but a completion line."""
    import torch

    from paper_2112_06396_gb300 import ckks

    primes = ckks.ckks_gen_primes(BITS, LOGN, L + K_SP)
    ctx = ckks.Context(LOGN, primes[:L], primes[L:], DNUM)
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    levels = synth.uniform_ints(64, 4, 24, "batch/levels")[:args.profile_batch]
    s = dev(synth.ternary(N, "bench/batch/s"))
    seeds = None
    if args.profile_compressed:
        seed = synth.stream_seed("bench/batch/seed")
        e_key = np.stack([synth.gaussian(N, f"bench/batch/key/e{j}") for j in range(DNUM)])
        key = ctx.keygen_ksk_seeded(s, dev(e_key), seed, 0)
        seeds = [seed] * len(levels)
    else:
        key = _keygen(ctx, torch, s, 0, "bench/batch/key")
    a = [dev(synth.uniform_residues(ctx.q[:ell], N, f"bench/batch/ct{i}")) for i, ell in enumerate(levels)]
    outs = [(ctx.empty(ell), ctx.empty(ell)) for ell in levels]
    ws = ctx.batch_workspace(levels)
    for _ in range(args.warmup + args.steps):
        ctx.keyswitch_batch(a, None, levels, None, [key] * len(levels), outs=outs, ws=ws, seeds=seeds)
    torch.cuda.synchronize()
    print(f"profile case done: {len(levels)} batched KeySwitches, levels {levels}, "
          f"{'compressed' if seeds else 'full'} key", flush=True)
    return 0


def run_profile_pmv(args):
    """A small case for ncu: `--profile-pmv` runs the first CoeffToSlot-shaped
    PtMatVecMult level (ell=24, 8 baby x 4 giant steps, 32 diagonals, 10 keys)
    `--warmup` + `--steps` times; nothing is printed but a completion line."""
    import torch

    from paper_2112_06396_gb300 import ckks

    primes = ckks.ckks_gen_primes(BITS, LOGN, L + K_SP)
    ctx = ckks.Context(LOGN, primes[:L], primes[L:], DNUM)
    N = ctx.N
    dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(ctx.device)
    nb, ng = 8, 4
    s = dev(synth.ternary(N, "bench/rows/s"))
    g_baby = [1] + [pow(5, i, 2 * N) for i in range(1, nb)]
    g_giant = [1] + [pow(5, t * nb, 2 * N) for t in range(1, ng)]
    kb = [None] + [_keygen(ctx, torch, s, g, f"bench/rows/l0/kb{i}") for i, g in enumerate(g_baby) if i > 0]
    kg = [None] + [_keygen(ctx, torch, s, g, f"bench/rows/l0/kg{t}") for t, g in enumerate(g_giant) if t > 0]
    diags = [dev(synth.uniform_residues(ctx.ext_primes(L), N, f"bench/rows/l0/M{d}")) for d in range(nb * ng)]
    a = dev(synth.uniform_residues(ctx.q, N, "bench/rows/a"))
    b = dev(synth.uniform_residues(ctx.q, N, "bench/rows/b"))
    oa, ob = ctx.empty(L - 1), ctx.empty(L - 1)
    ws = ctx.workspace(ckks.OP_PTMATVEC, L, ng)
    for _ in range(args.warmup + args.steps):
        ctx.ptmatvecmult(a, b, L, nb, ng, g_baby, g_giant, kb, kg, diags, True, oa, ob, ws)
    torch.cuda.synchronize()
    print(f"profile case done: {args.warmup + args.steps} PtMatVecMult levels at ell={L}", flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--batch", type=int, default=16, help="ciphertexts (each with its own key) per step")
    ap.add_argument("--streams", type=int, default=8, help="CUDA streams the independent ciphertexts are spread over")
    ap.add_argument("--e2e-streams", type=int, default=8,
                    help="compute streams of the end-to-end measurement (host copies run on two more)")
    ap.add_argument("--e2e-sets", type=int, default=3,
                    help="sets of device input and output buffers the end-to-end steps rotate through")
    ap.add_argument("--impl", default="gpu", choices=["gpu", "reference"])
    ap.add_argument("--oracle-procs", type=int, default=0,
                    help="oracle processes for the CPU baseline and the reference arm (0: one per host core)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-rows", action="store_true", help="skip the Rescale / PtMatVecMult side measurements")
    ap.add_argument("--no-tune", action="store_true", help="keep the default NTT tile shapes (no autotuning)")
    ap.add_argument("--profile-pmv", action="store_true",
                    help="profiling case: only run PtMatVecMult levels (no JSON line)")
    ap.add_argument("--fuse", action="store_true",
                    help="run the headline's HRotates through the fused ModUp tail + KSKInnerProd kernel")
    ap.add_argument("--profile-batch", type=int, default=0,
                    help="profiling case: only run this many batched KeySwitches at uneven levels (no JSON line)")
    ap.add_argument("--profile-compressed", action="store_true",
                    help="with --profile-batch: the shared key compressed (rows b only, a from a seed)")
    args = ap.parse_args()
    global STREAMS
    STREAMS = args.streams
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", str(args.gpus if args.impl == "reference" else 1)))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        return run_reference(args, rank, world)
    if args.warmup < 3:
        args.warmup = 3
    if args.profile_batch:
        return run_profile_batch(args)
    if args.profile_pmv:
        return run_profile_pmv(args)
    return run_gpu(args, rank, world, local_rank)


if __name__ == "__main__":
    sys.exit(main())
