"""The benchmark's own launch configuration against the oracle.

The headline step is run exactly as bench.py times it: 16 HRotates (Alg. 4,
r = 1, Galois element 5^(c+1) for ciphertext c) at N=2^16, ell=24, k=8,
dnum=3 with 54-bit primes, one rotation key per ciphertext generated on the
GPU, the ciphertexts spread over 8 streams with a workspace each, NTT tile
shapes autotuned, the concurrency hint at the stream count, the tensor-core
basis conversion on.  Every step must give
the same bits, and sampled ciphertexts (first, middle, last) must equal the
oracle bit for bit, keys included.
"""
import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

SAMPLES = (0, 7, 15)


def test_bench_step_matches_oracle(oracle_lib):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2112_06396_gb300 import ckks

    o = oracle_lib
    L = bench.L
    primes = ckks.ckks_gen_primes(bench.BITS, bench.LOGN, L + bench.K_SP)
    assert primes == o.gen_primes(bench.BITS, bench.LOGN, L + bench.K_SP)
    ctx = ckks.Context(bench.LOGN, primes[:L], primes[L:], bench.DNUM)
    ctx.autotune(limbs=128)
    ctx.concurrency_hint(bench.STREAMS)
    items = bench.make_workload(ctx, 16, 0, torch)
    lanes = bench.Lanes(ctx, bench.STREAMS, torch, ckks)

    bench.step(ctx, items, lanes)
    torch.cuda.synchronize()
    first = [(it["oa"].cpu().numpy().copy(), it["ob"].cpu().numpy().copy()) for it in items]
    for _ in range(3):
        bench.step(ctx, items, lanes)
    torch.cuda.synchronize()
    for c, (it, (fa, fb)) in enumerate(zip(items, first)):
        assert np.array_equal(it["oa"].cpu().numpy(), fa), c
        assert np.array_equal(it["ob"].cpu().numpy(), fb), c
    assert ctx.poll_status()

    P = o.Params(bench.LOGN, L, bench.K_SP, bench.DNUM, primes=primes)
    N = P.N
    s = synth.ternary(N, "bench/r0/s")
    for c in SAMPLES:
        it = items[c]
        g = pow(5, c + 1, 2 * N)
        assert it["g"] == g
        a_key = np.stack([synth.uniform_residues(primes, N, f"bench/r0/key{c}/a{j}") for j in range(P.dnum)])
        e_key = np.stack([synth.gaussian(N, f"bench/r0/key{c}/e{j}") for j in range(P.dnum)])
        key = o.keygen(P, a_key, s, o.rot_secret(P, s, g), e_key)
        np.testing.assert_array_equal(it["key"].cpu().numpy(), key)
        a = synth.uniform_residues(primes[:L], N, f"bench/r0/ct{c}/a")
        b = synth.uniform_residues(primes[:L], N, f"bench/r0/ct{c}/b")
        (ra, rb), = o.hrotate(P, L, a, b, [g], [key])
        np.testing.assert_array_equal(first[c][0], ra)
        np.testing.assert_array_equal(first[c][1], rb)


@pytest.mark.parametrize("choice", [[0, 0, 0, 0, 0, 0, 0, 0], [1, 1, 1, 1, 0, 0, 0, 0], [2, 2, 1, 0, 0, 0, 0, 0],
                                    [0, 0, 0, 0, -1, -1, -1, -1], [0, 0, 0, 0, 1, 1, 1, 1]])
def test_concurrent_streams_equal_one_at_a_time(choice):
    """Sixteen HRotates on 8 streams, repeated, against the same HRotates run
    one at a time, for several NTT tile shapes and radix splits.  The
    tensor-core conversion keeps a ring of source stages per CTA; with other
    kernels sharing the SMs (the small tile shapes put the most CTAs beside it)
    a stage handed back too early was overwritten before it was fully read.
    Every output of every step must carry the one-at-a-time bits (tolerance 0)."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    from paper_2112_06396_gb300 import ckks

    L = bench.L
    primes = ckks.ckks_gen_primes(bench.BITS, bench.LOGN, L + bench.K_SP)
    ctx = ckks.Context(bench.LOGN, primes[:L], primes[L:], bench.DNUM)
    ctx.tune_set(choice)
    ctx.concurrency_hint(bench.STREAMS)
    items = bench.make_workload(ctx, 16, 0, torch)
    one = bench.Lanes(ctx, 1, torch, ckks)
    ref = []
    for it in items:
        ctx.hrotate(it["a"], it["b"], L, [it["g"]], [it["key"]], outs=[(it["oa"], it["ob"])], ws=one.ws[0])
        torch.cuda.synchronize()
        ref.append((it["oa"].clone(), it["ob"].clone()))
    lanes = bench.Lanes(ctx, bench.STREAMS, torch, ckks)
    bad = []
    for s in range(16):
        for it in items:
            it["oa"].zero_()
            it["ob"].zero_()
        bench.step(ctx, items, lanes)
        torch.cuda.synchronize()
        bad += [(s, c) for c, it in enumerate(items)
                if not (torch.equal(it["oa"], ref[c][0]) and torch.equal(it["ob"], ref[c][1]))]
    assert not bad, f"(step, ciphertext) with wrong bits: {bad[:10]}"
    assert ctx.poll_status()
