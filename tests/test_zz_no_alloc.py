"""ckks_moddown_noalloc: ModDown for callers that cannot allocate device memory.

Some callers have no way to hand the library a workspace (they run inside a
framework that owns all device memory, or must not allocate after start-up);
this entry point keeps its scratch in a fixed array inside the library.  The
test calls it through the C ABI twice in a row, with different inputs, and
checks each result against the existing ckks_moddown entry point and against
the oracle's ModDown (the division by P with rounding of Sec. 2.4), bit for bit
(the tolerance of every parity test here is 0: the arithmetic is exact).
It also checks that a request larger than the fixed array is refused.

This file is named to run last, so a stop-at-first-failure run has already run
everything else; it also passes on its own in a fresh process.
"""
import ctypes

import numpy as np
import pytest

import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu


def _ckks():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2112_06396_gb300 import ckks

    return ckks


def _noalloc(ckks, ctx, x, level, out):
    """Call the new entry point directly through the C ABI."""
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    return ckks.lib().ckks_moddown_noalloc(ctx.handle, ctypes.c_void_p(x.data_ptr()), level,
                                           ctypes.c_void_p(out.data_ptr()), stream)


@pytest.mark.parametrize("logN,L,k,dnum,bits,level", [(16, 24, 8, 3, 54, 24), (12, 6, 3, 2, 50, 5)])
def test_moddown_noalloc_matches_moddown_twice(oracle_lib, logN, L, k, dnum, bits, level):
    ckks = _ckks()
    ctx = ckks.Context.from_bits(logN, L, k, dnum, bits)
    P = oracle_lib.Params(logN, L, k, dnum, primes=list(ctx.q) + list(ctx.p))
    ext = ctx.ext_primes(level)
    for call in range(2):
        xh = synth.uniform_residues(ext, ctx.N, f"noalloc/{logN}/{call}")
        x = torch.from_numpy(xh).cuda()
        want = ctx.moddown(x, level)
        got = torch.full((level, ctx.N), 7, dtype=torch.uint64, device="cuda")
        assert _noalloc(ckks, ctx, x, level, got) == ckks.CKKS_OK
        torch.cuda.synchronize()
        g = got.cpu().numpy()
        assert np.array_equal(g, want.cpu().numpy()), f"call {call} vs ckks_moddown"
        assert np.array_equal(g, oracle_lib.moddown(P, level, xh)), f"call {call} vs the oracle"


def test_moddown_noalloc_rejects_oversize():
    ckks = _ckks()
    ctx = ckks.Context.from_bits(17, 24, 8, 3, 54)  # (24 + 8) * 2^17 words > 2^21
    x = torch.zeros((32, ctx.N), dtype=torch.uint64, device="cuda")
    out = torch.zeros((24, ctx.N), dtype=torch.uint64, device="cuda")
    assert _noalloc(ckks, ctx, x, 24, out) == ckks.CKKS_EUNSUPPORTED
    with pytest.raises(ckks.CkksError, match="exceeds"):
        ctx.moddown_noalloc(x, 24, out)
    torch.cuda.synchronize()
    assert bool((out.cpu().numpy() == 0).all())  # nothing was launched
