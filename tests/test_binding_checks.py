"""Host checks of the binding's argument validation (no GPU).

The library receives bare device pointers, so the binding checks every tensor
(device, dtype, contiguity, size) before its pointer is passed on.  Here the
library is replaced by a recorder and the tensors live on the CPU: correctly
shaped arguments must reach the library call, wrong ones must raise
CkksError(CKKS_EINVAL) before any call that launches work.
"""
import ctypes

import pytest

torch = pytest.importorskip("torch")

from paper_2112_06396_gb300 import ckks  # noqa: E402

N, L, K, DNUM = 16, 6, 3, 2  # alpha = 3
WS_WORDS = 64
U64, I64 = torch.uint64, torch.int64


class Recorder:
    """Stands in for libckks_ks.so: records every call; the workspace-size
    queries answer WS_WORDS words."""

    def __init__(self):
        self.calls = []

    def __getattr__(self, name):
        if not name.startswith("ckks_"):
            raise AttributeError(name)

        def fn(*args):
            self.calls.append(name)
            if name.endswith("workspace_bytes"):
                args[-1]._obj.value = WS_WORDS * 8
            return ckks.CKKS_OK

        return fn


class HostContext(ckks.Context):
    """A Context whose tensors live on the CPU and whose handle is a dummy."""

    def __init__(self):
        self.logN, self.N, self.L, self.k, self.dnum = 4, N, L, K, DNUM
        self.alpha = (L + DNUM - 1) // DNUM
        self.q, self.p = list(range(L)), list(range(L, L + K))
        self.device = torch.device("cpu")
        self._h = ctypes.c_void_p(1)
        self._compressed = {}
        self._ws_bytes = {}

    def close(self):
        self._h = None


class HostServer(ckks.Server):
    def __init__(self, contexts):
        self.contexts = list(contexts)
        self._h = ctypes.c_void_p(2)
        self._keys = []
        self._live = {}

    def close(self):
        self._h = None


class Stream:
    cuda_stream = 0


S = Stream()


@pytest.fixture
def env(monkeypatch):
    rec = Recorder()
    monkeypatch.setattr(ckks, "_lib", rec)
    ctx = HostContext()
    yield ctx, rec
    ctx.close()


def poly(n):
    return torch.zeros((n, N), dtype=U64)


def key(rows=2):
    return torch.zeros((DNUM, rows, L + K, N), dtype=U64) if rows == 2 else torch.zeros((DNUM, L + K, N), dtype=U64)


def test_well_formed_arguments_reach_the_library(env):
    ctx, rec = env
    k = key()
    ctx.ntt(poly(L + K), L, stream=S)
    ctx.intt(poly(L + K), L, 1, 2, stream=S)
    ctx.automorph(poly(4), 5, stream=S)
    ctx.modup(poly(L), L, 0, stream=S)
    ctx.ksk_inner_prod(torch.zeros((ctx.beta(L), L + K, N), dtype=U64), L, k, stream=S)
    ctx.moddown(poly(L + K), L, stream=S)
    ctx.moddown_noalloc(poly(L + K), L, stream=S)
    ctx.pmodup(poly(L), L, stream=S)
    ctx.rescale(poly(L), L, stream=S)
    ctx.keyswitch(poly(L), L, k, stream=S)
    ctx.rotate(poly(L), poly(L), L, 5, k, stream=S)
    ctx.hrotate(poly(L), poly(L), L, [5, 25], [k, k], stream=S)
    ctx.keyswitch_batch([poly(L), poly(3)], [None, poly(3)], [L, 3], [1, 5], [k, k], stream=S)
    ctx.keyswitch_batch([poly(3)], None, [3], None, [key(1)], stream=S, seeds=[7])
    ctx.hrotate_batch([(poly(L), poly(L))], [L], [[(5, k), (25, k)]], stream=S)
    ctx.mult(poly(L), poly(L), poly(L), poly(L), L, k, stream=S)
    ctx.mult_batch([(poly(L), poly(L))], [(poly(L), poly(L))], [L], [k], stream=S)
    ctx.newmult_sum([(poly(L), poly(L))] * 2, [(poly(L), poly(L))] * 2, L, k, stream=S)
    ctx.ptmatvecmult(poly(L), poly(L), L, 2, 2, [1, 5], [1, 25], [None, k], [None, k],
                     [poly(L + K) for _ in range(4)], stream=S)
    s, e = torch.zeros(N, dtype=I64), torch.zeros((DNUM, N), dtype=I64)
    ctx.keygen_ksk(s, e, key(1), 5, stream=S)
    kb = ctx.keygen_ksk_seeded(s, e, 3, 5, stream=S)
    ctx.ksk_expand(kb, 3, stream=S)
    ctx.register_compressed_key(kb, 3)
    assert ctx._compressed[kb.data_ptr()] is kb  # held while registered
    ctx.keyswitch(poly(L), L, kb, stream=S)  # a registered compressed key: rows b_j only
    ctx.unregister_compressed_key(kb)
    assert kb.data_ptr() not in ctx._compressed
    for name in ("ckks_ntt", "ckks_intt", "ckks_automorph", "ckks_modup", "ckks_ksk_inner_prod", "ckks_moddown",
                 "ckks_moddown_noalloc", "ckks_pmodup", "ckks_rescale", "ckks_keyswitch", "ckks_rotate",
                 "ckks_hrotate", "ckks_keyswitch_batch", "ckks_keyswitch_batch_seeded", "ckks_hrotate_batch",
                 "ckks_mult", "ckks_mult_batch", "ckks_newmult_sum", "ckks_ptmatvecmult", "ckks_keygen_ksk",
                 "ckks_keygen_ksk_seeded", "ckks_ksk_expand", "ckks_key_register_seed", "ckks_key_unregister"):
        assert name in rec.calls, name


def _rejected(rec, fn, launch):
    with pytest.raises(ckks.CkksError) as err:
        fn()
    assert err.value.code == ckks.CKKS_EINVAL
    assert launch not in rec.calls


def test_wrong_arguments_are_rejected_before_the_library(env):
    ctx, rec = env
    k = key()
    # a ciphertext with fewer limbs than its level, of the wrong dtype, not
    # contiguous, or on another device
    _rejected(rec, lambda: ctx.keyswitch(poly(L - 1), L, k, stream=S), "ckks_keyswitch")
    _rejected(rec, lambda: ctx.keyswitch(poly(L).to(I64), L, k, stream=S), "ckks_keyswitch")
    _rejected(rec, lambda: ctx.keyswitch(torch.zeros((N, L), dtype=U64).t(), L, k, stream=S), "ckks_keyswitch")
    _rejected(rec, lambda: ctx.keyswitch(torch.zeros((L, N), dtype=U64, device="meta"), L, k, stream=S),
              "ckks_keyswitch")
    _rejected(rec, lambda: ctx.keyswitch(poly(L).numpy(), L, k, stream=S), "ckks_keyswitch")
    # an output too small, a workspace too small
    _rejected(rec, lambda: ctx.keyswitch(poly(L), L, k, u=poly(L - 1), stream=S), "ckks_keyswitch")
    _rejected(rec, lambda: ctx.keyswitch(poly(L), L, k, ws=torch.zeros(WS_WORDS - 1, dtype=U64), stream=S),
              "ckks_keyswitch")
    # a compressed key that is not registered is read as a full key
    _rejected(rec, lambda: ctx.keyswitch(poly(L), L, key(1), stream=S), "ckks_keyswitch")
    # a one-dimensional polynomial would be read as N limbs
    _rejected(rec, lambda: ctx.automorph(torch.zeros(N, dtype=U64), 5, stream=S), "ckks_automorph")
    _rejected(rec, lambda: ctx.ntt(poly(L + K), L, 0, L + K + 1, stream=S), "ckks_ntt")
    # list lengths
    _rejected(rec, lambda: ctx.hrotate(poly(L), poly(L), L, [5, 25], [k], stream=S), "ckks_hrotate")
    _rejected(rec, lambda: ctx.keyswitch_batch([poly(L)], None, [L, 3], None, [k], stream=S),
              "ckks_keyswitch_batch")
    _rejected(rec, lambda: ctx.keyswitch_batch([poly(3)], None, [3], None, [key(1)[:1]], stream=S, seeds=[7]),
              "ckks_keyswitch_batch_seeded")
    _rejected(rec, lambda: ctx.ptmatvecmult(poly(L), poly(L), L, 2, 2, [1, 5], [1, 25], [None, None], [None, k],
                                            [poly(L + K) for _ in range(4)], stream=S), "ckks_ptmatvecmult")
    _rejected(rec, lambda: ctx.ptmatvecmult(poly(L), poly(L), L, 2, 2, [1, 5], [1, 25], [None, k], [None, k],
                                            [poly(L + K) for _ in range(3)], stream=S), "ckks_ptmatvecmult")
    _rejected(rec, lambda: ctx.mult(poly(L), poly(L), poly(L), poly(L - 1), L, k, stream=S), "ckks_mult")
    _rejected(rec, lambda: ctx.keygen_ksk(torch.zeros(N, dtype=U64), torch.zeros((DNUM, N), dtype=I64), key(1), 5,
                                          stream=S), "ckks_keygen_ksk")


def test_server_requests_are_checked(env):
    ctx, rec = env
    srv = HostServer([ctx])
    k = key()
    srv.add_key(0, k)
    srv.submit_hrotate(0, poly(4), poly(4), 4, 5, 0, poly(4), poly(4))
    srv.submit_mult(0, (poly(4), poly(4)), (poly(4), poly(4)), 4, 0, poly(3), poly(3))
    assert rec.calls.count("ckks_server_submit") == 2
    n = len(rec.calls)
    with pytest.raises(ckks.CkksError):
        srv.add_key(0, key(1))  # a compressed key given without its seed
    with pytest.raises(ckks.CkksError):
        srv.submit_keyswitch(0, poly(4), 4, 0, poly(3), poly(4))  # output below the level
    with pytest.raises(ckks.CkksError):
        srv.submit_mult(0, (poly(4), poly(3)), (poly(4), poly(4)), 4, 0, poly(3), poly(3))
    assert len(rec.calls) == n
    srv.submit_keyswitch(5, poly(4), 4, 0, poly(4), poly(4))  # unknown context: left to the library
    assert rec.calls[-1] == "ckks_server_submit"
    srv.close()


def test_tuning_and_scheduling_knobs(env):
    """tune_set takes the 8-int choice that autotune returns (4 widths, 4 radix
    splits) and rejects any other length before the library call; the
    concurrency hint, batch streams and fusion switch reach the library."""
    ctx, rec = env
    ctx.tune_set([0, 2, 1, 0, -1, 0, 1, 0])
    assert rec.calls[-1] == "ckks_tune_set"
    for bad in ([0, 0, 0, 0], [0] * 9, []):
        n = len(rec.calls)
        with pytest.raises(ckks.CkksError):
            ctx.tune_set(bad)
        assert len(rec.calls) == n
    ctx.concurrency_hint(8)
    assert rec.calls[-1] == "ckks_concurrency_hint"
    ctx.batch_streams(2)
    assert rec.calls[-1] == "ckks_batch_streams"
    ctx.fuse_modup(False)
    assert rec.calls[-1] == "ckks_fuse_select"
