"""Thin ctypes binding of the C ABI in include/ckks_ks.h.

Argument marshalling only: every step of the key-switching path runs in the
CUDA kernels of libckks_ks.so.  PyTorch supplies device memory (uint64 tensors)
and streams.  There is no CPU fallback: if the library is missing, importing
the binding raises.

The module-level functions carry the C names (``ckks_ntt`` ...); the
:class:`Context` class wraps a context handle and allocates workspace with
torch.  All tensors are torch.uint64, contiguous, limb-major [nlimbs][N] on the
context's device.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p
_i = ctypes.c_int
_lib = None

CKKS_OK, CKKS_EINVAL, CKKS_ENOMEM, CKKS_ECUDA, CKKS_EUNSUPPORTED, CKKS_ETIMEOUT = 0, 1, 2, 3, 4, 5
(OP_MODUP, OP_MODDOWN, OP_KEYSWITCH, OP_ROTATE, OP_HROTATE, OP_RESCALE, OP_PTMATVEC, OP_KEYGEN, OP_MULT,
 OP_NEWMULT, OP_KEYGEN_SEEDED) = range(1, 12)


class CkksError(RuntimeError):
    """A status other than CKKS_OK; .code holds it."""

    def __init__(self, msg, code=None):
        super().__init__(msg)
        self.code = code


class _Params(ctypes.Structure):
    _fields_ = [("logN", _i), ("L", _i), ("k", _i), ("dnum", _i), ("q", _u64p), ("p", _u64p)]


REQ_HROTATE, REQ_MULT, REQ_KEYSWITCH, REQ_NEWMULT = 1, 2, 3, 4


class _Request(ctypes.Structure):
    _fields_ = [("op", _i), ("ctx", _i), ("level", _i), ("a", _vp), ("b", _vp), ("a2", _vp), ("b2", _vp),
                ("galois", ctypes.c_uint32), ("key", _i), ("oa", _vp), ("ob", _vp), ("arrival_ms", ctypes.c_double)]


class _Stats(ctypes.Structure):
    _fields_ = [("pending", _i), ("in_flight", _i), ("finished_unpolled", _i), ("lanes_busy", _i),
                ("mem_budget", ctypes.c_size_t), ("mem_keys", ctypes.c_size_t), ("mem_in_flight", ctypes.c_size_t),
                ("batches", ctypes.c_longlong), ("requests_launched", ctypes.c_longlong), ("last_cuda_error", _i)]


_SIGS = {
    "ckks_strerror": (ctypes.c_char_p, [_i]),
    "ckks_gen_primes": (_i, [_i, _i, _i, _u64p]),
    "ckks_ctx_create": (_i, [ctypes.POINTER(_Params), _i, ctypes.POINTER(_vp)]),
    "ckks_ctx_destroy": (_i, [_vp]),
    "ckks_last_cuda_error": (_i, [_vp]),
    "ckks_ctx_table_bytes": (ctypes.c_size_t, [_vp]),
    "ckks_workspace_bytes": (_i, [_vp, _i, _i, _i, ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_ntt": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "ckks_intt": (_i, [_vp, _vp, _i, _i, _i, _vp]),
    "ckks_automorph": (_i, [_vp, _vp, _vp, _i, ctypes.c_uint32, _vp]),
    "ckks_modup": (_i, [_vp, _vp, _i, _i, _vp, _vp, _vp]),
    "ckks_ksk_inner_prod": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp]),
    "ckks_moddown": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "ckks_pmodup": (_i, [_vp, _vp, _i, _vp, _vp]),
    "ckks_rescale": (_i, [_vp, _vp, _i, _vp, _vp, _vp]),
    "ckks_keyswitch": (_i, [_vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "ckks_rotate": (_i, [_vp, _vp, _vp, _i, ctypes.c_uint32, _vp, _vp, _vp, _vp, _vp]),
    "ckks_hrotate": (_i, [_vp, _vp, _vp, _i, _i, ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_vp),
                          ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]),
    "ckks_ptmatvecmult": (_i, [_vp, _vp, _vp, _i, _i, _i, ctypes.POINTER(ctypes.c_uint32),
                               ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                               ctypes.POINTER(_vp), _i, _vp, _vp, _vp, _vp]),
    "ckks_keygen_ksk": (_i, [_vp, _vp, _vp, _vp, ctypes.c_uint32, _vp, _vp, _vp]),
    "ckks_batch_workspace_bytes": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_keyswitch_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i),
                                  ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                  ctypes.POINTER(_vp), _vp, _vp]),
    "ckks_mult": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "ckks_mult_batch_workspace_bytes": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_newmult": (_i, [_vp, _vp, _vp, _vp, _vp, _i, _vp, _vp, _vp, _vp, _vp]),
    "ckks_hrotate_batch_workspace_bytes": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                                                ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_hrotate_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i),
                                ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_vp),
                                ctypes.POINTER(_vp), ctypes.POINTER(_vp), _vp, _vp]),
    "ckks_newmult_sum": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                              ctypes.POINTER(_vp), _i, _vp, _vp, _vp, _vp, _vp]),
    "ckks_newmult_batch_workspace_bytes": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_newmult_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                ctypes.POINTER(_vp), _vp, _vp]),
    "ckks_mult_batch": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                             ctypes.POINTER(_vp), ctypes.POINTER(_i), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                             ctypes.POINTER(_vp), _vp, _vp]),
    "ckks_moddown_noalloc": (_i, [_vp, _vp, _i, _vp, _vp]),
    "ckks_server_create": (_i, [ctypes.POINTER(_vp), _i, ctypes.c_size_t, _i, _i, ctypes.POINTER(_vp)]),
    "ckks_server_destroy": (_i, [_vp]),
    "ckks_server_add_key": (_i, [_vp, _i, _vp, ctypes.POINTER(_i)]),
    "ckks_poll_status": (_i, [_vp, _vp, ctypes.POINTER(_i)]),
    "ckks_autotune": (_i, [_vp, _vp, ctypes.c_size_t, _vp, ctypes.POINTER(_i), ctypes.POINTER(ctypes.c_float)]),
    "ckks_tune_set": (_i, [_vp, ctypes.POINTER(_i)]),
    "ckks_bconv_select": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "ckks_selftest_bounded_wait": (_i, [_vp, ctypes.c_uint32, _vp]),
    "ckks_server_add_key_seeded": (_i, [_vp, _i, _vp, ctypes.c_uint64, ctypes.POINTER(_i)]),
    "ckks_keygen_ksk_seeded": (_i, [_vp, _vp, _vp, ctypes.c_uint64, ctypes.c_uint32, _vp, _vp, _vp]),
    "ckks_ksk_expand": (_i, [_vp, _vp, ctypes.c_uint64, _vp, _vp]),
    "ckks_key_register_seed": (_i, [_vp, _vp, ctypes.c_uint64]),
    "ckks_key_unregister": (_i, [_vp, _vp]),
    "ckks_keyswitch_batch_seeded": (_i, [_vp, _i, ctypes.POINTER(_vp), ctypes.POINTER(_vp), ctypes.POINTER(_i),
                                         ctypes.POINTER(ctypes.c_uint32), ctypes.POINTER(_vp),
                                         ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(_vp), ctypes.POINTER(_vp),
                                         _vp, _vp]),
    "ckks_server_now_ms": (ctypes.c_double, [_vp]),
    "ckks_server_submit": (_i, [_vp, ctypes.POINTER(_Request), ctypes.POINTER(ctypes.c_uint64)]),
    "ckks_server_step": (_i, [_vp, ctypes.POINTER(_i)]),
    "ckks_server_poll": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_uint64), ctypes.POINTER(ctypes.c_double),
                              ctypes.POINTER(ctypes.c_double), ctypes.POINTER(_i), ctypes.POINTER(_i)]),
    "ckks_server_selftest_timeout": (_i, [_vp, ctypes.c_uint32]),
    "ckks_fuse_select": (_i, [_vp, _i, ctypes.POINTER(_i)]),
    "ckks_batch_streams": (_i, [_vp, _i]),
    "ckks_concurrency_hint": (_i, [_vp, _i]),
    "ckks_butterfly_peak_sink_bytes": (_i, [_vp, ctypes.POINTER(ctypes.c_size_t)]),
    "ckks_butterfly_peak": (_i, [_vp, _i, _vp, _vp, ctypes.POINTER(ctypes.c_float),
                                 ctypes.POINTER(ctypes.c_double)]),
    "ckks_server_stats": (_i, [_vp, ctypes.POINTER(_Stats)]),
    "ckks_profile_enable": (_i, [_vp, _i]),
    "ckks_profile_reset": (_i, [_vp]),
    "ckks_profile_read": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_longlong),
                               ctypes.POINTER(ctypes.c_double)]),
}

K_NTT_FWD, K_NTT_INV, K_BCONV, K_INNER, K_PMV, K_ELEMWISE = range(6)
K_NAMES = ["ntt_fwd", "ntt_inv", "bconv", "inner_prod", "pmv_accum", "elementwise", "fused_modup_ip"]


def library_path() -> str:
    return _build.LIB


def lib():
    """Load libckks_ks.so (built in-tree by ``build.build()``); raise if absent."""
    global _lib
    if _lib is None:
        path = _build.LIB
        if not os.path.exists(path):
            raise CkksError(f"{path} is missing: run paper_2112_06396_gb300.build.build() (needs nvcc)")
        L = ctypes.CDLL(path)
        for name, (res, args) in _SIGS.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def exported_symbols():
    return list(_SIGS)


def _check(rc, ctx=None):
    if rc != CKKS_OK:
        msg = lib().ckks_strerror(rc).decode()
        if ctx is not None and rc == CKKS_ECUDA:
            msg += f" (cudaError {lib().ckks_last_cuda_error(ctx)})"
        raise CkksError(msg, rc)


def _p(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    if stream is None:
        stream = torch.cuda.current_stream()
    return ctypes.c_void_p(stream.cuda_stream)


def ckks_gen_primes(bits: int, logN: int, count: int) -> list[int]:
    out = (ctypes.c_uint64 * count)()
    _check(lib().ckks_gen_primes(bits, logN, count, out))
    return [int(x) for x in out]


class Context:
    """One parameter set on one device: N = 2^logN, chain q (L primes),
    special primes p (k primes), dnum digits."""

    def __init__(self, logN, q, p, dnum, device=0):
        self.logN, self.L, self.k, self.dnum = int(logN), len(q), len(p), int(dnum)
        self.N = 1 << self.logN
        # registered compressed keys by data pointer; holding the tensor keeps its
        # memory from being reused by another key while the library treats that
        # address as compressed
        self._compressed = {}
        self._ws_bytes = {}  # (op, level, r) -> ckks_workspace_bytes
        self.q, self.p = [int(x) for x in q], [int(x) for x in p]
        self.device = torch.device("cuda", device)
        qa = (ctypes.c_uint64 * self.L)(*self.q)
        pa = (ctypes.c_uint64 * self.k)(*self.p)
        prm = _Params(self.logN, self.L, self.k, self.dnum, ctypes.cast(qa, _u64p), ctypes.cast(pa, _u64p))
        h = ctypes.c_void_p()
        _check(lib().ckks_ctx_create(ctypes.byref(prm), device, ctypes.byref(h)))
        self._h = h
        self.alpha = (self.L + self.dnum - 1) // self.dnum

    @classmethod
    def from_bits(cls, logN, L, k, dnum, bits, device=0):
        primes = ckks_gen_primes(bits, logN, L + k)
        return cls(logN, primes[:L], primes[L:], dnum, device)

    def close(self):
        if getattr(self, "_h", None):
            lib().ckks_ctx_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def handle(self):
        return self._h

    def beta(self, ell):
        return (ell + self.alpha - 1) // self.alpha

    def ext_primes(self, ell):
        return self.q[:ell] + self.p

    # ------------------------------------------------------------ argument checks
    # The library receives bare device pointers and cannot see how large a
    # buffer is, so every tensor is checked here before its pointer is passed
    # on: it must be on this context's device, of the expected dtype,
    # contiguous, and hold at least the words the call reads or writes.  A
    # failed check raises CkksError (CKKS_EINVAL) and nothing is launched.
    def _arg(self, t, what, words, dtype=torch.uint64):
        if not isinstance(t, torch.Tensor):
            raise CkksError(f"{what}: expected a torch tensor, got {type(t).__name__}", CKKS_EINVAL)
        if t.device != self.device:
            raise CkksError(f"{what}: tensor on {t.device}, the context is on {self.device}", CKKS_EINVAL)
        if t.dtype != dtype:
            raise CkksError(f"{what}: dtype {t.dtype}, expected {dtype}", CKKS_EINVAL)
        if not t.is_contiguous():
            raise CkksError(f"{what}: the tensor is not contiguous", CKKS_EINVAL)
        if t.numel() < words:
            raise CkksError(f"{what}: {t.numel()} elements, the call needs {words}", CKKS_EINVAL)
        return t

    def _poly(self, t, what, nlimbs):
        """A polynomial of at least nlimbs limbs of N words."""
        return self._arg(t, what, max(int(nlimbs), 0) * self.N)

    def _key_words(self, rows):
        return rows * self.dnum * (self.L + self.k) * self.N

    def _key(self, key, what="key"):
        """A key-switching key [dnum][2][L+k][N], or its rows b_j [dnum][L+k][N]
        when it is registered as a compressed key."""
        compressed = isinstance(key, torch.Tensor) and key.data_ptr() in self._compressed
        return self._arg(key, what, self._key_words(1 if compressed else 2))

    def _ws(self, ws, nbytes, what="ws"):
        return self._arg(ws, what, (int(nbytes) + 7) // 8)

    def _ws_op(self, ws, op, level, r=1):
        """The caller's workspace for `op` at `level` (checked), or a new one."""
        if ws is None:
            return self.workspace(op, level, r)
        k = (int(op), int(level), int(r))
        nbytes = self._ws_bytes.get(k)
        if nbytes is None:
            nbytes = self._ws_bytes[k] = self.workspace_bytes(op, level, r)
        return self._ws(ws, nbytes)

    @staticmethod
    def _same_len(n, **lists):
        for name, xs in lists.items():
            if xs is not None and len(xs) != n:
                raise CkksError(f"{name}: {len(xs)} entries, expected {n}", CKKS_EINVAL)

    def table_bytes(self):
        return int(lib().ckks_ctx_table_bytes(self._h))

    # ------------------------------------------------------------ measurement hook
    def profile(self, on=True):
        _check(lib().ckks_profile_enable(self._h, int(bool(on))), self._h)

    def profile_reset(self):
        _check(lib().ckks_profile_reset(self._h), self._h)

    def profile_read(self):
        """{class name: (total_ms, launches, units)} of the launches since the last reset."""
        out = {}
        for i, name in enumerate(K_NAMES):
            ms, n, u = ctypes.c_double(), ctypes.c_longlong(), ctypes.c_double()
            _check(lib().ckks_profile_read(self._h, i, ctypes.byref(ms), ctypes.byref(n), ctypes.byref(u)), self._h)
            out[name] = (ms.value, int(n.value), u.value)
        return out

    def butterfly_peak(self, rounds=20000, stream=None):
        """(butterflies per second, ms, butterflies) of the register-only butterfly
        ceiling (ckks_butterfly_peak); blocks until the measurement is done."""
        nb = ctypes.c_size_t()
        _check(lib().ckks_butterfly_peak_sink_bytes(self._h, ctypes.byref(nb)))
        sink = torch.empty(nb.value // 8, dtype=torch.uint64, device=self.device)
        ms, bf = ctypes.c_float(), ctypes.c_double()
        _check(lib().ckks_butterfly_peak(self._h, int(rounds), _p(sink), _stream(stream), ctypes.byref(ms),
                                         ctypes.byref(bf)), self._h)
        return bf.value / (ms.value * 1e-3), ms.value, bf.value

    def poll_status(self, stream=None):
        """True once the stream's work has finished; raises on an asynchronous CUDA error."""
        done = _i()
        _check(lib().ckks_poll_status(self._h, _stream(stream), ctypes.byref(done)), self._h)
        return bool(done.value)

    def autotune(self, limbs=128, stream=None, cache=None):
        """Time the NTT tile shapes and radix splits and keep the fastest
        (ckks_autotune).  Returns (choice[8], times_ms[24]): the widths of the
        column and block pass per launch size (0 default, 1 half, 2 double),
        then the radix split of the forward and inverse transform per launch
        size (-1, 0, +1).  With cache (a JSON file path), a choice stored for
        this GPU model and parameter shape is applied without timing, and a new
        one is stored."""
        import json

        key = None
        if cache is not None:
            key = f"{torch.cuda.get_device_name(self.device)}|logN={self.logN}|L={self.L}|k={self.k}|dnum={self.dnum}"
            try:
                with open(cache) as f:
                    saved = json.load(f)
            except (OSError, ValueError):
                saved = {}
            if key in saved and len(saved[key].get("choice", [])) == 8:
                self.tune_set(saved[key]["choice"])
                return list(saved[key]["choice"]), list(saved[key]["times_ms"])
        ws = torch.empty((limbs, self.N), dtype=torch.uint64, device=self.device)
        ch = (_i * 8)()
        tm = (ctypes.c_float * 24)()
        _check(lib().ckks_autotune(self._h, _p(ws), limbs * self.N * 8, _stream(stream), ch, tm), self._h)
        choice, times = list(ch), list(tm)
        if cache is not None:
            saved[key] = {"choice": choice, "times_ms": times}
            with open(cache, "w") as f:
                json.dump(saved, f, indent=1)
        return choice, times

    def tune_set(self, choice):
        """Apply a tuner choice (8 ints, the layout autotune returns)."""
        if len(choice) != 8:
            raise CkksError("tune_set: choice must hold 8 ints (4 widths, 4 radix splits)")
        ch = (_i * 8)(*[int(x) for x in choice])
        _check(lib().ckks_tune_set(self._h, ch))

    def selftest_bounded_wait(self, limit_us, stream=None):
        """Launch the bounded-wait self-test (ckks_selftest_bounded_wait): a wait
        on a barrier nothing arrives on, which gives up after limit_us."""
        _check(lib().ckks_selftest_bounded_wait(self._h, int(limit_us), _stream(stream)), self._h)

    def batch_streams(self, n):
        """Streams a batched call is split over (ckks_batch_streams, 1 .. 4)."""
        _check(lib().ckks_batch_streams(self._h, int(n)))

    def concurrency_hint(self, n):
        """Operations the caller runs at once on this context (ckks_concurrency_hint,
        1 .. 64): the basis conversion sizes its grids for a 1/n share of the GPU."""
        _check(lib().ckks_concurrency_hint(self._h, int(n)))

    def fuse_modup(self, on=True):
        """Run single KeySwitches and one-rotation HRotates through the fused
        ModUp tail + KSKInnerProd kernel (ckks_fuse_select); returns whether the
        context supports it."""
        avail = _i()
        _check(lib().ckks_fuse_select(self._h, 1 if on else 0, ctypes.byref(avail)))
        return bool(avail.value)

    def bconv_tensor_cores(self, on=True):
        """Run the basis conversions on the tensor cores (on) or the integer
        units (ckks_bconv_select); returns whether the tensor-core form exists
        for this context."""
        avail = _i()
        _check(lib().ckks_bconv_select(self._h, 1 if on else 0, ctypes.byref(avail)))
        return bool(avail.value)

    # ------------------------------------------------------------ memory
    def empty(self, nlimbs):
        return torch.empty((nlimbs, self.N), dtype=torch.uint64, device=self.device)

    def workspace_bytes(self, op, level, r=1):
        n = ctypes.c_size_t()
        _check(lib().ckks_workspace_bytes(self._h, op, level, r, ctypes.byref(n)))
        return int(n.value)

    def workspace(self, op, level, r=1):
        nbytes = self.workspace_bytes(op, level, r)
        return torch.empty((max(nbytes, 16) + 7) // 8, dtype=torch.uint64, device=self.device)

    # ------------------------------------------------------------ operations
    def ntt(self, x, level, first=0, count=None, stream=None):
        self._arg(x, "x", 0)
        count = (x.shape[0] if x.dim() else 0) - first if count is None else count
        self._poly(x, "x", first + count)
        _check(lib().ckks_ntt(self._h, _p(x), level, first, count, _stream(stream)), self._h)
        return x

    def intt(self, x, level, first=0, count=None, stream=None):
        self._arg(x, "x", 0)
        count = (x.shape[0] if x.dim() else 0) - first if count is None else count
        self._poly(x, "x", first + count)
        _check(lib().ckks_intt(self._h, _p(x), level, first, count, _stream(stream)), self._h)
        return x

    def automorph(self, x, galois, out=None, stream=None):
        self._arg(x, "x", 0)
        nlimbs = x.shape[0] if x.dim() else 0
        self._poly(x, "x", nlimbs)
        out = torch.empty_like(x) if out is None else self._poly(out, "out", nlimbs)
        _check(lib().ckks_automorph(self._h, _p(x), _p(out), nlimbs, galois, _stream(stream)), self._h)
        return out

    def modup(self, a, level, digit, out=None, ws=None, stream=None):
        self._poly(a, "a", level)
        out = self.empty(level + self.k) if out is None else self._poly(out, "out", level + self.k)
        ws = self._ws_op(ws, OP_MODUP, level)
        _check(lib().ckks_modup(self._h, _p(a), level, digit, _p(out), _p(ws), _stream(stream)), self._h)
        return out

    def ksk_inner_prod(self, digits, level, key, u=None, v=None, stream=None):
        self._poly(digits, "digits", self.beta(level) * (level + self.k))
        self._key(key)
        u = self.empty(level + self.k) if u is None else self._poly(u, "u", level + self.k)
        v = self.empty(level + self.k) if v is None else self._poly(v, "v", level + self.k)
        _check(lib().ckks_ksk_inner_prod(self._h, _p(digits), level, _p(key), _p(u), _p(v), _stream(stream)),
               self._h)
        return u, v

    def moddown(self, x, level, out=None, ws=None, stream=None):
        self._poly(x, "x", level + self.k)
        out = self.empty(level) if out is None else self._poly(out, "out", level)
        ws = self._ws_op(ws, OP_MODDOWN, level)
        _check(lib().ckks_moddown(self._h, _p(x), level, _p(out), _p(ws), _stream(stream)), self._h)
        return out

    def moddown_noalloc(self, x, level, out=None, stream=None):
        """ModDown with its scratch in the library's fixed 16 MiB device array
        (no workspace; (k + level) * N must not exceed 2^21 words)."""
        self._poly(x, "x", level + self.k)
        out = self.empty(level) if out is None else self._poly(out, "out", level)
        rc = lib().ckks_moddown_noalloc(self._h, _p(x), level, _p(out), _stream(stream))
        if rc == CKKS_EUNSUPPORTED:
            raise CkksError(f"ckks_moddown_noalloc: (k + level) * N = {(self.k + level) * self.N} words exceeds "
                            f"the fixed scratch of 2^21 words")
        _check(rc, self._h)
        return out

    def pmodup(self, x, level, out=None, stream=None):
        self._poly(x, "x", level)
        out = self.empty(level + self.k) if out is None else self._poly(out, "out", level + self.k)
        _check(lib().ckks_pmodup(self._h, _p(x), level, _p(out), _stream(stream)), self._h)
        return out

    def rescale(self, x, level, out=None, ws=None, stream=None):
        self._poly(x, "x", level)
        out = self.empty(level - 1) if out is None else self._poly(out, "out", level - 1)
        ws = self._ws_op(ws, OP_RESCALE, level)
        _check(lib().ckks_rescale(self._h, _p(x), level, _p(out), _p(ws), _stream(stream)), self._h)
        return out

    def keyswitch(self, a, level, key, u=None, v=None, ws=None, stream=None):
        self._poly(a, "a", level)
        self._key(key)
        u = self.empty(level) if u is None else self._poly(u, "u", level)
        v = self.empty(level) if v is None else self._poly(v, "v", level)
        ws = self._ws_op(ws, OP_KEYSWITCH, level)
        _check(lib().ckks_keyswitch(self._h, _p(a), level, _p(key), _p(u), _p(v), _p(ws), _stream(stream)), self._h)
        return u, v

    def rotate(self, a, b, level, galois, key, oa=None, ob=None, ws=None, stream=None):
        self._poly(a, "a", level)
        self._poly(b, "b", level)
        self._key(key)
        oa = self.empty(level) if oa is None else self._poly(oa, "oa", level)
        ob = self.empty(level) if ob is None else self._poly(ob, "ob", level)
        ws = self._ws_op(ws, OP_ROTATE, level)
        _check(lib().ckks_rotate(self._h, _p(a), _p(b), level, galois, _p(key), _p(oa), _p(ob), _p(ws),
                                 _stream(stream)), self._h)
        return oa, ob

    def hrotate(self, a, b, level, galois, keys, outs=None, ws=None, stream=None):
        r = len(galois)
        self._same_len(r, keys=keys, outs=outs)
        self._poly(a, "a", level)
        self._poly(b, "b", level)
        for i, k in enumerate(keys):
            self._key(k, f"keys[{i}]")
        if outs is None:
            outs = [(self.empty(level), self.empty(level)) for _ in range(r)]
        else:
            for i, (oa, ob) in enumerate(outs):
                self._poly(oa, f"outs[{i}][0]", level)
                self._poly(ob, f"outs[{i}][1]", level)
        ws = self._ws_op(ws, OP_HROTATE, level, r)
        g = (ctypes.c_uint32 * r)(*galois)
        kp = (_vp * r)(*[k.data_ptr() for k in keys])
        oa = (_vp * r)(*[o[0].data_ptr() for o in outs])
        ob = (_vp * r)(*[o[1].data_ptr() for o in outs])
        _check(lib().ckks_hrotate(self._h, _p(a), _p(b), level, r, g, kp, oa, ob, _p(ws), _stream(stream)), self._h)
        return outs

    def batch_workspace_bytes(self, levels):
        n = len(levels)
        lv = (_i * max(n, 1))(*[int(x) for x in levels])
        nbytes = ctypes.c_size_t()
        _check(lib().ckks_batch_workspace_bytes(self._h, n, lv, ctypes.byref(nbytes)))
        return int(nbytes.value)

    def batch_workspace(self, levels):
        nbytes = self.batch_workspace_bytes(levels)
        return torch.empty(max(nbytes // 8, 2), dtype=torch.uint64, device=self.device)

    def keyswitch_batch(self, a, b, levels, galois, keys, outs=None, ws=None, stream=None, seeds=None):
        """Batched key switching.  a, keys: lists of tensors; b: None or a list
        whose None entries make KeySwitch entries (others are one-rotation
        HRotates by galois[i]); levels: list of ints; seeds: None (full keys)
        or one seed per entry (keys are then compressed, b rows only).
        Returns [(oa, ob)]."""
        n = len(a)
        self._same_len(n, levels=levels, keys=keys, b=b, galois=galois, outs=outs, seeds=seeds)
        for i in range(n):
            self._poly(a[i], f"a[{i}]", levels[i])
            if b is not None and b[i] is not None:
                self._poly(b[i], f"b[{i}]", levels[i])
            if seeds is None:
                self._key(keys[i], f"keys[{i}]")
            else:
                self._arg(keys[i], f"keys[{i}]", self._key_words(1))
        if outs is None:
            outs = [(self.empty(levels[i]), self.empty(levels[i])) for i in range(n)]
        else:
            for i, (oa, ob) in enumerate(outs):
                self._poly(oa, f"outs[{i}][0]", levels[i])
                self._poly(ob, f"outs[{i}][1]", levels[i])
        ws = self.batch_workspace(levels) if ws is None else self._ws(ws, self.batch_workspace_bytes(levels))
        m = max(n, 1)
        ap = (_vp * m)(*[x.data_ptr() for x in a])
        bp = None if b is None else (_vp * m)(*[None if x is None else x.data_ptr() for x in b])
        lv = (_i * m)(*[int(x) for x in levels])
        gp = None if galois is None else (ctypes.c_uint32 * m)(*[int(x) for x in galois])
        kp = (_vp * m)(*[x.data_ptr() for x in keys])
        oa = (_vp * m)(*[o[0].data_ptr() for o in outs])
        ob = (_vp * m)(*[o[1].data_ptr() for o in outs])
        if seeds is None:
            _check(lib().ckks_keyswitch_batch(self._h, n, ap, bp, lv, gp, kp, oa, ob, _p(ws), _stream(stream)),
                   self._h)
        else:
            sd = (ctypes.c_uint64 * m)(*[int(x) & 0xFFFFFFFFFFFFFFFF for x in seeds])
            _check(lib().ckks_keyswitch_batch_seeded(self._h, n, ap, bp, lv, gp, kp, sd, oa, ob, _p(ws),
                                                     _stream(stream)), self._h)
        return outs

    def hrotate_batch(self, cts, levels, rotations, outs=None, ws=None, stream=None):
        """cts: list of (a, b); rotations: per ciphertext a list of (galois, key).
        Returns per ciphertext a list of (oa, ob), one per rotation."""
        n = len(cts)
        self._same_len(n, levels=levels, rotations=rotations, outs=outs)
        nrot = [len(r) for r in rotations]
        flat = [gk for r in rotations for gk in r]
        for c in range(n):
            self._poly(cts[c][0], f"cts[{c}][0]", levels[c])
            self._poly(cts[c][1], f"cts[{c}][1]", levels[c])
            for i, (_, k) in enumerate(rotations[c]):
                self._key(k, f"rotations[{c}][{i}] key")
        if outs is None:
            outs = [[(self.empty(levels[c]), self.empty(levels[c])) for _ in rotations[c]] for c in range(n)]
        else:
            for c in range(n):
                self._same_len(nrot[c], **{f"outs[{c}]": outs[c]})
                for i, (oa, ob) in enumerate(outs[c]):
                    self._poly(oa, f"outs[{c}][{i}][0]", levels[c])
                    self._poly(ob, f"outs[{c}][{i}][1]", levels[c])
        flat_out = [o for oc in outs for o in oc]
        m = max(len(flat), 1)
        lv = (_i * max(n, 1))(*[int(x) for x in levels])
        nr = (_i * max(n, 1))(*nrot)
        nbytes = ctypes.c_size_t()
        _check(lib().ckks_hrotate_batch_workspace_bytes(self._h, n, lv, nr, ctypes.byref(nbytes)))
        if ws is None:
            ws = torch.empty(max(nbytes.value // 8, 2), dtype=torch.uint64, device=self.device)
        else:
            self._ws(ws, nbytes.value)
        arr = lambda xs, k: (_vp * k)(*[x.data_ptr() for x in xs])
        _check(lib().ckks_hrotate_batch(self._h, n, arr([c[0] for c in cts], max(n, 1)),
                                        arr([c[1] for c in cts], max(n, 1)), lv, nr,
                                        (ctypes.c_uint32 * m)(*[int(g) for g, _ in flat]),
                                        arr([k for _, k in flat], m), arr([o[0] for o in flat_out], m),
                                        arr([o[1] for o in flat_out], m), _p(ws), _stream(stream)), self._h)
        return outs

    def keygen_ksk_seeded(self, s, e, seed, galois, key_b=None, ws=None, stream=None):
        """Compressed key (rows b_j only, [dnum][L+k][N]); a_j comes from seed."""
        self._arg(s, "s", self.N, torch.int64)
        self._arg(e, "e", self.dnum * self.N, torch.int64)
        key_b = torch.empty((self.dnum, self.L + self.k, self.N), dtype=torch.uint64,
                            device=self.device) if key_b is None else self._arg(key_b, "key_b", self._key_words(1))
        ws = self._ws_op(ws, OP_KEYGEN_SEEDED, 1)
        _check(lib().ckks_keygen_ksk_seeded(self._h, _p(s), _p(e), int(seed) & 0xFFFFFFFFFFFFFFFF, int(galois),
                                            _p(key_b), _p(ws), _stream(stream)), self._h)
        return key_b

    def register_compressed_key(self, key_b, seed):
        """Every call of this context that receives key_b treats it as a compressed key.
        The context keeps key_b referenced until unregister_compressed_key."""
        self._arg(key_b, "key_b", self._key_words(1))
        _check(lib().ckks_key_register_seed(self._h, _p(key_b), int(seed) & 0xFFFFFFFFFFFFFFFF))
        self._compressed[key_b.data_ptr()] = key_b

    def unregister_compressed_key(self, key_b):
        self._arg(key_b, "key_b", 0)
        _check(lib().ckks_key_unregister(self._h, _p(key_b)))
        self._compressed.pop(key_b.data_ptr(), None)

    def ksk_expand(self, key_b, seed, key=None, stream=None):
        self._arg(key_b, "key_b", self._key_words(1))
        key = torch.empty((self.dnum, 2, self.L + self.k, self.N), dtype=torch.uint64,
                          device=self.device) if key is None else self._arg(key, "key", self._key_words(2))
        _check(lib().ckks_ksk_expand(self._h, _p(key_b), int(seed) & 0xFFFFFFFFFFFFFFFF, _p(key), _stream(stream)),
               self._h)
        return key

    def mult(self, a1, b1, a2, b2, level, key, oa=None, ob=None, ws=None, stream=None, new=False):
        """Algorithm 2 (Mult + relinearisation + Rescale), or Algorithm 7 (NewMult)
        with new=True; outputs at level-1."""
        for name, t in (("a1", a1), ("b1", b1), ("a2", a2), ("b2", b2)):
            self._poly(t, name, level)
        self._key(key)
        oa = self.empty(level - 1) if oa is None else self._poly(oa, "oa", level - 1)
        ob = self.empty(level - 1) if ob is None else self._poly(ob, "ob", level - 1)
        ws = self._ws_op(ws, OP_NEWMULT if new else OP_MULT, level)
        fn = lib().ckks_newmult if new else lib().ckks_mult
        _check(fn(self._h, _p(a1), _p(b1), _p(a2), _p(b2), level, _p(key), _p(oa), _p(ob), _p(ws), _stream(stream)),
               self._h)
        return oa, ob

    def newmult(self, a1, b1, a2, b2, level, key, oa=None, ob=None, ws=None, stream=None):
        return self.mult(a1, b1, a2, b2, level, key, oa, ob, ws, stream, new=True)

    def mult_batch_workspace_bytes(self, levels, new=False):
        n = len(levels)
        lv = (_i * max(n, 1))(*[int(x) for x in levels])
        nbytes = ctypes.c_size_t()
        fn = lib().ckks_newmult_batch_workspace_bytes if new else lib().ckks_mult_batch_workspace_bytes
        _check(fn(self._h, n, lv, ctypes.byref(nbytes)))
        return int(nbytes.value)

    def mult_batch_workspace(self, levels, new=False):
        nbytes = self.mult_batch_workspace_bytes(levels, new)
        return torch.empty(max(nbytes // 8, 2), dtype=torch.uint64, device=self.device)

    def mult_batch(self, cts1, cts2, levels, keys, outs=None, ws=None, stream=None, new=False):
        """cts1, cts2: lists of (a, b); returns [(oa, ob)] at level-1 each."""
        n = len(cts1)
        self._same_len(n, cts2=cts2, levels=levels, keys=keys, outs=outs)
        for i in range(n):
            for name, t in ((f"cts1[{i}][0]", cts1[i][0]), (f"cts1[{i}][1]", cts1[i][1]),
                            (f"cts2[{i}][0]", cts2[i][0]), (f"cts2[{i}][1]", cts2[i][1])):
                self._poly(t, name, levels[i])
            self._key(keys[i], f"keys[{i}]")
        if outs is None:
            outs = [(self.empty(levels[i] - 1), self.empty(levels[i] - 1)) for i in range(n)]
        else:
            for i, (oa, ob) in enumerate(outs):
                self._poly(oa, f"outs[{i}][0]", levels[i] - 1)
                self._poly(ob, f"outs[{i}][1]", levels[i] - 1)
        ws = (self.mult_batch_workspace(levels, new) if ws is None
              else self._ws(ws, self.mult_batch_workspace_bytes(levels, new)))
        m = max(n, 1)
        arr = lambda xs: (_vp * m)(*[x.data_ptr() for x in xs])
        lv = (_i * m)(*[int(x) for x in levels])
        fn = lib().ckks_newmult_batch if new else lib().ckks_mult_batch
        _check(fn(self._h, n, arr([c[0] for c in cts1]), arr([c[1] for c in cts1]), arr([c[0] for c in cts2]),
                  arr([c[1] for c in cts2]), lv, arr(keys), arr([o[0] for o in outs]), arr([o[1] for o in outs]),
                  _p(ws), _stream(stream)), self._h)
        return outs

    def newmult_sum(self, cts1, cts2, level, key, oa=None, ob=None, ws=None, stream=None):
        """Sum of NewMult products with one merged ModDown; cts: lists of (a, b) at one level."""
        n = len(cts1)
        self._same_len(n, cts2=cts2)
        for i in range(n):
            for name, t in ((f"cts1[{i}][0]", cts1[i][0]), (f"cts1[{i}][1]", cts1[i][1]),
                            (f"cts2[{i}][0]", cts2[i][0]), (f"cts2[{i}][1]", cts2[i][1])):
                self._poly(t, name, level)
        self._key(key)
        oa = self.empty(level - 1) if oa is None else self._poly(oa, "oa", level - 1)
        ob = self.empty(level - 1) if ob is None else self._poly(ob, "ob", level - 1)
        ws = (self.mult_batch_workspace([level] * n, new=True) if ws is None
              else self._ws(ws, self.mult_batch_workspace_bytes([level] * n, new=True)))
        arr = lambda xs: (_vp * n)(*[x.data_ptr() for x in xs])
        _check(lib().ckks_newmult_sum(self._h, n, arr([c[0] for c in cts1]), arr([c[1] for c in cts1]),
                                      arr([c[0] for c in cts2]), arr([c[1] for c in cts2]), level, _p(key), _p(oa),
                                      _p(ob), _p(ws), _stream(stream)), self._h)
        return oa, ob

    def ptmatvecmult(self, a, b, level, nb, ng, g_baby, g_giant, key_baby, key_giant, diags, rescale=True,
                     oa=None, ob=None, ws=None, stream=None):
        out_l = level - 1 if rescale else level
        self._same_len(nb, g_baby=g_baby, key_baby=key_baby)
        self._same_len(ng, g_giant=g_giant, key_giant=key_giant)
        self._same_len(nb * ng, diags=diags)
        self._poly(a, "a", level)
        self._poly(b, "b", level)
        # baby step 0 and giant step 0 are the identity: their keys are not read
        for i in range(1, nb):
            self._key(key_baby[i], f"key_baby[{i}]")
        for t in range(1, ng):
            self._key(key_giant[t], f"key_giant[{t}]")
        for d, x in enumerate(diags):
            self._poly(x, f"diags[{d}]", level + self.k)
        oa = self.empty(out_l) if oa is None else self._poly(oa, "oa", out_l)
        ob = self.empty(out_l) if ob is None else self._poly(ob, "ob", out_l)
        ws = self._ws_op(ws, OP_PTMATVEC, level, ng)
        gb = (ctypes.c_uint32 * nb)(*[int(x) for x in g_baby])
        gg = (ctypes.c_uint32 * ng)(*[int(x) for x in g_giant])
        kb = (_vp * nb)(*[None if k is None else k.data_ptr() for k in key_baby])
        kg = (_vp * ng)(*[None if k is None else k.data_ptr() for k in key_giant])
        dp = (_vp * (nb * ng))(*[d.data_ptr() for d in diags])
        _check(lib().ckks_ptmatvecmult(self._h, _p(a), _p(b), level, nb, ng, gb, gg, kb, kg, dp, int(bool(rescale)),
                                       _p(oa), _p(ob), _p(ws), _stream(stream)), self._h)
        return oa, ob

    def keygen_ksk(self, s, e, a, galois, key=None, ws=None, stream=None):
        """s: int64 [N]; e: int64 [dnum][N]; a: uint64 [dnum][L+k][N]; galois 0 = relinearisation."""
        self._arg(s, "s", self.N, torch.int64)
        self._arg(e, "e", self.dnum * self.N, torch.int64)
        self._arg(a, "a", self._key_words(1))
        key = torch.empty((self.dnum, 2, self.L + self.k, self.N), dtype=torch.uint64,
                          device=self.device) if key is None else self._arg(key, "key", self._key_words(2))
        ws = self._ws_op(ws, OP_KEYGEN, 1)
        _check(lib().ckks_keygen_ksk(self._h, _p(s), _p(e), _p(a), galois, _p(key), _p(ws), _stream(stream)),
               self._h)
        return key


class Server:
    """Serving loop of the C ABI (ckks_server_*): continuous batching of
    HRotate / KeySwitch / Mult requests over several contexts, admitted by
    device memory.  The tensors of a request are kept referenced here until
    the request is polled as finished."""

    def __init__(self, contexts, mem_budget, max_batch=64, streams=4):
        self.contexts = list(contexts)
        arr = (_vp * len(self.contexts))(*[c._h for c in self.contexts])
        h = ctypes.c_void_p()
        _check(lib().ckks_server_create(arr, len(self.contexts), int(mem_budget), int(max_batch), int(streams),
                                        ctypes.byref(h)))
        self._h = h
        self._keys = []
        self._live = {}

    def close(self):
        if getattr(self, "_h", None):
            _check(lib().ckks_server_destroy(self._h))
            self._h = None
            self._live.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def add_key(self, ctx, key, seed=None):
        """Register a resident key; with seed, key is a compressed key (rows b_j only)."""
        c = self._ctx(ctx)
        if c is not None:
            if seed is None:
                c._key(key)
            else:
                c._arg(key, "key", c._key_words(1))
        hd = _i()
        if seed is None:
            _check(lib().ckks_server_add_key(self._h, int(ctx), _p(key), ctypes.byref(hd)))
        else:
            _check(lib().ckks_server_add_key_seeded(self._h, int(ctx), _p(key), int(seed) & 0xFFFFFFFFFFFFFFFF,
                                                    ctypes.byref(hd)))
        self._keys.append(key)
        return hd.value

    def now_ms(self):
        return float(lib().ckks_server_now_ms(self._h))

    def _ctx(self, ctx):
        """The context of index ctx (None when out of range: the library rejects it)."""
        try:
            i = int(ctx)
        except (TypeError, ValueError):
            return None
        return self.contexts[i] if 0 <= i < len(self.contexts) else None

    def _submit(self, op, ctx, level, a, b, a2, b2, galois, key, oa, ob, arrival_ms):
        c = self._ctx(ctx)
        if c is not None:
            for name, t in (("a", a), ("b", b), ("a2", a2), ("b2", b2)):
                if t is not None:
                    c._poly(t, name, level)
            out_l = level - 1 if op in (REQ_MULT, REQ_NEWMULT) else level
            c._poly(oa, "oa", out_l)
            c._poly(ob, "ob", out_l)
        r = _Request(op, int(ctx), int(level), _p(a), _p(b), _p(a2), _p(b2), int(galois), int(key), _p(oa), _p(ob),
                     float(arrival_ms))
        rid = ctypes.c_uint64()
        _check(lib().ckks_server_submit(self._h, ctypes.byref(r), ctypes.byref(rid)))
        self._live[rid.value] = (a, b, a2, b2, oa, ob)
        return rid.value

    def submit_hrotate(self, ctx, a, b, level, galois, key, oa, ob, arrival_ms=-1.0):
        return self._submit(REQ_HROTATE, ctx, level, a, b, None, None, galois, key, oa, ob, arrival_ms)

    def submit_keyswitch(self, ctx, a, level, key, oa, ob, arrival_ms=-1.0):
        return self._submit(REQ_KEYSWITCH, ctx, level, a, None, None, None, 1, key, oa, ob, arrival_ms)

    def submit_mult(self, ctx, ct1, ct2, level, key, oa, ob, arrival_ms=-1.0, new=False):
        return self._submit(REQ_NEWMULT if new else REQ_MULT, ctx, level, ct1[0], ct1[1], ct2[0], ct2[1], 1, key, oa,
                            ob, arrival_ms)

    def step(self):
        n = _i()
        _check(lib().ckks_server_step(self._h, ctypes.byref(n)))
        return n.value

    def poll(self, max_n=4096, with_status=False):
        """Finished requests as (id, latency_ms, done_ms), or (id, latency_ms,
        done_ms, status) with with_status; status is CKKS_OK, or CKKS_ETIMEOUT
        when the request's outputs are not valid.  Without with_status a failed
        request raises CkksError."""
        ids = (ctypes.c_uint64 * max_n)()
        lat = (ctypes.c_double * max_n)()
        done = (ctypes.c_double * max_n)()
        sts = (ctypes.c_int * max_n)()
        n = _i()
        _check(lib().ckks_server_poll(self._h, max_n, ids, lat, done, sts, ctypes.byref(n)))
        out = []
        failed = []
        for i in range(n.value):
            self._live.pop(ids[i], None)
            if with_status:
                out.append((int(ids[i]), float(lat[i]), float(done[i]), int(sts[i])))
            else:
                out.append((int(ids[i]), float(lat[i]), float(done[i])))
                if sts[i] != CKKS_OK:
                    failed.append(int(ids[i]))
        if failed:
            raise CkksError(f"served requests {failed} failed: a bounded device wait ran out", CKKS_ETIMEOUT)
        return out

    def selftest_timeout(self, limit_us=20000):
        """Arm the test hook: the next batch runs the bounded-wait self-test first,
        so its requests come back with CKKS_ETIMEOUT."""
        _check(lib().ckks_server_selftest_timeout(self._h, int(limit_us)))

    def stats(self):
        st = _Stats()
        _check(lib().ckks_server_stats(self._h, ctypes.byref(st)))
        return {f: getattr(st, f) for f, _ in _Stats._fields_}

    def drain(self, sleep_s=0.0):
        """Step until nothing is pending or in flight; returns the finished requests."""
        import time

        out = []
        while True:
            self.step()
            out += self.poll()
            st = self.stats()
            if st["pending"] == 0 and st["in_flight"] == 0:
                return out + self.poll()
            if sleep_s:
                time.sleep(sleep_s)
