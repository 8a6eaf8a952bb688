"""CPU oracle for the CKKS key-switching path (arXiv 2112.06396).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the
benchmark's CPU-baseline / reference leg may import this package; the product
package never does.  The arithmetic lives in ``ckks_oracle.c`` (plain C,
``unsigned __int128`` and ``%``); this module compiles it with gcc and wraps
it with ctypes over numpy arrays.  It shares no code with the CUDA library.

Every function follows one passage of the paper:

* ``ntt`` / ``intt`` / ``ntt_naive`` -- Sec. 2.3, "Polynomial Representation".
* ``automorph_eval`` / ``automorph_coeff`` -- the Automorph subroutine of the
  table "CKKS Subroutines".
* ``modup`` -- Algorithm 6 (ModUp, NewLimb basis conversion).
* ``ksk_inner_prod`` -- KSKInnerProd, table "CKKS Subroutines".
* ``moddown`` -- ModDown_{B,d}, table "CKKS Subroutines"; rounding per Sec. 2.4.
* ``rescale`` -- Algorithm 1's ModDown_{B,1}.
* ``pmodup`` -- PModUp, Sec. 5.1.
* ``keyswitch`` / ``rotate`` / ``hrotate`` -- Algorithms 3 and 4.
* ``ptmatvec`` -- Algorithm 8 with baby-step/giant-step (Sec. 5.2).
* ``keygen`` / ``encrypt`` / ``decrypt`` -- the key shape of Eq. (kskShape).

Parity status: every function is pinned by a test in ``tests/test_oracle_*.py``
against brute force, big-integer CRT, closed forms or decryption bounds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ckks_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "libckks_oracle.so")
_lock = threading.Lock()
_lib = None

u64p = ctypes.POINTER(ctypes.c_uint64)
i64p = ctypes.POINTER(ctypes.c_int64)


class _Params(ctypes.Structure):
    _fields_ = [("logN", ctypes.c_int), ("L", ctypes.c_int), ("k", ctypes.c_int),
                ("dnum", ctypes.c_int), ("primes", u64p)]


def build(force: bool = False) -> str:
    """Compile the oracle shared library with gcc (plain -O2, no OpenMP)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".{os.getpid()}.tmp"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER(_Params)
            sig = {
                "or_is_prime": (ctypes.c_int, [ctypes.c_uint64]),
                "or_gen_primes": (ctypes.c_int, [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p]),
                "or_min_psi": (ctypes.c_uint64, [ctypes.c_uint64, ctypes.c_int]),
                "or_ntt_naive": (None, [u64p, u64p, ctypes.c_int, ctypes.c_uint64]),
                "or_ntt": (None, [u64p, ctypes.c_int, ctypes.c_uint64]),
                "or_intt": (None, [u64p, ctypes.c_int, ctypes.c_uint64]),
                "or_automorph_coeff": (None, [u64p, u64p, ctypes.c_int, ctypes.c_uint64, ctypes.c_uint64]),
                "or_automorph_eval": (None, [u64p, u64p, ctypes.c_int, ctypes.c_uint64]),
                "or_alpha": (ctypes.c_int, [P]),
                "or_beta": (ctypes.c_int, [P, ctypes.c_int]),
                "or_modup": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, u64p, u64p]),
                "or_ksk_inner_prod": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, u64p, u64p]),
                "or_moddown": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p]),
                "or_rescale": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p]),
                "or_pmodup": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p]),
                "or_keyswitch": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, u64p, u64p]),
                "or_rotate": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, ctypes.c_uint64, u64p, u64p, u64p]),
                "or_mult": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, u64p, u64p, u64p, u64p, u64p]),
                "or_newmult": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, u64p, u64p, u64p, u64p, u64p]),
                "or_moddown_merged": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p]),
                "or_newmult_sum": (ctypes.c_int, [P, ctypes.c_int, ctypes.c_int, ctypes.POINTER(u64p),
                                                  ctypes.POINTER(u64p), ctypes.POINTER(u64p), ctypes.POINTER(u64p),
                                                  u64p, u64p, u64p]),
                "or_prng_key_a": (ctypes.c_uint64, [P, ctypes.c_uint64, ctypes.c_int, ctypes.c_int, ctypes.c_uint64]),
                "or_prng_key_a_fill": (ctypes.c_int, [P, ctypes.c_uint64, u64p]),
                "or_hrotate": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, ctypes.c_int, u64p,
                                              ctypes.POINTER(u64p), ctypes.POINTER(u64p), ctypes.POINTER(u64p)]),
                "or_ptmatvec": (ctypes.c_int, [P, ctypes.c_int, u64p, u64p, ctypes.c_int, ctypes.c_int,
                                               u64p, u64p, ctypes.POINTER(u64p), ctypes.POINTER(u64p),
                                               ctypes.POINTER(u64p), ctypes.c_int, u64p, u64p]),
                "or_signed_to_eval": (ctypes.c_int, [P, i64p, u64p]),
                "or_keygen": (ctypes.c_int, [P, u64p, i64p, u64p, i64p, u64p]),
                "or_rot_secret": (ctypes.c_int, [P, i64p, ctypes.c_uint64, u64p]),
                "or_sq_secret": (ctypes.c_int, [P, i64p, u64p]),
                "or_encrypt": (ctypes.c_int, [P, ctypes.c_int, i64p, i64p, u64p, u64p]),
                "or_decrypt": (ctypes.c_int, [P, ctypes.c_int, i64p, u64p, u64p, u64p]),
                "or_ntt_limbs": (ctypes.c_int, [P, ctypes.c_int, u64p, ctypes.c_int, ctypes.c_int, ctypes.c_int]),
            }
            for name, (res, args) in sig.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
    return _lib


def _u(a: np.ndarray):
    assert a.dtype == np.uint64 and a.flags["C_CONTIGUOUS"], (a.dtype, a.flags)
    return a.ctypes.data_as(u64p)


def _i(a: np.ndarray):
    assert a.dtype == np.int64 and a.flags["C_CONTIGUOUS"]
    return a.ctypes.data_as(i64p)


def _ptr_array(arrs):
    return (u64p * len(arrs))(*[(_u(a) if a is not None else u64p()) for a in arrs])


class Params:
    """Parameter set (N = 2^logN, L chain limbs, k special primes, dnum digits).

    ``primes`` lists the chain q_0..q_{L-1} followed by p_0..p_{k-1}; when not
    given it is generated by :func:`gen_primes` (largest NTT-friendly primes
    below 2^bits, chain first).
    """

    def __init__(self, logN, L, k, dnum, bits=None, primes=None):
        self.logN, self.L, self.k, self.dnum = int(logN), int(L), int(k), int(dnum)
        self.N = 1 << self.logN
        if primes is None:
            primes = gen_primes(bits, logN, L + k)
        self.primes = np.ascontiguousarray(np.asarray(primes, dtype=np.uint64))
        assert self.primes.size == L + k
        self._c = _Params(self.logN, self.L, self.k, self.dnum, _u(self.primes))

    @property
    def alpha(self):
        return (self.L + self.dnum - 1) // self.dnum

    def beta(self, ell):
        return (ell + self.alpha - 1) // self.alpha

    def ext_primes(self, ell):
        """Moduli of the level-ell extended basis q_0..q_{ell-1}, p_0..p_{k-1}."""
        return [int(x) for x in self.primes[:ell]] + [int(x) for x in self.primes[self.L:]]

    @property
    def c(self):
        return ctypes.byref(self._c)


# ---------------------------------------------------------------- scalars
def is_prime(n: int) -> bool:
    return bool(_load().or_is_prime(n))


def gen_primes(bits, logN, count):
    out = np.zeros(count, dtype=np.uint64)
    rc = _load().or_gen_primes(bits, logN, count, _u(out))
    if rc != 0:
        raise ValueError(f"not enough NTT-friendly primes below 2^{bits} for 2N=2^{logN + 1}")
    return [int(x) for x in out]


def min_psi(q, logN):
    return int(_load().or_min_psi(q, logN))


# ---------------------------------------------------------------- transforms
def ntt_naive(a, logN, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    _load().or_ntt_naive(_u(a), _u(out), logN, q)
    return out


def ntt(a, logN, q):
    a = np.array(a, dtype=np.uint64, copy=True, order="C")
    _load().or_ntt(_u(a), logN, q)
    return a


def intt(a, logN, q):
    a = np.array(a, dtype=np.uint64, copy=True, order="C")
    _load().or_intt(_u(a), logN, q)
    return a


def ntt_limbs(P: Params, ell, x, first=0, count=None, inverse=False):
    """Per-limb (i)NTT of an [ell+k][N] array over the level-ell extended basis."""
    x = np.array(x, dtype=np.uint64, copy=True, order="C")
    if count is None:
        count = x.shape[0] - first
    _load().or_ntt_limbs(P.c, ell, _u(x), first, count, int(bool(inverse)))
    return x


def automorph_coeff(a, logN, g, q):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    _load().or_automorph_coeff(_u(a), _u(out), logN, g, q)
    return out


def automorph_eval(a, logN, g):
    """Evaluation-form automorphism; accepts [N] or [nl][N]."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros_like(a)
    N = 1 << logN
    flat_in, flat_out = a.reshape(-1, N), out.reshape(-1, N)
    for r in range(flat_in.shape[0]):
        _load().or_automorph_eval(_u(flat_in[r]), _u(flat_out[r]), logN, g)
    return out


# ---------------------------------------------------------------- key switching
def modup(P: Params, ell, j, a):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    out = np.zeros((ell + P.k, P.N), dtype=np.uint64)
    if _load().or_modup(P.c, ell, j, _u(a), _u(out)) != 0:
        raise ValueError("bad digit")
    return out


def ksk_inner_prod(P: Params, ell, digits, key):
    digits = np.ascontiguousarray(digits, dtype=np.uint64)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    u = np.zeros((ell + P.k, P.N), dtype=np.uint64)
    v = np.zeros_like(u)
    _load().or_ksk_inner_prod(P.c, ell, _u(digits), _u(key), _u(u), _u(v))
    return u, v


def moddown(P: Params, ell, x):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros((ell, P.N), dtype=np.uint64)
    _load().or_moddown(P.c, ell, _u(x), _u(out))
    return out


def rescale(P: Params, ell, x):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros((ell - 1, P.N), dtype=np.uint64)
    if _load().or_rescale(P.c, ell, _u(x), _u(out)) != 0:
        raise ValueError("rescale needs ell >= 2")
    return out


def pmodup(P: Params, ell, x):
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros((ell + P.k, P.N), dtype=np.uint64)
    _load().or_pmodup(P.c, ell, _u(x), _u(out))
    return out


def keyswitch(P: Params, ell, a, key):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    u = np.zeros((ell, P.N), dtype=np.uint64)
    v = np.zeros_like(u)
    _load().or_keyswitch(P.c, ell, _u(a), _u(key), _u(u), _u(v))
    return u, v


def mult(P: Params, ell, a1, b1, a2, b2, key):
    """Algorithm 2 (Mult + relinearisation + Rescale): outputs at level ell-1."""
    c = [np.ascontiguousarray(x, dtype=np.uint64) for x in (a1, b1, a2, b2, key)]
    oa = np.zeros((ell - 1, P.N), dtype=np.uint64)
    ob = np.zeros_like(oa)
    if _load().or_mult(P.c, ell, *[_u(x) for x in c], _u(oa), _u(ob)) != 0:
        raise ValueError("mult needs ell >= 2")
    return oa, ob


def newmult(P: Params, ell, a1, b1, a2, b2, key):
    """Algorithm 7 (NewMult): merged ModDown by P*q_{ell-1}; outputs at level ell-1."""
    c = [np.ascontiguousarray(x, dtype=np.uint64) for x in (a1, b1, a2, b2, key)]
    oa = np.zeros((ell - 1, P.N), dtype=np.uint64)
    ob = np.zeros_like(oa)
    if _load().or_newmult(P.c, ell, *[_u(x) for x in c], _u(oa), _u(ob)) != 0:
        raise ValueError("newmult needs ell >= 2")
    return oa, ob


def newmult_sum(P: Params, ell, cts1, cts2, key):
    """Sum of NewMult over pairs with one merged ModDown (Sec. 5.1); cts: lists of (a, b)."""
    keep = []

    def arr(xs):
        xs = [np.ascontiguousarray(x, dtype=np.uint64) for x in xs]
        keep.extend(xs)
        return _ptr_array(xs)

    key = np.ascontiguousarray(key, dtype=np.uint64)
    oa = np.zeros((ell - 1, P.N), dtype=np.uint64)
    ob = np.zeros_like(oa)
    rc = _load().or_newmult_sum(P.c, ell, len(cts1), arr([c[0] for c in cts1]), arr([c[1] for c in cts1]),
                                arr([c[0] for c in cts2]), arr([c[1] for c in cts2]), _u(key), _u(oa), _u(ob))
    if rc != 0:
        raise ValueError("newmult_sum needs ell >= 2 and at least one pair")
    return oa, ob


def moddown_merged(P: Params, ell, x):
    """ModDown by P*q_{ell-1} of an [ell+k][N] polynomial: [ell-1][N]."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    out = np.zeros((ell - 1, P.N), dtype=np.uint64)
    if _load().or_moddown_merged(P.c, ell, _u(x), _u(out)) != 0:
        raise ValueError("moddown_merged needs ell >= 2")
    return out


def rotate(P: Params, ell, a, b, g, key):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    key = np.ascontiguousarray(key, dtype=np.uint64)
    oa = np.zeros((ell, P.N), dtype=np.uint64)
    ob = np.zeros_like(oa)
    _load().or_rotate(P.c, ell, _u(a), _u(b), g, _u(key), _u(oa), _u(ob))
    return oa, ob


def hrotate(P: Params, ell, a, b, gs, keys):
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    keys = [np.ascontiguousarray(k, dtype=np.uint64) for k in keys]
    r = len(gs)
    g_arr = np.ascontiguousarray(np.asarray(gs, dtype=np.uint64))
    oas = [np.zeros((ell, P.N), dtype=np.uint64) for _ in range(r)]
    obs = [np.zeros((ell, P.N), dtype=np.uint64) for _ in range(r)]
    _load().or_hrotate(P.c, ell, _u(a), _u(b), r, _u(g_arr), _ptr_array(keys), _ptr_array(oas), _ptr_array(obs))
    return list(zip(oas, obs))


def ptmatvec(P: Params, ell, a, b, nb, ng, g_baby, g_giant, key_baby, key_giant, diags, rescale_out=True):
    """Algorithm 8 with nb baby steps and ng giant steps.

    g_baby[0] / key_baby[0] and g_giant[0] / key_giant[0] are unused (identity).
    diags is a list of nb*ng arrays [ell+k][N], index t*nb + i."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    gb = np.ascontiguousarray(np.asarray(g_baby, dtype=np.uint64))
    gg = np.ascontiguousarray(np.asarray(g_giant, dtype=np.uint64))
    kb = [None if k is None else np.ascontiguousarray(k, dtype=np.uint64) for k in key_baby]
    kg = [None if k is None else np.ascontiguousarray(k, dtype=np.uint64) for k in key_giant]
    ds = [np.ascontiguousarray(d, dtype=np.uint64) for d in diags]
    out_l = ell - 1 if rescale_out else ell
    oa = np.zeros((out_l, P.N), dtype=np.uint64)
    ob = np.zeros_like(oa)
    _load().or_ptmatvec(P.c, ell, _u(a), _u(b), nb, ng, _u(gb), _u(gg), _ptr_array(kb), _ptr_array(kg),
                        _ptr_array(ds), int(bool(rescale_out)), _u(oa), _u(ob))
    return oa, ob


# ---------------------------------------------------------------- keys and encryption (test data)
def signed_to_eval(P: Params, c):
    c = np.ascontiguousarray(c, dtype=np.int64)
    out = np.zeros((P.L + P.k, P.N), dtype=np.uint64)
    _load().or_signed_to_eval(P.c, _i(c), _u(out))
    return out


def rot_secret(P: Params, s, g):
    s = np.ascontiguousarray(s, dtype=np.int64)
    out = np.zeros((P.L + P.k, P.N), dtype=np.uint64)
    _load().or_rot_secret(P.c, _i(s), g, _u(out))
    return out


def sq_secret(P: Params, s):
    s = np.ascontiguousarray(s, dtype=np.int64)
    out = np.zeros((P.L + P.k, P.N), dtype=np.uint64)
    _load().or_sq_secret(P.c, _i(s), _u(out))
    return out


def keygen(P: Params, a, s, sp_eval, e):
    """Key [dnum][2][L+k][N] switching s' (sp_eval) to s."""
    a = np.ascontiguousarray(a, dtype=np.uint64)
    s = np.ascontiguousarray(s, dtype=np.int64)
    sp_eval = np.ascontiguousarray(sp_eval, dtype=np.uint64)
    e = np.ascontiguousarray(e, dtype=np.int64)
    key = np.zeros((P.dnum, 2, P.L + P.k, P.N), dtype=np.uint64)
    _load().or_keygen(P.c, _u(a), _i(s), _u(sp_eval), _i(e), _u(key))
    return key


def prng_key_a(P: Params, seed: int):
    """The uniform half a of a compressed key: [dnum][L+k][N] from the seed (Sec. 5.3)."""
    a = np.zeros((P.dnum, P.L + P.k, P.N), dtype=np.uint64)
    _load().or_prng_key_a_fill(P.c, seed & 0xFFFFFFFFFFFFFFFF, _u(a))
    return a


def prng_key_a_element(P: Params, seed: int, j: int, l: int, n: int) -> int:
    return int(_load().or_prng_key_a(P.c, seed & 0xFFFFFFFFFFFFFFFF, j, l, n))


def encrypt(P: Params, ell, s, m_plus_e, a):
    s = np.ascontiguousarray(s, dtype=np.int64)
    me = np.ascontiguousarray(m_plus_e, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.zeros((ell, P.N), dtype=np.uint64)
    _load().or_encrypt(P.c, ell, _i(s), _i(me), _u(a), _u(b))
    return b


def decrypt_residues(P: Params, ell, s, a, b):
    s = np.ascontiguousarray(s, dtype=np.int64)
    a = np.ascontiguousarray(a, dtype=np.uint64)
    b = np.ascontiguousarray(b, dtype=np.uint64)
    out = np.zeros((ell, P.N), dtype=np.uint64)
    _load().or_decrypt(P.c, ell, _i(s), _u(a), _u(b), _u(out))
    return out
