"""Algorithmic (compulsory) bytes and operation counts of the key-switching
path, used as roofline numerators.

Two models:

* ``compulsory_*``: what this library must move between HBM and the chip for
  one operation if every intermediate stays on chip -- inputs, keys and
  outputs, 8-byte words, ell and L counting limbs.
* ``paper_*``: the per-subroutine DRAM counts of the paper's tables "Hardware
  Cost of Auxiliary Subroutines" and "Hardware Cost of FHE APIs" (Sec. 2.5),
  whose limb counts use the paper's own convention of ell+1 chain limbs and a
  raised basis of ell+1+alpha limbs with alpha = ceil((L+1)/dnum).  They pin
  the accounting against the numbers the paper prints.
"""
from __future__ import annotations

from math import ceil

WORD = 8


def limb_bytes(N: int) -> int:
    return N * WORD


# ------------------------------------------------------------------ this library
def alpha_of(L: int, dnum: int) -> int:
    return ceil(L / dnum)


def beta_of(ell: int, L: int, dnum: int) -> int:
    return ceil(ell / alpha_of(L, dnum))


def key_limbs(ell: int, k: int, L: int, dnum: int) -> int:
    """Key limbs one KeySwitch at level ell reads: 2 rows x beta digits x (ell+k)."""
    return 2 * beta_of(ell, L, dnum) * (ell + k)


def compulsory_keyswitch_bytes(N, ell, k, L, dnum) -> int:
    """a in (ell limbs) + key + (u, v) out (2 ell limbs)."""
    return (ell + key_limbs(ell, k, L, dnum) + 2 * ell) * limb_bytes(N)


def compulsory_hrotate_bytes(N, ell, k, L, dnum, r) -> int:
    """(a, b) in once, then per rotation a key and an output ciphertext."""
    return (2 * ell + r * (key_limbs(ell, k, L, dnum) + 2 * ell)) * limb_bytes(N)


def compulsory_batch_keyswitch_bytes(N, levels, keys, k, L, dnum) -> int:
    """A batch of KeySwitches: every entry's a in and (u, v) out (3 ell limbs),
    plus every key limb some entry touches, read once (keys[i] names entry i's
    key; entries with equal names share it)."""
    touched = set()
    for ell, key in zip(levels, keys):
        for j in range(beta_of(ell, L, dnum)):
            for row in range(2):
                for t in range(ell + k):
                    prime = t if t < ell else L + (t - ell)
                    touched.add((key, j, row, prime))
    return (3 * sum(levels) + len(touched)) * limb_bytes(N)


def ntt_bytes_per_limb(N) -> int:
    """One transform of one limb: read it once, write it once."""
    return 2 * limb_bytes(N)


def ntt_butterflies_per_limb(N) -> int:
    return (N // 2) * (N.bit_length() - 1)


def keyswitch_ntt_limbs(ell, k, L, dnum) -> int:
    """Limb transforms in one KeySwitch: iNTT of the ell input limbs, NTT of the
    beta*(ell+k) - ell new ModUp limbs, iNTT of 2k P-limbs and NTT of 2 ell
    ModDown limbs."""
    beta = beta_of(ell, L, dnum)
    return ell + (beta * (ell + k) - ell) + 2 * k + 2 * ell


# ------------------------------------------------------------------ the paper's tables
def paper_alpha(L: int, dnum: int) -> int:
    """alpha = ceil((L+1)/dnum) of Table 1 (L counts the limbs above q_0)."""
    return ceil((L + 1) / dnum)


def paper_raised_limbs(ell: int, dnum: int) -> int:
    return ell + 1 + paper_alpha(ell, dnum)


def paper_key_read_bytes(N, ell, dnum) -> int:
    """KSKInnerProd key reads: 2 rows x dnum digits x raised limbs."""
    return 2 * dnum * paper_raised_limbs(ell, dnum) * limb_bytes(N)


def paper_kskinnerprod_limb_read_bytes(N, ell, dnum) -> int:
    return dnum * paper_raised_limbs(ell, dnum) * limb_bytes(N)


def paper_moddown_limb_read_bytes(N, ell, dnum) -> int:
    return 2 * paper_raised_limbs(ell, dnum) * limb_bytes(N)


def paper_decomp_read_bytes(N, ell) -> int:
    return ell * limb_bytes(N)


def paper_automorph_read_bytes(N, ell) -> int:
    return 2 * ell * limb_bytes(N)


def paper_ciphertext_bytes(N, ell) -> int:
    return 2 * N * ell * WORD


def bootstrap_throughput(n, ell, bp, dram_gb, bw_gbs) -> float:
    """Eq. (bootThroughput) with DRAM time as the runtime proxy, in 10^6."""
    return n * ell * bp / (dram_gb / bw_gbs) / 1e6
