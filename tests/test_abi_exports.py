"""The C-ABI library loads and exports every function include/ckks_ks.h
declares (no GPU needed: no compute call is made)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            src = open(os.path.join(ROOT, "include", fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ckks_[a-z0-9_]+)\s*\(", src))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    from paper_2112_06396_gb300 import build

    try:
        path = build.build()
    except RuntimeError as e:  # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(path)
    names = declared_functions()
    assert len(names) >= 18
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_declared_symbol():
    from paper_2112_06396_gb300 import ckks

    assert sorted(ckks.exported_symbols()) == declared_functions()


def test_host_prime_generation_matches_oracle(oracle_lib):
    from paper_2112_06396_gb300 import build, ckks

    try:
        build.build()
    except RuntimeError as e:
        pytest.skip(str(e))
    for bits, logN, count in [(50, 12, 9), (54, 16, 32), (54, 15, 32)]:
        assert ckks.ckks_gen_primes(bits, logN, count) == oracle_lib.gen_primes(bits, logN, count)
