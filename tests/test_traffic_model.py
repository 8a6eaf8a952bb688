"""The byte accounting used for roofline numerators, pinned to the numbers the
paper prints (tests/golden/paper_tables.json, each entry cites its table)."""
import json
import os

import pytest

from paper_2112_06396_gb300 import traffic as T

G = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_tables.json")))
N, ELL, DNUM = 1 << G["params"]["logN"], G["params"]["ell"], G["params"]["dnum"]


def gb(x):
    return x / 1e9


def test_ciphertext_size():
    assert round(T.paper_ciphertext_bytes(N, ELL) / 1e6, 1) == G["ciphertext_MB"]["value"]


@pytest.mark.parametrize("name,fn", [
    ("kskinnerprod_key_reads_GB", lambda: T.paper_key_read_bytes(N, ELL, DNUM)),
    ("kskinnerprod_limb_reads_GB", lambda: T.paper_kskinnerprod_limb_read_bytes(N, ELL, DNUM)),
    ("moddown_limb_reads_GB", lambda: T.paper_moddown_limb_read_bytes(N, ELL, DNUM)),
    ("decomp_limb_reads_GB", lambda: T.paper_decomp_read_bytes(N, ELL)),
    ("automorph_limb_reads_GB", lambda: T.paper_automorph_read_bytes(N, ELL)),
    ("hrotate8_key_reads_GB", lambda: 8 * T.paper_key_read_bytes(N, ELL, DNUM)),
])
def test_paper_dram_counts(name, fn):
    assert round(gb(fn()), 4) == G[name]["value"]


def test_alpha_example():
    e = G["alpha_example"]
    assert T.paper_alpha(e["L"], e["dnum"]) == e["value"]


def test_bootstrapping_throughput_arithmetic():
    for row in G["bootstrapping_comparison"]["rows"]:
        got = T.bootstrap_throughput(row["n"], row["ell"], row["bp"], row["dram_GB"], row["bw_GBs"])
        assert abs(got - row["throughput"]) <= 0.011 * max(1.0, row["throughput"] / 100), (row["work"], got)


def test_headline_compulsory_bytes():
    # N=2^16, ell=L=24, k=8, dnum=3: 24 + 192 + 48 limbs of 512 KiB
    assert T.key_limbs(24, 8, 24, 3) == 192
    assert T.compulsory_keyswitch_bytes(1 << 16, 24, 8, 24, 3) == 264 * (1 << 19)
    assert T.compulsory_hrotate_bytes(1 << 16, 24, 8, 24, 3, 1) == 288 * (1 << 19)
    assert T.keyswitch_ntt_limbs(24, 8, 24, 3) == 160
