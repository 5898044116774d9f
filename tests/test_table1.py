"""The byte accounting against the paper's Table 1 (tests/golden/table1_paper.json,
values typed from Sec. 3.2 of arXiv:1206.0675): the per-thread loads and stores
of k2, k5 and k6 for 18- and 12-real storage, and the FFT flop formula."""

import json
import os

import pytest

from paper_1206_0675_gb300 import accounting

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "table1_paper.json")


def test_loads_and_stores_match_table1():
    with open(GOLDEN) as f:
        t1 = json.load(f)
    for storage, rows in (("18real", 3), ("12real", 2)):
        ours = accounting.table1_counts(rows)
        for k in ("k2", "k5", "k6"):
            loads, stores, _flop = t1[storage][k]
            assert ours[k] == (loads, stores), (storage, k)


def test_fft_flop_formula():
    # 32^4: 5 (log2 1024 + log2 1024) = 100 flop per site and FFT
    assert accounting.paper_fft_flops_per_site((32, 32, 32, 32)) == 100.0
    # 48^3 x 96: 5 (2 log2 48 + 2 log2 48 + 1) with log2 48 = 4 + log2 3
    assert accounting.paper_fft_flops_per_site((48, 48, 48, 96)) == pytest.approx(116.69925001442312, rel=1e-14)
