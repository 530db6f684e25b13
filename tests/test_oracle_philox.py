"""Pins for the oracle's Philox-4x32-10 and its (0,1) mapping.

Philox is the counter-based generator both sides implement from its
published definition (Salmon et al., SC'11); these known answers come with
that publication's reference library.
"""
import os

import numpy as np

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "philox4x32_10_kat.txt")


def _kat_rows():
    rows = []
    for line in open(GOLDEN):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        rows.append([int(w, 16) for w in line.split()])
    return rows


def test_known_answers():
    rows = _kat_rows()
    assert len(rows) == 3
    for r in rows:
        out = oracle.philox4x32_10(r[0:4], r[4:6])
        assert out.tolist() == r[6:10]


def test_u01_open_interval_and_exact_in_fp32():
    for r in [0, 1, 511, 512, 0x7FFFFFFF, 0x80000000, 0xFFFFFFFF, 0x12345678]:
        u = oracle.u01(r)
        assert 0.0 < u < 1.0
        assert float(np.float32(u)) == u
    assert oracle.u01(0) == 2.0 ** -24
    assert oracle.u01(0xFFFFFFFF) == 1.0 - 2.0 ** -24


def test_uniformity_chi_square():
    # 4 x 8192 words from consecutive counters, 64 equal bins.
    us = []
    for i in range(8192):
        out = oracle.philox4x32_10([i, 0, 0, 0], [7, 0])
        us += [oracle.u01(int(w)) for w in out]
    us = np.asarray(us)
    counts, _ = np.histogram(us, bins=64, range=(0.0, 1.0))
    exp = us.size / 64
    chi2 = np.sum((counts - exp) ** 2 / exp)
    # 63 dof: mean 63, sd ~11.2; 5-sigma band
    assert 63 - 56 < chi2 < 63 + 56
    assert abs(us.mean() - 0.5) < 5 * np.sqrt(1 / 12 / us.size)
