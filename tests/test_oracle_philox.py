"""Pins for the oracle's Philox4x32-10 and the input generator's copy of it.

Both are checked against the generator's published known-answer values
(tests/golden/philox4x32_10_kat.txt) and against distribution statistics.
"""
import os

import numpy as np
import pytest

import oracle
from paper_2605_30294_gb300 import inputs


def _kat(golden_dir):
    rows = []
    with open(os.path.join(golden_dir, "philox4x32_10_kat.txt")) as f:
        for line in f:
            line = line.strip()
            if not line or line.startswith("#"):
                continue
            rows.append([int(x, 16) for x in line.split()])
    return np.array(rows, dtype=np.uint64).astype(np.uint32)


def test_oracle_philox_known_answers(golden_dir):
    kat = _kat(golden_dir)
    out = oracle.philox4x32_10(kat[:, 0:4], kat[:, 4:6])
    np.testing.assert_array_equal(out, kat[:, 6:10])


def test_input_generator_philox_known_answers(golden_dir):
    kat = _kat(golden_dir)
    for row in kat:
        r = inputs.philox4x32_10(row[0], row[1], row[2], row[3], row[4], row[5])
        assert [int(x) for x in r] == [int(x) for x in row[6:10]]


def test_philox_oracle_and_generator_agree_on_many_counters():
    rng = np.random.default_rng(7)
    ctr = rng.integers(0, 2**32, size=(4096, 4), dtype=np.uint64).astype(np.uint32)
    key = np.array([12345, 1], np.uint32)
    a = oracle.philox4x32_10(ctr, key)
    b = np.stack(inputs.philox4x32_10(ctr[:, 0], ctr[:, 1], ctr[:, 2], ctr[:, 3], 12345, 1), 1)
    np.testing.assert_array_equal(a, b)


def test_philox_statistics():
    # 2^16 counters x 4 words: bit balance and byte-histogram chi^2.
    n = 1 << 16
    ctr = np.zeros((n, 4), np.uint32)
    ctr[:, 0] = np.arange(n, dtype=np.uint32)
    out = oracle.philox4x32_10(ctr, np.array([1, 0], np.uint32))
    bits = np.unpackbits(out.view(np.uint8)).reshape(-1)
    frac = bits.mean()
    assert abs(frac - 0.5) < 5 * 0.5 / np.sqrt(bits.size)
    hist = np.bincount(out.view(np.uint8).reshape(-1), minlength=256)
    exp = out.size * 4 / 256
    chi2 = ((hist - exp) ** 2 / exp).sum()
    # 255 dof: mean 255, sd ~22.6; a 6-sigma band
    assert 120 < chi2 < 400
    # consecutive counters decorrelate: lag-1 correlation of word 0
    x = out[:, 0].astype(np.float64)
    c = np.corrcoef(x[:-1], x[1:])[0, 1]
    assert abs(c) < 5 / np.sqrt(n)


def test_c1_items_layout():
    items = inputs.c1_items(9, seed=3)
    for i in (0, 5, 8):
        for j in range(4):
            r = oracle.philox4x32_10(np.array([[i, j, 0, 0]], np.uint32), np.array([3, 0], np.uint32))
            np.testing.assert_array_equal(items[i, 4 * j:4 * j + 4], r[0])


@pytest.mark.parametrize("n", [0, 1, 1000])
def test_c1_items_sizes(n):
    assert inputs.c1_items(n).shape == (n, 16)
