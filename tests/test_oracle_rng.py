"""Pins of the oracle's noise source: Philox4x32-10 against published known-answer vectors, and
the Box-Muller normals against the standard normal law (thermal field after Eq. 1)."""
import numpy as np
import pytest
from scipy import stats

from helpers import read_golden


def test_philox_known_answers(orc):
    rows = read_golden("philox_kat.txt")
    assert len(rows) == 3
    for row in rows:
        w = [int(x, 16) for x in row]
        out = orc.philox4x32_10(w[0:4], w[4:6])
        assert [int(v) for v in out] == w[6:10]


def test_uniform24_range(orc):
    # 24-bit uniforms are strictly inside (0, 1) and symmetric about 1/2
    assert orc.uniform24(0) == pytest.approx(0.5 / 2 ** 24, rel=0, abs=0)
    assert orc.uniform24(0xFFFFFFFF) == 1.0 - 0.5 / 2 ** 24
    assert orc.uniform24(0x80000000) == 0.5 + 0.5 / 2 ** 24
    assert orc.uniform24(0x000000FF) == orc.uniform24(0)  # low byte is dropped


def test_normals_are_standard_normal(orc):
    # 3 x 20000 draws over cells and steps: mean 0, variance 1, Kolmogorov-Smirnov vs N(0,1),
    # and the three components uncorrelated.
    draws = np.array([orc.thermal_normals(5, 3, cell, step)
                      for cell in range(200) for step in range(100)])
    assert draws.shape == (20000, 3)
    for k in range(3):
        x = draws[:, k]
        assert abs(x.mean()) < 4 / np.sqrt(len(x))
        assert abs(x.var() - 1.0) < 4 * np.sqrt(2 / len(x))
        assert stats.kstest(x, "norm").pvalue > 1e-3
    c = np.corrcoef(draws.T)
    assert np.all(np.abs(c[np.triu_indices(3, 1)]) < 4 / np.sqrt(len(draws)))


def test_normals_depend_on_every_key_and_counter_word(orc):
    base = orc.thermal_normals(1, 2, 3, 4)
    for args in [(9, 2, 3, 4), (1, 9, 3, 4), (1, 2, 9, 4), (1, 2, 3, 9), (1, 2, 3, 4 + (1 << 32))]:
        assert not np.allclose(orc.thermal_normals(*args), base)
    assert np.array_equal(orc.thermal_normals(1, 2, 3, 4), base)
