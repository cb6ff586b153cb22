"""Pins of the loop observables (m_H averaged over realisations, coercive field with one
standard error, loop area) against analytic loops."""
import math

import numpy as np
import pytest


def _triangle(Hm, n_half):
    down = np.linspace(Hm, -Hm, n_half + 1)
    return np.concatenate([down, down[-2::-1]])


def test_tanh_loop_coercive_field_and_area(orc):
    Hm, Hc, w, n_half = 1500.0, 300.0, 60.0, 3000
    H = _triangle(Hm, n_half)
    m = np.where(np.arange(len(H)) <= n_half, np.tanh((H + Hc) / w), np.tanh((H - Hc) / w))
    hc, down, up = orc.coercive_field(H, m, n_half)
    assert down == pytest.approx(-Hc, abs=1e-3)
    assert up == pytest.approx(Hc, abs=1e-3)
    assert hc == pytest.approx(Hc, abs=1e-3)
    F = lambda x: w * math.log(math.cosh(x / w))
    exact = (F(Hm + Hc) - F(-Hm + Hc)) - (F(Hm - Hc) - F(-Hm - Hc))
    assert orc.loop_area(H, m) == pytest.approx(exact, rel=1e-5)


def test_rectangular_loop_area_is_four_hc(orc):
    Hm, Hc, n_half = 1000.0, 250.5, 2000
    H = _triangle(Hm, n_half)
    k = np.arange(len(H))
    m = np.where(k <= n_half, np.where(H > -Hc, 1.0, -1.0), np.where(H < Hc, -1.0, 1.0))
    assert orc.loop_area(H, m) == pytest.approx(4 * Hc, abs=1e-9)
    hc, _, _ = orc.coercive_field(H, m, n_half)
    assert hc == pytest.approx(Hc, abs=1e-9)


def test_first_crossing_after_turning_point(orc):
    # a noisy branch that recrosses zero: the first crossing after the start is taken
    H = _triangle(100.0, 200)
    m = np.ones_like(H)
    m[50:] = -1.0  # descending crosses at H between samples 49 and 50
    m[60] = 0.5    # a later recrossing is ignored
    m[250:] = 1.0  # ascending crosses between samples 249 and 250
    _, down, up = orc.coercive_field(H, m, 200)
    assert down == pytest.approx(0.5 * (H[49] + H[50]))
    assert up == pytest.approx(0.5 * (H[249] + H[250]))


def test_jackknife_errors(orc):
    Hm, n_half, R = 500.0, 500, 40
    H = _triangle(Hm, n_half)
    rng = np.random.default_rng(0)
    hcs = rng.normal(100.0, 10.0, size=R)
    k = np.arange(len(H))
    samples = np.stack([np.where(k <= n_half, np.tanh((H + h) / 50.0), np.tanh((H - h) / 50.0))
                        for h in hcs])
    st = orc.loop_stats(H, samples, n_half)
    assert np.allclose(st["mean"], samples.mean(axis=0))
    # the area is linear in m, so its delete-one jackknife error equals the standard error of
    # the per-realisation areas
    areas = np.array([orc.loop_area(H, s) for s in samples])
    assert st["area"] == pytest.approx(areas.mean(), rel=1e-12)
    assert st["area_se"] == pytest.approx(areas.std(ddof=1) / math.sqrt(R), rel=1e-9)
    # Hc error is of the order of the spread of the per-realisation coercive fields / sqrt(R)
    assert 0.3 < st["Hc_se"] / (hcs.std(ddof=1) / math.sqrt(R)) < 3.0
    # identical realisations have zero error
    same = orc.loop_stats(H, np.repeat(samples[:1], 5, axis=0), n_half)
    assert same["Hc_se"] == pytest.approx(0.0, abs=1e-12)
    assert same["area_se"] == pytest.approx(0.0, abs=1e-9)
