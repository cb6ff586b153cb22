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


def test_loss_power_is_the_dissipated_energy_per_cycle(orc):
    """Energy balance of Eq. 1 pins the specific-loss-power formula: at T = 0 the damping term
    dissipates mu0 Ms alpha g1 |m x H_eff|^2 per unit volume and time, and over a closed loop this
    equals the field's work, mu0 Ms times the loop area (H in A/m).  A single macrospin with a
    5-degree tilted easy axis, relaxed at +H_max and then driven through one full loop, is
    integrated step by step with the oracle; the dissipated energy from the trajectory must equal
    the energy per cycle that the formula implies, SLP rho / f."""
    u = (math.sin(math.radians(5)), 0.0, math.cos(math.radians(5)))
    kw = dict(a0=5e-9, b=1, A0=0.0, K0=1e4, Ms=480e3, alpha=1.0, T=0.0, dt=1e-12, mode=0, u=u)
    p = orc.material_problem(1, 1, 1, H_start_Oe=1000.0, H_turn_Oe=-1000.0, rate_Oe_per_ns=200.0, **kw)
    relax = orc.material_problem(1, 1, 1, H_start_Oe=1000.0, H_turn_Oe=1000.0, rate_Oe_per_ns=0.0, **kw)
    c = orc.coefficients(p)
    m = orc.uniform_state(1, 1)
    orc.run(relax, m, n_steps=5000, threads=1)
    N = 2 * p.n_half
    mv = np.empty((N + 1, 3))
    H = np.empty(N + 1)
    mv[0], H[0] = m[0, 0], orc.field_Oe(p, 0)
    for n in range(N):
        orc.run(p, m, step0=n, n_steps=1, threads=1)
        mv[n + 1], H[n + 1] = m[0, 0], orc.field_Oe(p, n + 1)
    assert mv[:, 2].min() < -0.99 and np.abs(mv[-1] - mv[0]).max() < 1e-3  # switched and closed
    uu = np.asarray(u)
    Heff = c["c_an"] * (mv @ uu)[:, None] * uu[None, :] + np.outer(H * 1000.0 / (4 * math.pi), [0, 0, 1])
    cr = np.cross(mv, Heff)
    power = c["ag1"] * np.sum(cr * cr, axis=1)  # alpha g1 |m x H|^2, A^2 / (m^2 s)
    mu0 = 4e-7 * math.pi
    dissipated = mu0 * p.Ms * np.sum(0.5 * (power[1:] + power[:-1])) * p.dt  # J / m^3 per cycle
    area = orc.loop_area(H, mv[:, 2])
    f, rho = 1e5, 5.17  # Hz, g/cm^3
    per_cycle = orc.specific_loss_power(f, p.Ms, area, rho) * rho * 1e6 / f
    assert per_cycle == pytest.approx(dissipated, rel=1e-4)
    assert area > 1000.0
