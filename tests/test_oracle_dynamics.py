"""Deterministic (T = 0) pins of the oracle's integrator: Eq. 1 against closed forms."""
import math
import threading

import numpy as np
import pytest

from workloads import random_unit_state


def _single(orc, *, alpha, K=0.0, H_Oe=1000.0, dt=1e-14, u=(0, 0, 1), Ms=480e3, n_half=0,
            H_turn=None):
    return orc.Problem(1, 1, 1, a=3e-9, A=0.0, K=K, Ms=Ms, alpha=alpha, T=0.0, dt=dt,
                       H_start_Oe=H_Oe, H_turn_Oe=H_Oe if H_turn is None else H_turn,
                       n_half=n_half, u=u)


def _angles(m):
    return math.acos(max(-1.0, min(1.0, m[2]))), math.atan2(m[1], m[0])


def test_larmor_precession(orc):
    """alpha = 0, K = 0: m precesses counter-clockwise about +z at g0 H with theta fixed; the
    Heun phase error converges at least quadratically in dt."""
    H_Oe, th0, t_end = 1000.0, 0.5, 2e-11
    g0 = orc.MU0 * orc.GAMMA_E
    errs = []
    for dt in (1e-14, 5e-15):
        p = _single(orc, alpha=0.0, H_Oe=H_Oe, dt=dt)
        m = np.array([[[math.sin(th0), 0.0, math.cos(th0)]]])
        orc.run(p, m, n_steps=int(round(t_end / dt)))
        th, ph = _angles(m[0, 0])
        expect = math.remainder(g0 * H_Oe * orc.OE * t_end, 2 * math.pi)
        errs.append(abs(math.remainder(ph - expect, 2 * math.pi)))
        assert abs(th - th0) < 1e-9
    assert errs[0] < 1e-7
    assert errs[0] / errs[1] > 3.5  # order >= 2


def test_damped_precession(orc):
    """alpha > 0, K = 0: tan(theta/2) = tan(theta0/2) exp(-alpha g1 H t), phi' = g1 H."""
    alpha, H_Oe, th0, dt, n = 0.5, 1000.0, 2.5, 5e-15, 8000
    g1 = orc.MU0 * orc.GAMMA_E / (1 + alpha * alpha)
    H = H_Oe * orc.OE
    p = _single(orc, alpha=alpha, H_Oe=H_Oe, dt=dt)
    m = np.array([[[math.sin(th0), 0.0, math.cos(th0)]]])
    orc.run(p, m, n_steps=n)
    t = n * dt
    th, ph = _angles(m[0, 0])
    th_x = 2 * math.atan(math.tan(th0 / 2) * math.exp(-alpha * g1 * H * t))
    assert th == pytest.approx(th_x, rel=1e-6)
    assert math.remainder(ph - g1 * H * t, 2 * math.pi) == pytest.approx(0.0, abs=1e-6)


def test_stoner_wohlfarth_astroid(orc):
    """T = 0 single macrospin with the easy axis at psi from the swept field: the magnetisation
    jumps at h_sw H_K, h_sw = (cos^(2/3) psi + sin^(2/3) psi)^(-3/2), H_K = 2K/(mu0 Ms).  A slow
    sweep (0.1 Oe/ns, alpha = 1) lands within 1%."""
    K, Ms, rate, dt, dH = 1e4, 480e3, 0.1, 2e-13, 0.02
    HK_Oe = 2 * K / (orc.MU0 * Ms) / orc.OE
    results = {}

    def one(psi_deg):
        psi = math.radians(psi_deg)
        u = (math.sin(psi), 0.0, math.cos(psi))
        n_half = orc.sweep_steps(0.0, -400.0, rate, dt)
        p = _single(orc, alpha=1.0, K=K, H_Oe=0.0, H_turn=-400.0, dt=dt, u=u, Ms=Ms,
                    n_half=n_half)
        m = np.array([[list(u)]])
        every = orc.sample_interval(dH, rate, dt)
        ns = n_half // every + 1
        s, _ = orc.run(p, m, n_steps=n_half, sample_every=every, n_samples=ns, threads=1)
        s[0, 0] = u[2]
        H = np.array([orc.field_Oe(p, k * every) for k in range(ns)])
        _, down, _ = orc.coercive_field(H, s[0], ns - 1)
        results[psi_deg] = -down / HK_Oe

    ts = [threading.Thread(target=one, args=(d,)) for d in (5.0, 30.0)]
    [t.start() for t in ts]
    [t.join() for t in ts]
    for psi_deg, got in results.items():
        psi = math.radians(psi_deg)
        h_sw = (math.cos(psi) ** (2 / 3) + math.sin(psi) ** (2 / 3)) ** -1.5
        assert abs(got - h_sw) / h_sw < 0.01, (psi_deg, got, h_sw)
        assert got > h_sw  # a finite sweep rate only delays the jump


def _grid(orc, dims, *, A=1e-11, K=1e4, alpha=0.1, H_Oe=300.0, dt=5e-15, periodic=0, T=0.0,
          a=2e-9, u=(0, 0, 1)):
    return orc.Problem(*dims, a=a, A=A, K=K, Ms=480e3, alpha=alpha, T=T, dt=dt, H_start_Oe=H_Oe,
                       H_turn_Oe=H_Oe, n_half=0, periodic=periodic, u=u)


@pytest.mark.parametrize("periodic", [0, 0b111, 0b011])
def test_energy_decreases_at_zero_temperature(orc, periodic):
    """At T = 0 and constant field, damping makes the energy whose gradient is H_eff
    non-increasing; a field term inconsistent with that energy (wrong neighbour, sign or factor)
    breaks monotonicity."""
    dims = (3, 4, 5)
    u = (0.3, -0.2, 0.933)
    un = np.array(u) / np.linalg.norm(u)
    p = _grid(orc, dims, periodic=periodic, u=tuple(un))
    m = np.ascontiguousarray(random_unit_state(1, 60, seed=3))
    e_prev = orc.energy(p, m[0], 300.0)
    e0 = e_prev
    for n in range(300):
        orc.run(p, m, n_steps=1, step0=n)
        e = orc.energy(p, m[0], 300.0)
        assert e <= e_prev + 1e-12 * abs(e0), n
        e_prev = e
    assert e_prev < e0


@pytest.mark.parametrize("periodic", [0, 0b111])
def test_exchange_conserves_total_moment(orc, periodic):
    """Exchange alone (K = 0, H = 0, alpha = 0, T = 0): pairwise torques cancel, so sum_i m_i and
    the exchange energy are invariants of Eq. 1.  The Heun drift is a discretisation error: it
    must shrink at least fourfold when dt halves (an asymmetric neighbour would leave an O(1)
    drift that does not converge)."""
    drifts, edrifts = [], []
    for dt, n in ((1e-15, 2000), (5e-16, 4000)):
        p = _grid(orc, (3, 4, 5), K=0.0, alpha=0.0, H_Oe=0.0, dt=dt, periodic=periodic)
        m = np.ascontiguousarray(random_unit_state(1, 60, seed=4, cone=1.0))
        s0 = m[0].sum(axis=0)
        e0 = orc.energy(p, m[0], 0.0)
        orc.run(p, m, n_steps=n)
        drifts.append(np.max(np.abs(m[0].sum(axis=0) - s0)))
        edrifts.append(abs(orc.energy(p, m[0], 0.0) - e0) / abs(e0))
        assert np.max(np.abs(np.linalg.norm(m[0], axis=-1) - 1)) < 1e-14
    assert drifts[0] < 1e-4 * 60
    assert drifts[1] < drifts[0] / 4
    assert edrifts[0] < 1e-3
    assert edrifts[1] < edrifts[0] / 4


@pytest.mark.parametrize("axis", [0, 1, 2])
def test_two_spin_exchange_precession(orc, axis):
    """Two cells along one axis, exchange only, alpha = 0: each spin precesses about
    S = m1 + m2 at g0 c_ex |S|, c_ex = 2A/(mu0 Ms a^2)."""
    dims = [1, 1, 1]
    dims[axis] = 2
    A, a, Ms, dt, n = 1e-11, 2e-9, 480e3, 2e-16, 5000
    p = orc.Problem(*dims, a=a, A=A, K=0.0, Ms=Ms, alpha=0.0, T=0.0, dt=dt)
    m = np.ascontiguousarray(random_unit_state(1, 2, seed=10 + axis))
    m1, S = m[0, 0].copy(), m[0].sum(axis=0)
    c_ex = 2 * A / (orc.MU0 * Ms * a * a)
    w = orc.MU0 * orc.GAMMA_E * c_ex * np.linalg.norm(S)
    orc.run(p, m, n_steps=n)
    s = S / np.linalg.norm(S)
    ang = w * n * dt
    par = np.dot(m1, s) * s
    perp = m1 - par
    expect = par + perp * math.cos(ang) + np.cross(s, perp) * math.sin(ang)
    assert ang > 1.0
    assert np.max(np.abs(m[0, 0] - expect)) < 1e-6
    assert np.max(np.abs(m[0].sum(axis=0) - S)) < 1e-9


def test_uniform_grid_matches_single_macrospin(orc):
    """A uniformly magnetised grid feels no exchange torque: at T = 0 every cell follows the
    single-macrospin trajectory under anisotropy and a swept field."""
    dims = (2, 3, 4)
    kw = dict(A=1e-11, K=2e4, alpha=0.2, dt=5e-15, T=0.0)
    n_half = orc.sweep_steps(500.0, -500.0, 1e4, kw["dt"])
    pg = orc.Problem(*dims, a=2e-9, Ms=480e3, H_start_Oe=500.0, H_turn_Oe=-500.0, n_half=n_half,
                     u=(0.1, 0.0, 0.995), **kw)
    ps = orc.Problem(1, 1, 1, a=2e-9, Ms=480e3, H_start_Oe=500.0, H_turn_Oe=-500.0, n_half=n_half,
                     u=(0.1, 0.0, 0.995), **kw)
    d = (0.3, 0.1, 0.95)
    mg = orc.uniform_state(1, 24, d)
    ms = orc.uniform_state(1, 1, d)
    orc.run(pg, mg, n_steps=20000)
    orc.run(ps, ms, n_steps=20000)
    assert np.max(np.abs(mg[0] - ms[0, 0])) < 1e-12


def test_triangle_sweep(orc):
    p = orc.Problem(1, 1, 1, a=1e-9, A=0, K=0, Ms=1, alpha=0.1, T=0, dt=1e-14, H_start_Oe=1500.0,
                    H_turn_Oe=-1500.0, n_half=orc.sweep_steps(1500, -1500, 1000, 1e-14))
    assert p.n_half == 300000
    assert orc.field_Oe(p, 0) == 1500.0
    assert orc.field_Oe(p, 100) == pytest.approx(1499.0, abs=1e-9)
    assert orc.field_Oe(p, 300000) == -1500.0
    assert orc.field_Oe(p, 450000) == pytest.approx(0.0, abs=1e-9)
    assert orc.field_Oe(p, 600000) == 1500.0
    assert orc.field_Oe(p, 600100) == pytest.approx(1499.0, abs=1e-9)
    assert orc.sample_interval(1.0, 1000.0, 1e-14) == 100


def test_sinusoidal_sweep(orc):
    """The paper's sinusoid H_max sin(2 pi f t) with SR = 4 H_max f: a cycle of 4 H_max / SR,
    extremes +-H_max a half cycle apart, zeros at the quarter points, total variation 4 H_max
    per cycle (so the mean |dH/dt| is SR) and peak slope 2 pi f H_max."""
    dt, Hm, rate = 1e-14, 1500.0, 1000.0
    p = orc.material_problem(1, 1, 1, a0=1e-9, b=1, A0=0.0, K0=0.0, Ms=1.0, alpha=0.1, T=0.0, dt=dt,
                             mode=0, H_start_Oe=Hm, rate_Oe_per_ns=rate, shape=1)
    P = p.period
    assert P == 600000 and P * dt == pytest.approx(4 * Hm / (rate * 1e9), rel=1e-12)
    H = np.array([orc.field_Oe(p, n) for n in range(0, P + 1, 100)])
    assert H[0] == Hm and H[-1] == Hm
    assert orc.field_Oe(p, P // 2) == pytest.approx(-Hm, abs=1e-9)
    for q in (P // 4, 3 * P // 4):
        assert orc.field_Oe(p, q) == pytest.approx(0.0, abs=1e-9)
    assert orc.field_Oe(p, P // 8) == pytest.approx(Hm / math.sqrt(2.0), rel=1e-12)
    assert np.sum(np.abs(np.diff(H))) == pytest.approx(4 * Hm, rel=1e-12)
    f = 1.0 / (P * dt)
    peak = max(abs(orc.field_Oe(p, n + 1) - orc.field_Oe(p, n)) for n in (P // 4, 3 * P // 4))
    assert peak / dt == pytest.approx(2 * math.pi * f * Hm, rel=1e-6)
    assert orc.field_Oe(p, 5 * P + 12345) == orc.field_Oe(p, 12345)
    for n in (1, 777, 123456):
        assert orc.field_Oe(p, P - n) == pytest.approx(orc.field_Oe(p, n), abs=1e-9)
        assert orc.field_Oe(p, n + P // 2) == pytest.approx(-orc.field_Oe(p, n), abs=1e-9)


def test_block_volume_is_a_cube_of_the_same_volume(orc):
    """The thermal field depends on the cell only through its volume: a single block of volume
    10752 a0^3 (the b = 22 prism) has the coefficients of a cube of edge (10752)^(1/3) a0."""
    a0, V = 0.8396e-9, 10752 * 0.8396e-9 ** 3
    kw = dict(A=0.0, K=1e4, Ms=480e3, alpha=0.1, T=310.0, dt=20e-15)
    blk = orc.Problem(1, 1, 1, a=22 * a0, volume=V, **kw)
    cube = orc.Problem(1, 1, 1, a=V ** (1.0 / 3.0), **kw)
    assert orc.coefficients(blk)["sigma"] == pytest.approx(orc.coefficients(cube)["sigma"], rel=1e-14)
    assert orc.coefficients(blk)["c_an"] == orc.coefficients(cube)["c_an"]
