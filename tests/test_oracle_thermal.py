"""Pins of the thermal field (Brown's fluctuating field, the paragraph after Eq. 1): with the
variance sigma^2 = 2 alpha kB T / (g0 mu0 Ms V dt) the stochastic Heun scheme must sample the
Boltzmann distribution exp(-E/kB T).  Time averages over 64 realisations are compared with
closed forms or quadrature: within 0.5%, with a standard error below 0.15% (a factor of two in
sigma^2, e.g. an extra 1 + alpha^2 at alpha = 1, moves every value below by more than 10%)."""
import math

import numpy as np
import pytest
from scipy import integrate, special

T, MS, A_CELL = 310.0, 480e3, 3e-9
V = A_CELL ** 3
N_REAL, N_STEPS, BURN = 64, 2_000_000, 20_000


def _timeavg(orc, p, seed, n_steps=N_STEPS):
    m = orc.uniform_state(N_REAL, p.ncells)
    _, tav = orc.run(p, m, n_steps=n_steps, timeavg_burn_in=BURN, seed=seed)
    return tav.mean(), tav.std(ddof=1) / math.sqrt(N_REAL)


def _dt_for(orc, H_max):
    return 0.008 / (orc.MU0 * orc.GAMMA_E * H_max)


def test_langevin_equilibrium(orc):
    """K = 0: <m_z> = L(xi) = coth(xi) - 1/xi, xi = mu0 Ms V H / kB T."""
    xi = 3.0
    kT = orc.KB * T
    H = xi * kT / (orc.MU0 * MS * V)
    p = orc.Problem(1, 1, 1, a=A_CELL, A=0.0, K=0.0, Ms=MS, alpha=1.0, T=T, dt=_dt_for(orc, H),
                    H_start_Oe=H / orc.OE, H_turn_Oe=H / orc.OE)
    mean, se = _timeavg(orc, p, seed=11)
    exact = 1 / math.tanh(xi) - 1 / xi
    assert se / exact < 1.5e-3
    assert abs(mean - exact) / exact < 5e-3


def test_uniaxial_equilibrium_by_quadrature(orc):
    """K > 0 along z: <cos theta> under E = -K V cos^2 theta - mu0 Ms V H cos theta."""
    kT = orc.KB * T
    beta_kv, xi = 1.0, 2.5
    K = beta_kv * kT / V
    H = xi * kT / (orc.MU0 * MS * V)
    c_an = 2 * K / (orc.MU0 * MS)
    p = orc.Problem(1, 1, 1, a=A_CELL, A=0.0, K=K, Ms=MS, alpha=1.0, T=T,
                    dt=_dt_for(orc, H + c_an), H_start_Oe=H / orc.OE, H_turn_Oe=H / orc.OE)
    mean, se = _timeavg(orc, p, seed=12, n_steps=4_000_000)
    w = lambda c: math.exp(beta_kv * c * c + xi * c)
    num = integrate.quad(lambda c: c * w(c), -1, 1, epsabs=1e-13)[0]
    den = integrate.quad(w, -1, 1, epsabs=1e-13)[0]
    exact = num / den
    assert se / exact < 1.5e-3
    assert abs(mean - exact) / exact < 5e-3


def test_two_cell_exchange_equilibrium_by_quadrature(orc):
    """Two exchange-coupled cells (bond energy 2 A a (1 - m1.m2)) in a field along z: <m_z> from
    the two-sphere Boltzmann integral, the azimuth done in closed form (2 pi I0).  Pins the
    exchange energy scale and that each cell draws its own noise."""
    kT = orc.KB * T
    beta_j, xi = 1.0, 2.0
    A = beta_j * kT / (2 * A_CELL)
    H = xi * kT / (orc.MU0 * MS * V)
    c_ex = 2 * A / (orc.MU0 * MS * A_CELL ** 2)
    p = orc.Problem(2, 1, 1, a=A_CELL, A=A, K=0.0, Ms=MS, alpha=1.0, T=T,
                    dt=_dt_for(orc, H + c_ex), H_start_Oe=H / orc.OE, H_turn_Oe=H / orc.OE)
    mean, se = _timeavg(orc, p, seed=13, n_steps=3_000_000)
    x, wts = np.polynomial.legendre.leggauss(200)  # cos(theta) nodes on [-1, 1]
    c1, c2 = np.meshgrid(x, x, indexing="ij")
    s1, s2 = np.sqrt(1 - c1 ** 2), np.sqrt(1 - c2 ** 2)
    # exp(beta_j (c1 c2 + s1 s2 cos dphi) + xi (c1 + c2)), dphi integrated: 2 pi I0(beta_j s1 s2);
    # the scaled Bessel function keeps the exponent finite.
    arg = beta_j * s1 * s2
    wgt = np.outer(wts, wts) * special.i0e(arg) * np.exp(arg + beta_j * c1 * c2 + xi * (c1 + c2))
    exact = float((wgt * 0.5 * (c1 + c2)).sum() / wgt.sum())
    assert se / exact < 1.5e-3
    assert abs(mean - exact) / exact < 5e-3
    # the coupled pair is more aligned with the field than an isolated cell at the same xi
    assert exact > 1 / math.tanh(xi) - 1 / xi


def test_norm_preserved_at_finite_temperature(orc):
    p = orc.Problem(2, 3, 4, a=2e-9, A=1e-11, K=1e4, Ms=MS, alpha=0.1, T=T, dt=5e-15,
                    H_start_Oe=200.0, H_turn_Oe=200.0)
    m = orc.uniform_state(2, 24)
    orc.run(p, m, n_steps=3000, seed=1)
    assert np.max(np.abs(np.linalg.norm(m, axis=-1) - 1.0)) < 1e-14
    assert np.std(m[..., 2]) > 1e-3  # the noise did act
