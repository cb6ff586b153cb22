"""Pins of the easy-axis dispersion (the material paragraph's 5 degree spread of the anisotropy
axis): the axes are uniform over the solid angle of the cone, one per (seed, realisation, cell),
and the anisotropy field of each cell uses its own axis (a cell relaxes onto it)."""
import math

import numpy as np
import pytest
from scipy import stats

from workloads import MAGNETITE as M

DISP = math.radians(5.0)


def _problem(orc, dims, disp=DISP, **kw):
    base = dict(a=1e-9, A=0.0, K=1e4, Ms=480e3, alpha=0.1, T=0.0, dt=10e-15)
    base.update(kw)
    return orc.Problem(*dims, disp=disp, **base)


def test_axes_are_uniform_on_the_cap(orc):
    p = _problem(orc, (20, 25, 40))  # 20000 cells
    u = orc.easy_axes(p, seed=7, n_real=1)[0]
    assert np.max(np.abs(np.linalg.norm(u, axis=1) - 1.0)) < 1e-14
    cos_t = u[:, 2]
    assert cos_t.min() >= math.cos(DISP) - 1e-15
    # 1 - cos(theta) uniform on [0, 1 - cos(disp)]: the cap's area element
    w = (1.0 - cos_t) / (1.0 - math.cos(DISP))
    assert stats.kstest(w, "uniform").pvalue > 1e-3
    phi = np.arctan2(u[:, 1], u[:, 0]) % (2 * math.pi)
    assert stats.kstest(phi / (2 * math.pi), "uniform").pvalue > 1e-3
    # mean axis of a uniform cap: (0, 0, (1 + cos disp) / 2)
    se = np.std(u, axis=0) / math.sqrt(len(u))
    assert abs(u[:, 0].mean()) < 4 * se[0] and abs(u[:, 1].mean()) < 4 * se[1]
    assert u[:, 2].mean() == pytest.approx((1 + math.cos(DISP)) / 2, abs=4 * se[2])


def test_axes_are_keyed_by_seed_realisation_and_cell(orc):
    p = _problem(orc, (2, 3, 4))
    a = orc.easy_axes(p, seed=1, n_real=3)
    assert np.array_equal(a, orc.easy_axes(p, seed=1, n_real=3))
    assert np.array_equal(a[1:], orc.easy_axes(p, seed=1, n_real=2, real0=1))
    assert not np.allclose(a[0], a[1])
    assert not np.allclose(a, orc.easy_axes(p, seed=2, n_real=3))
    assert len({tuple(v) for v in a.reshape(-1, 3)}) == a.shape[0] * a.shape[1]
    # no dispersion: every cell has the material axis
    q = _problem(orc, (2, 3, 4), disp=0.0, u=(0.6, 0.0, 0.8))
    assert np.array_equal(orc.easy_axes(q, seed=1, n_real=2),
                          np.broadcast_to([0.6, 0.0, 0.8], (2, 24, 3)))


def test_each_cell_relaxes_onto_its_own_axis(orc):
    """T = 0, no exchange and no applied field, strong damping: starting from +z, every cell
    settles on the minimum of -K (m.u_i)^2 nearest to it, i.e. its own axis +u_i."""
    p = _problem(orc, (1, 2, 3), disp=0.4, alpha=1.0, K=2e5)
    u = orc.easy_axes(p, seed=5, n_real=2)
    m = orc.uniform_state(2, 6)
    orc.run(p, m, seed=5, n_steps=40000)
    assert np.max(np.abs(m - u)) < 1e-6
    assert np.min(np.einsum("rci,rci->rc", u, np.array([[[0, 0, 1.0]]]))) < math.cos(0.1)


def test_tiny_dispersion_is_a_perturbation_of_the_z_axis(orc):
    kw = dict(A=1e-11, T=310.0, alpha=0.5)
    p0 = _problem(orc, (2, 3, 4), disp=0.0, **kw)
    p1 = _problem(orc, (2, 3, 4), disp=1e-7, **kw)
    m0, m1 = orc.uniform_state(2, 24), orc.uniform_state(2, 24)
    orc.run(p0, m0, seed=2, n_steps=300)
    orc.run(p1, m1, seed=2, n_steps=300)
    d = np.max(np.abs(m0 - m1))
    assert 0 < d < 1e-8
