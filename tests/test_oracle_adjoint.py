"""Pin of the oracle's loss gradient (forward-mode differentiation of the discrete Heun map)
against central finite differences of the oracle's own forward run with common random numbers
(the same thermal normals at every parameter value)."""
import numpy as np
import pytest

from workloads import MAGNETITE as M, random_unit_state


def _setup(orc, dims=(1, 2, 3), n_real=16, disp=0.0, shape=0):
    p = orc.material_problem(*dims, a0=M["a0"], b=4, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=10e-15, mode=1, Tc=M["Tc"],
                             H_start_Oe=1500.0, H_turn_Oe=-1500.0, rate_Oe_per_ns=1000.0,
                             disp=disp, shape=shape)
    m0 = np.ascontiguousarray(random_unit_state(n_real, p.ncells, seed=21, cone=0.6))
    n_samples = 2 * p.n_half // 100 + 1
    target = 0.92 + 0.05 * np.cos(np.arange(n_samples) / 7.0)
    return p, m0, target


def _loss(orc, p, m0, target, scale, step0, n_steps, every):
    q = orc.scaled_problem(p, scale)
    m = m0.copy()
    k_first, k_last = step0 // every + 1, (step0 + n_steps) // every
    s, _ = orc.run(q, m, seed=3, step0=step0, n_steps=n_steps, sample_every=every,
                   n_samples=k_last + 1)
    mbar = s[:, k_first:k_last + 1].mean(axis=0)
    return float(np.mean((mbar - target[k_first:k_last + 1]) ** 2)), mbar


@pytest.mark.parametrize("scale,disp,shape", [((1.0, 1.0, 1.0), 0.0, 0), ((1.3, 0.7, 1.15), 0.0, 0),
                                              ((1.1, 0.9, 1.05), 0.0872664626, 0),
                                              ((0.9, 1.2, 0.95), 0.0872664626, 1)])
def test_gradient_matches_central_differences(orc, scale, disp, shape):
    p, m0, target = _setup(orc, disp=disp, shape=shape)
    step0, n_steps, every = 300, 2000, 100
    L, g, mbar = orc.loss_grad(p, m0, target=target, scale=scale, seed=3, step0=step0,
                               n_steps=n_steps, sample_every=every)
    L0, mbar0 = _loss(orc, p, m0, target, scale, step0, n_steps, every)
    assert L == pytest.approx(L0, rel=1e-12)
    assert np.allclose(mbar, mbar0, rtol=0, atol=1e-13)
    for k in range(3):
        h = 1e-5 * scale[k]
        up, dn = list(scale), list(scale)
        up[k] += h
        dn[k] -= h
        fd = (_loss(orc, p, m0, target, up, step0, n_steps, every)[0]
              - _loss(orc, p, m0, target, dn, step0, n_steps, every)[0]) / (2 * h)
        assert g[k] == pytest.approx(fd, rel=1e-5, abs=1e-12 * abs(L)), (k, g[k], fd)
    assert np.all(np.abs(g) > 0)


def test_gradient_of_zero_temperature_macrospin_is_analytic(orc):
    """One macrospin at T = 0 with the field along z and no anisotropy: m_z(t) follows the
    damped-precession closed form, so d<m_z>/d s_alpha can be differentiated by hand:
    tan(theta/2) = tan(theta0/2) exp(-alpha g1 H t) with alpha g1 = g0 alpha / (1 + alpha^2)."""
    import math
    H_Oe, th0, dt, n = 2000.0, 1.2, 2e-15, 4000
    p = orc.Problem(1, 1, 1, a=2e-9, A=0.0, K=0.0, Ms=480e3, alpha=0.3, T=0.0, dt=dt,
                    H_start_Oe=H_Oe, H_turn_Oe=H_Oe)
    m0 = np.array([[[math.sin(th0), 0.0, math.cos(th0)]]])
    target = np.zeros(n + 1)
    L, g, mbar = orc.loss_grad(p, m0, target=target, step0=0, n_steps=n, sample_every=n)
    t = n * dt
    g0 = orc.MU0 * orc.GAMMA_E
    H = H_Oe * orc.OE

    def mz(alpha):
        rate = g0 * alpha / (1 + alpha * alpha) * H
        return math.cos(2 * math.atan(math.tan(th0 / 2) * math.exp(-rate * t)))

    a = 0.3
    eps = 1e-6
    dmz_dalpha = (mz(a + eps) - mz(a - eps)) / (2 * eps)
    # L = mz^2 (target 0, one sample); dL/ds_alpha = 2 mz dmz/dalpha * alpha
    assert mbar[0] == pytest.approx(mz(a), abs=1e-6)
    assert g[1] == pytest.approx(2 * mz(a) * dmz_dalpha * a, rel=1e-4)
    assert g[0] == 0.0  # no anisotropy term to scale
    assert abs(g[2]) < 1e-12  # Ms enters only exchange, anisotropy and the thermal field
