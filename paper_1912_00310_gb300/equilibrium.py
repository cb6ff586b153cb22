"""Equilibrium magnetisation against temperature: the temperature dependence behind Eq. 12 and
Fig. 3 of arXiv:1912.00310.

The coarse-graining map gives a level-b simulation at temperature T0 the reduced temperature
T* = k_B T Lambda / A of the unscaled rod at T(b) = T0 / (b zeta(b, T0)) (Eq. 12).  The paper's
correction of the magnetisation, M0 = (delta zeta + 1 - delta) M(b) (Eq. 13, delta = 0.511), is
fitted to the unscaled rod's M(T) at those temperatures (Fig. 3).  This runner measures, on the
GPU through the library's C ABI, the time-averaged magnetisation of

  * the unscaled rod (b = 1, 8 x 24 x 56 cells of a0) at T0 = 310 K and at T(b) for each level b;
  * the coarse-grained rod at each level b (A(b), K(b) of Eqs. 8-9) at T0;

in zero field from the saturated state, and prints each level's values beside the two
statements: m_b(T0) against m_1(T(b)) (Eq. 12 read for the magnetisation) and m_1(T0) against
(delta zeta + 1 - delta) m_b(T0) (Eq. 13), with the delta that would make Eq. 13 exact at that
level; and the delta of the M(T) fit (Fig. 3), where Eqs. 12 and 13 together give the unscaled
rod's magnetisation at T(b) as m_1(T0) / (delta zeta + 1 - delta).  The magnetisation is |<m_z>| of the cell average at each sample (the rod's moment stays
along its easy axis; its sign may flip at the coarser levels, whose anisotropy barrier is a few
k_B T), averaged over the samples after the burn-in and then over realisations (standard error
over realisations).

    python -m paper_1912_00310_gb300.equilibrium --b 2 4 8 --n-real 152 --steps 200000
"""
import argparse
import json
import math
import time

import numpy as np

from . import ENGINE_AUTO, Grid

MAGNETITE = dict(a0=0.839e-9, A0=0.98e-11, Ms=480e3, K0=10e3, alpha=0.1, T=310.0, Tc=858.0, delta=0.511)
ROD_CELLS = (8, 24, 56)
DT_BY_B = {1: 2e-15, 2: 5e-15, 4: 10e-15, 8: 20e-15}


def make_grid(b: int, T: float, *, H_Oe=0.0, sample_every=100, device=None, stream=None, engine=ENGINE_AUTO,
              dt=None):
    """The rod at level b (A(b), K(b) of Eqs. 8-9 for b > 1) at temperature T in a held field."""
    M = MAGNETITE
    if any(n % b for n in ROD_CELLS):
        raise ValueError(f"b = {b} does not divide the 8 x 24 x 56 rod")
    g = Grid(*(n // b for n in ROD_CELLS), a0=M["a0"], b=b, device=device, stream=stream)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=T)
    g.set_scaling(mode=1 if b > 1 else 0, Tc=M["Tc"])
    g.set_sweep(H_start=H_Oe, H_turn=H_Oe, rate=0.0, dt=dt or DT_BY_B[b], sample_dH=float(sample_every))
    g.set_engine(engine)
    return g


def level_temperature(b: int, T0: float = MAGNETITE["T"]) -> float:
    """T(b) = T0 / (b zeta(b, T0)) (Eq. 12), zeta from the library's coarse-graining map."""
    g = make_grid(b, T0)
    try:
        return T0 / (b * g.coefficients()["zeta"])
    finally:
        g.close()


def measure(b: int, T: float, n_real: int, steps: int, *, burn_in=None, sample_every=100, seed=0, **kw) -> dict:
    """Time-averaged |m_z| of the cell-averaged magnetisation of n_real realisations after the
    burn-in (default: the first quarter of the run)."""
    import torch
    burn_in = steps // 4 if burn_in is None else burn_in
    g = make_grid(b, T, sample_every=sample_every, **kw)
    try:
        n_cols = steps // sample_every + 1
        g.set_held_samples(n_cols)
        g.reset(seed=seed, n_real=n_real)
        S = torch.zeros((n_real, n_cols), device=f"cuda:{g.device}")
        t0 = time.perf_counter()
        g.advance(steps, S)
        g.sync(0)
        sec = time.perf_counter() - t0
        k0 = (burn_in + sample_every - 1) // sample_every
        per_real = S[:, max(1, k0):].abs().double().mean(1).cpu().numpy()
        return dict(b=b, T=T, n_real=n_real, steps=steps, burn_in=burn_in, sample_every=sample_every,
                    m=float(per_real.mean()), m_se=float(per_real.std(ddof=1) / math.sqrt(n_real)),
                    zeta=g.coefficients()["zeta"], seconds=sec,
                    cell_steps_per_s=g.ncells * n_real * steps / sec)
    finally:
        g.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--b", type=int, nargs="+", default=[2, 4, 8])
    ap.add_argument("--n-real", type=int, default=152)
    ap.add_argument("--steps", type=int, default=200000, help="Heun steps of the b = 1 runs")
    ap.add_argument("--seed", type=int, default=0)
    a = ap.parse_args(argv)
    M = MAGNETITE
    T0, delta = M["T"], M["delta"]
    ref = measure(1, T0, a.n_real, a.steps, seed=a.seed)
    print(json.dumps(dict(ref, role="unscaled rod at T0")), flush=True)
    for b in a.b:
        Tb = level_temperature(b, T0)
        # the same simulated time at each level: steps scale with 1 / dt
        steps_b = max(1000, int(round(a.steps * DT_BY_B[1] / DT_BY_B[b])) // 100 * 100)
        lev = measure(b, T0, a.n_real, steps_b, seed=a.seed)
        cold = measure(1, Tb, a.n_real, a.steps, seed=a.seed)
        z = lev["zeta"]
        f13 = delta * z + 1.0 - delta
        out = dict(b=b, T_b=Tb, zeta=z, m_level_T0=lev["m"], m_level_T0_se=lev["m_se"], m_rod_Tb=cold["m"],
                   m_rod_Tb_se=cold["m_se"], m_rod_T0=ref["m"], m_rod_T0_se=ref["m_se"],
                   eq12_ratio=lev["m"] / cold["m"], eq13_m0=f13 * lev["m"], eq13_ratio=f13 * lev["m"] / ref["m"],
                   delta_exact=(ref["m"] / lev["m"] - 1.0) / (z - 1.0) if z != 1.0 else None,
                   delta_mt=(ref["m"] / cold["m"] - 1.0) / (z - 1.0) if z != 1.0 else None,
                   seconds=lev["seconds"] + cold["seconds"])
        print(json.dumps(out), flush=True)


if __name__ == "__main__":
    main()
