"""Seeded synthetic inputs shared by the tests, the benchmark and the smoke check.

This module describes workloads only: material constants as the paper states them, grid shapes,
sweeps, realisation counts and seeds, plus seeded random initial states.  It holds none of the
method's arithmetic (no coarse-graining, no field, no integrator); each side derives its own
coefficients from these inputs.

Material (arXiv:1912.00310, material paragraph): magnetite, a0 = 0.839 nm, A0 = 0.98e-11 J/m,
Ms = 480 kA/m, K0 = 10 kJ/m^3 along z, alpha = 0.1, T = 310 K, Tc = 858 K, delta = 0.511 (Eq. 13).
"""
import numpy as np

MAGNETITE = dict(a0=0.839e-9, A0=0.98e-11, Ms=480e3, K0=10e3, alpha=0.1, T=310.0, Tc=858.0,
                 delta=0.511)

# Rod at level b: 8x24x56 cells of a0 at b = 1, (8/b)x(24/b)x(56/b) cells of b*a0 otherwise.
ROD_DIMS = {1: (8, 24, 56), 2: (4, 12, 28), 4: (2, 6, 14), 8: (1, 3, 7)}

# Time step per coarse-graining level (larger cells allow a larger step).
DT_BY_B = {1: 2e-15, 2: 5e-15, 4: 10e-15, 8: 20e-15}

# The five workloads.  Fields in Oe, rates in Oe/ns, dt in s.
CONFIGS = {
    # plain sLLG Heun on the b = 4 rod, 4 realisations (seed = r for r = 0..3 read as seed 0,
    # realisations 0..3), M sampled every 1 Oe over a full +1500 -> -1500 -> +1500 Oe loop
    "rod_b4_4real": dict(b=4, dims=ROD_DIMS[4], dt=10e-15, H_start=1500.0, H_turn=-1500.0,
                         rate=1000.0, sample_dH=1.0, n_real=4, seed=0, mode=1),
    # full-resolution rod, 256 realisations in one persistent launch
    "rod_b1_256real": dict(b=1, dims=ROD_DIMS[1], dt=2e-15, H_start=1500.0, H_turn=-1500.0,
                           rate=100.0, sample_dH=1.0, n_real=256, seed=0, mode=1),
    # uneven batch: b in {1,2,4,8} x rate in {1000,100,10} x alpha in {0.05,0.1,0.5,1.0}, 64 each
    "ladder_batch": dict(bs=(1, 2, 4, 8), rates=(1000.0, 100.0, 10.0),
                         alphas=(0.05, 0.1, 0.5, 1.0), n_real=64, H_start=1500.0, H_turn=-1500.0,
                         sample_dH=1.0, seed=0, mode=1),
    # periodic slab beyond shared memory
    "slab_512x512x56": dict(b=1, dims=(512, 512, 56), dt=2e-15, H_start=1500.0, H_turn=-1500.0,
                            rate=1000.0, n_steps=200_000, periodic=0b011, seed=0, mode=1),
    # adjoint calibration window on the b = 4 rod
    "adjoint_b4": dict(b=4, dims=ROD_DIMS[4], dt=10e-15, H_start=1500.0, H_turn=-1500.0,
                       rate=1000.0, window_steps=20_000, ckpt_every=512, n_real=64, seed=0,
                       mode=1),
}


def random_unit_state(n_real: int, ncells: int, seed: int, cone: float | None = None) -> np.ndarray:
    """Seeded random unit vectors [n_real][ncells][3] (float64).  With cone (radians), directions
    are uniform within that half-angle of +z; otherwise uniform on the sphere."""
    rng = np.random.default_rng(seed)
    if cone is None:
        v = rng.normal(size=(n_real, ncells, 3))
        return v / np.linalg.norm(v, axis=-1, keepdims=True)
    cz = rng.uniform(np.cos(cone), 1.0, size=(n_real, ncells))
    ph = rng.uniform(0, 2 * np.pi, size=(n_real, ncells))
    sz = np.sqrt(1 - cz * cz)
    return np.stack([sz * np.cos(ph), sz * np.sin(ph), cz], axis=-1)


def plus_z_state(n_real: int, ncells: int) -> np.ndarray:
    m = np.zeros((n_real, ncells, 3))
    m[..., 2] = 1.0
    return m
