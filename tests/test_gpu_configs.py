"""GPU parity at the sizes of the workloads themselves, through the C ABI, against the FP64 oracle
on the same seeds (Eq. 1 with the Brown thermal field; the loop observables of the realisation
paragraph, "one standard error" by delete-one jackknife over realisations).

  * the full-resolution b = 1 rod, 64 realisations: every realisation's state within 1e-4 after
    1000 steps, then the realisation-mean m_z at each sample of a 20,000-step window within three
    combined standard errors;
  * the uneven batch through llg_run_batch, reduced to loops that close within 2e5 steps (b = 4
    and 8, alpha = 0.5 and 1, 64 realisations each): every job's coercive field and loop area
    within three combined standard errors of the oracle's;
  * the 512 x 512 x 56 periodic slab in the streaming engine's launch configuration: every cell
    within 1e-4 of the oracle after 10 steps.

The oracle runs one thread per realisation on the host cores, so these tests take minutes.
"""
import math

import numpy as np
import pytest

from workloads import CONFIGS, DT_BY_B, MAGNETITE as M, ROD_DIMS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    assert torch.cuda.is_available()
    return P


def grid(pkg, dims, b, dt, *, alpha=None, H_start=1500.0, H_turn=-1500.0, rate=1000.0, sample_dH=1.0,
         periodic=0, engine=None):
    g = pkg.Grid(*dims, a0=M["a0"], b=b, periodic=periodic)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"] if alpha is None else alpha,
                   T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=H_start, H_turn=H_turn, rate=rate, dt=dt, sample_dH=sample_dH)
    if engine is not None:
        g.set_engine(engine)
    return g


def problem(orc, dims, b, dt, *, alpha=None, H_start=1500.0, H_turn=-1500.0, rate=1000.0, periodic=0):
    return orc.material_problem(*dims, a0=M["a0"], b=b, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                                alpha=M["alpha"] if alpha is None else alpha, T=M["T"], dt=dt, mode=1,
                                Tc=M["Tc"], H_start_Oe=H_start, H_turn_Oe=H_turn,
                                rate_Oe_per_ns=rate, periodic=periodic)


def state(g, n_real):
    out = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    g.get_state(out)
    g.sync(600)
    return out


def test_b1_rod_64_realisations_window(pkg, orc):
    """The full-resolution rod (8 x 24 x 56 cells, dt = 2 fs, 100 Oe/ns), 64 realisations: all of
    them within 1e-4 of the oracle after 1000 steps; then the mean m_z at the samples of a
    20,000-step window (every 5000 steps) within three combined standard errors."""
    cfg = CONFIGS["rod_b1_256real"]
    dims, dt, n_real, seed = cfg["dims"], cfg["dt"], 64, cfg["seed"]
    g = grid(pkg, dims, 1, dt, rate=cfg["rate"], engine=pkg.ENGINE_RESIDENT)
    g.reset(seed=seed, n_real=n_real)
    g.advance(1000)
    gpu = state(g, n_real).double().cpu().numpy()
    p = problem(orc, dims, 1, dt, rate=cfg["rate"])
    ref = orc.uniform_state(n_real, g.ncells)
    orc.run(p, ref, seed=seed, n_steps=1000)
    err = np.abs(gpu - ref).max(axis=(1, 2))
    assert err.max() <= 1e-4, (int(err.argmax()), float(err.max()))
    window, every = 20000, g.sample_every
    assert every == 5000
    S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
    g.advance(window - 1000, S)
    g.sync(600)
    k = window // every
    gs = S[:, 1:k + 1].double().cpu().numpy()
    rs, _ = orc.run(p, ref, seed=seed, step0=1000, n_steps=window - 1000, sample_every=every,
                    n_samples=k + 1)
    rs = rs[:, 1:k + 1]
    assert np.isfinite(gs).all() and np.isfinite(rs).all()
    se = np.hypot(gs.std(0, ddof=1), rs.std(0, ddof=1)) / math.sqrt(n_real)
    diff = np.abs(gs.mean(0) - rs.mean(0))
    assert np.all(diff <= 3 * se), (diff, se)
    g.close()


# The uneven batch reduced to loops that close within 2e5 Heun steps: (b, H_max Oe, rate Oe/ns,
# sample spacing Oe) at the workload's time step per b, each at alpha 0.5 and 1 (the dynamic
# coercive field of these small rods at such rates is 700-1350 Oe, so the sweeps reach past it).
LADDER = [(4, 1500.0, 3000.0, 3.0), (8, 1000.0, 1000.0, 2.0)]
ALPHAS = (0.5, 1.0)


def test_reduced_ladder_batch_statistics(pkg, orc):
    n_real, seed = 64, 0
    jobs, specs = [], []
    for b, Hm, rate, dH in LADDER:
        for alpha in ALPHAS:
            g = grid(pkg, ROD_DIMS[b], b, DT_BY_B[b], alpha=alpha, H_start=Hm, H_turn=-Hm, rate=rate,
                     sample_dH=dH, engine=pkg.ENGINE_RESIDENT)
            g.reset(seed=seed, n_real=n_real, real_offset=len(jobs) * n_real)
            assert g.steps_per_loop <= 200000
            jobs.append(g)
            specs.append((b, Hm, rate, dH, alpha))
    samples = [torch.zeros((n_real, g.n_samples), device="cuda") for g in jobs]
    for S in samples:
        S[:, 0] = 1.0
    calls = 0
    while any(pkg.run_batch(jobs, 60000, samples)):
        calls += 1
    assert calls >= 3  # the loops span several graph calls
    for j, (g, S, (b, Hm, rate, dH, alpha)) in enumerate(zip(jobs, samples, specs)):
        assert g.step == g.steps_per_loop
        gs = S.cpu().numpy()
        assert np.isfinite(gs).all()
        p = problem(orc, ROD_DIMS[b], b, DT_BY_B[b], alpha=alpha, H_start=Hm, H_turn=-Hm, rate=rate)
        ref = orc.uniform_state(n_real, g.ncells)
        rs, _ = orc.run(p, ref, seed=seed, real0=j * n_real, n_steps=g.steps_per_loop,
                        sample_every=g.sample_every, n_samples=g.n_samples)
        rs[:, 0] = 1.0
        H = g.sample_fields()
        k_turn = (g.n_samples - 1) // 2
        o = orc.loop_stats(H, rs, k_turn)
        mine = orc.loop_stats(H, gs.astype(np.float64), k_turn)
        lib = pkg.loop_stats(gs, H, k_turn, mode=1, zeta=g.coefficients()["zeta"])
        assert lib["Hc_Oe"] == pytest.approx(mine["Hc"], rel=1e-9)
        for key in ("Hc", "area"):
            assert math.isfinite(o[key]) and math.isfinite(mine[key]), (specs[j], key)
            se = math.hypot(o[key + "_se"], mine[key + "_se"])
            assert abs(o[key] - mine[key]) <= 3 * se, (specs[j], key, o[key], mine[key], se)
    for g in jobs:
        g.close()


def test_full_slab_against_oracle(pkg, orc):
    """The 512 x 512 x 56 periodic slab (14.7M cells) in the streaming engine, advanced in the
    benchmark's way (one call of several steps): every cell within 1e-4 of the oracle after 10
    steps."""
    cfg = CONFIGS["slab_512x512x56"]
    dims, periodic, steps = cfg["dims"], cfg["periodic"], 10
    g = grid(pkg, dims, 1, cfg["dt"], rate=cfg["rate"], periodic=periodic, engine=pkg.ENGINE_STREAM)
    assert g.engine == pkg.ENGINE_STREAM
    g.reset(seed=cfg["seed"], n_real=1)
    g.advance(steps)
    got = state(g, 1)[0].double().cpu().numpy()
    g.close()
    p = problem(orc, dims, 1, cfg["dt"], rate=cfg["rate"], periodic=periodic)
    ref = orc.uniform_state(1, p.ncells)
    orc.run(p, ref, seed=cfg["seed"], n_steps=steps)
    err = np.abs(got - ref[0])
    assert err.max() <= 1e-4, float(err.max())
    assert np.abs(ref[0, :, 2] - 1.0).max() > 1e-3  # the noise acted
