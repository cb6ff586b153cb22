"""GPU parity of the paper's own protocol: the sinusoidal field H_max sin(2 pi f t) with
SR = 4 H_max f (started at +H_max), the single-block limit (the whole rod as one macrospin of
volume 10752 a0^3 at b = 22, no exchange) and the 5-degree dispersion of the easy axis.

Every engine evaluates the field from the same integer phase, so the engines stay bitwise equal;
against the FP64 oracle the trajectories stay within 1e-4 over the first 1000 steps, past a
wrap of the cycle.
"""
import math

import numpy as np
import pytest

from workloads import MAGNETITE as M, ROD_DIMS, random_unit_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

# A short cycle: 1 Oe per step at 10 fs, H_max = 200 Oe -> 800 steps per cycle, samples every 10.
SINE = dict(H_start=200.0, rate=1e5, dt=10e-15, sample_dH=10.0)
BLOCK_V = 10752 * M["a0"] ** 3


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    assert torch.cuda.is_available()
    return P


def sine_grid(pkg, dims, b, *, engine, kind=0, alpha=None, H_start=None, rate=None, dt=None,
              sample_dH=None, volume=None, periodic=0):
    g = pkg.Grid(*dims, a0=M["a0"], b=b, periodic=periodic)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=alpha or M["alpha"], T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=H_start or SINE["H_start"], H_turn=0.0, rate=rate or SINE["rate"],
                dt=dt or SINE["dt"], sample_dH=sample_dH or SINE["sample_dH"], shape=1)
    if volume:
        g.set_cell_volume(volume)
    g.set_engine(engine)
    if kind:
        g.set_tuning(pkg.TUNE_ROD_KIND, kind)
    return g


def sine_problem(orc, dims, b, *, alpha=None, H_start=None, rate=None, dt=None, volume=None,
                 periodic=0):
    return orc.material_problem(*dims, a0=M["a0"], b=b, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                                alpha=alpha or M["alpha"], T=M["T"], dt=dt or SINE["dt"], mode=1,
                                Tc=M["Tc"], H_start_Oe=H_start or SINE["H_start"],
                                rate_Oe_per_ns=rate or SINE["rate"], shape=1, volume=volume,
                                periodic=periodic)


def state_of(g, n_real):
    out = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    g.get_state(out)
    g.sync(300.0)
    return out


ENGINES = [("plain", 0), ("resident", 1), ("resident", 2), ("stream", 0)]


def _engine(pkg, name):
    return {"plain": pkg.ENGINE_PLAIN, "resident": pkg.ENGINE_RESIDENT,
            "stream": pkg.ENGINE_STREAM}[name]


def test_sinusoid_engines_bitwise_and_oracle(pkg, orc):
    dims, b, n_real = ROD_DIMS[4], 4, 3
    p = sine_problem(orc, dims, b)
    assert p.period == 800
    ref = orc.uniform_state(n_real, p.ncells)
    orc.run(p, ref, seed=0, n_steps=1000)
    states = []
    for name, kind in ENGINES:
        g = sine_grid(pkg, dims, b, engine=_engine(pkg, name), kind=kind)
        assert g.steps_per_loop == 800 and g.n_samples == 81
        g.reset(seed=0, n_real=n_real)
        g.advance(600)
        g.advance(400)  # crosses the end of the cycle at step 800
        s = state_of(g, n_real)
        assert float(np.max(np.abs(s.double().cpu().numpy() - ref))) <= 1e-4, (name, kind)
        states.append(s)
        g.close()
    for s in states[1:]:
        assert torch.equal(s, states[0])


@pytest.mark.parametrize("disp", [0.0, math.radians(5.0)])
def test_sinusoid_b1_rod_specialised_kernel(pkg, orc, disp):
    """The b = 1 rod runs the shape-specialised plane-pipelined kernel (cosine variant, and its
    dispersed-axis instance); 160 rods take the balanced schedule.  Bitwise equal to the generic
    kernel and the plain engine; the last realisation against the oracle."""
    dims, n_real, steps = ROD_DIMS[1], 160, 300
    kw = dict(dt=2e-15, rate=1e5, H_start=40.0, sample_dH=2.0)  # 0.2 Oe/step, a cycle of 800 steps
    outs = []
    for eng, generic in ((pkg.ENGINE_RESIDENT, 0), (pkg.ENGINE_RESIDENT, 1), (pkg.ENGINE_PLAIN, 0)):
        g = sine_grid(pkg, dims, 1, engine=eng, **kw)
        g.set_axis_dispersion(disp)
        if generic:
            g.set_tuning(pkg.TUNE_GENERIC_KERNEL, 1)
        g.reset(seed=2, n_real=n_real)
        g.advance(steps)
        outs.append(state_of(g, n_real))
        g.close()
    assert torch.equal(outs[0], outs[1]) and torch.equal(outs[0], outs[2])
    p = sine_problem(orc, dims, 1, dt=2e-15, rate=1e5, H_start=40.0)
    p.disp = disp
    ref = orc.uniform_state(1, p.ncells)
    orc.run(p, ref, seed=2, real0=n_real - 1, n_steps=steps)
    assert float(np.max(np.abs(outs[0][-1].double().cpu().numpy() - ref[0]))) <= 1e-4


def test_sinusoid_samples_match_oracle(pkg, orc):
    """A whole cycle on the b = 8 rod: every sample of m_z against the oracle."""
    dims, b, n_real = ROD_DIMS[8], 8, 8
    kw = dict(H_start=400.0, rate=1e5, dt=20e-15, sample_dH=40.0)  # 2 Oe/step, 800 steps
    g = sine_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT, **kw)
    S = torch.zeros((n_real, g.n_samples), device="cuda")
    g.run_loops(seed=0, n_real=n_real, samples=S, stats=False)
    g.sync(60)
    p = sine_problem(orc, dims, b, H_start=400.0, rate=1e5, dt=20e-15)
    ref = orc.uniform_state(n_real, g.ncells)
    s_ref, _ = orc.run(p, ref, seed=0, n_steps=g.steps_per_loop, sample_every=g.sample_every,
                       n_samples=g.n_samples)
    s_ref[:, 0] = 1.0
    assert g.n_samples == 41 and g.sample_every == 20
    assert np.max(np.abs(S.double().cpu().numpy() - s_ref)) < 1e-4
    H = g.sample_fields()
    for k in range(g.n_samples):
        assert H[k] == pytest.approx(orc.field_Oe(p, k * g.sample_every), abs=1e-9)
    g.close()


def test_sinusoid_streaming_periodic_slab(pkg, orc):
    """The streaming engine on a periodic slab several tiles wide, under the sinusoid."""
    dims, n_real = (40, 45, 6), 1
    g = sine_grid(pkg, dims, 1, engine=pkg.ENGINE_STREAM, dt=2e-15, rate=5e5, H_start=500.0,
                  sample_dH=50.0, periodic=0b011)
    h = sine_grid(pkg, dims, 1, engine=pkg.ENGINE_PLAIN, dt=2e-15, rate=5e5, H_start=500.0,
                  sample_dH=50.0, periodic=0b011)
    assert g.steps_per_loop == 2000
    for x in (g, h):
        x.reset(seed=3, n_real=n_real)
        x.advance(300)
    a, c = state_of(g, n_real), state_of(h, n_real)
    assert torch.equal(a, c)
    p = sine_problem(orc, dims, 1, H_start=500.0, rate=5e5, dt=2e-15, periodic=0b011)
    ref = orc.uniform_state(n_real, p.ncells)
    orc.run(p, ref, seed=3, n_steps=300)
    assert float(np.max(np.abs(a.double().cpu().numpy() - ref))) <= 1e-4
    g.close()
    h.close()


def test_sinusoid_adjoint_matches_oracle_gradient(pkg, orc):
    dims, n_real, step0, n_steps = (1, 2, 3), 16, 130, 640  # the window holds the field's minimum
    g = sine_grid(pkg, dims, 4, engine=pkg.ENGINE_RESIDENT)
    g.reset(seed=0, n_real=n_real)
    m0 = random_unit_state(n_real, 6, seed=5, cone=0.6).astype(np.float32)
    g.set_state(m0, step0)
    target = 0.5 * np.cos(2 * np.pi * np.arange(g.n_samples) / (g.n_samples - 1))
    L, grad = g.loss_grad(n_steps, target, objective=0, ckpt_every=256)
    p = sine_problem(orc, dims, 4)
    Lo, go, _ = orc.loss_grad(p, m0.astype(np.float64), target=target, scale=(1.0, 1.0, 1.0),
                              seed=0, step0=step0, n_steps=n_steps, sample_every=g.sample_every)
    assert L == pytest.approx(Lo, rel=1e-3)
    for k in range(3):
        assert grad[k] == pytest.approx(go[k], rel=1e-2, abs=1e-3 * np.abs(go).max()), (k, grad, go)
    g.close()


def test_single_block_trajectory_and_loop(pkg, orc):
    """b = 22: one prism of volume 10752 a0^3, 512 realisations.  Trajectories against the oracle
    for 1000 steps, then a full +-400 Oe sinusoid at SR = 250 Oe/ns with alpha = 1 (at lower
    damping or faster sweeps the macrospin does not reverse within the cycle): coercive field and
    area of the GPU ensemble within 3 combined standard errors of the oracle's (same seeds)."""
    dims, b, n_real, dt = (1, 1, 1), 22, 512, 20e-15
    kw = dict(H_start=400.0, rate=250.0, dt=dt, alpha=1.0)
    g = sine_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT, sample_dH=4.0, volume=BLOCK_V, **kw)
    p = sine_problem(orc, dims, b, volume=BLOCK_V, **kw)
    assert g.steps_per_loop == p.period == 320000
    c, oc = g.coefficients(), orc.coefficients(p)
    assert c["sigma"] == pytest.approx(oc["sigma"], rel=1e-12)
    g.reset(seed=11, n_real=n_real)
    g.advance(1000)
    gpu = state_of(g, n_real).double().cpu().numpy()
    ref = orc.uniform_state(n_real, 1)
    orc.run(p, ref, seed=11, n_steps=1000)
    assert float(np.max(np.abs(gpu - ref))) <= 1e-4
    g.close()

    g = sine_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT, sample_dH=4.0, volume=BLOCK_V, **kw)
    S = np.zeros((n_real, g.n_samples), dtype=np.float32)
    st = g.run_loops(seed=11, n_real=n_real, samples=S)
    ref = orc.uniform_state(n_real, 1)
    s_ref, _ = orc.run(p, ref, seed=11, n_steps=g.steps_per_loop, sample_every=g.sample_every,
                       n_samples=g.n_samples)
    s_ref[:, 0] = 1.0
    H = g.sample_fields()
    k_turn = (g.n_samples - 1) // 2
    o = orc.loop_stats(H, s_ref, k_turn)
    mine = orc.loop_stats(H, S.astype(np.float64), k_turn)
    assert st["area_Oe"] == pytest.approx(mine["area"], rel=1e-6)
    for key in ("Hc", "area"):
        se = math.hypot(o[key + "_se"], mine[key + "_se"])
        assert abs(o[key] - mine[key]) <= 3 * se, (key, o[key], mine[key], se)
    assert 117 < mine["Hc"] < 400  # above the Stoner-Wohlfarth field 2K/(mu0 Ms), below H_max
    g.close()


# ---- the 5-degree easy-axis dispersion --------------------------------------------------------
DISP5 = math.radians(5.0)


def disp_grid(pkg, dims, b, *, engine, kind=0, disp=DISP5, periodic=0, dt=None):
    g = sine_grid(pkg, dims, b, engine=engine, kind=kind, periodic=periodic, dt=dt)
    g.set_axis_dispersion(disp)
    return g


def disp_problem(orc, dims, b, disp=DISP5, periodic=0, dt=None):
    p = sine_problem(orc, dims, b, periodic=periodic, dt=dt)
    p.disp = disp
    return p


def test_axes_match_oracle(pkg, orc):
    dims, b = ROD_DIMS[4], 4
    g = disp_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT)
    g.reset(seed=5, n_real=3, real_offset=40)
    u = np.zeros((3, g.ncells, 3), dtype=np.float32)
    g.get_axes(u)
    ref = orc.easy_axes(disp_problem(orc, dims, b), seed=5, n_real=3, real0=40)
    assert np.max(np.abs(u - ref)) < 1e-6
    d = torch.empty((3, g.ncells, 3), device="cuda")
    g.get_axes(d)
    g.sync(60)
    assert np.array_equal(d.cpu().numpy(), u)
    g.set_axis_dispersion(0.0)
    g.get_axes(u)
    assert np.array_equal(u, np.broadcast_to(np.float32([0, 0, 1]), u.shape))
    g.close()


def test_dispersion_engines_bitwise_and_oracle(pkg, orc):
    """A wide (0.3 rad) dispersion so that the axes matter within 1000 steps."""
    dims, b, n_real = ROD_DIMS[4], 4, 3
    p = disp_problem(orc, dims, b, disp=0.3)
    ref = orc.uniform_state(n_real, p.ncells)
    orc.run(p, ref, seed=0, n_steps=1000)
    z = orc.uniform_state(n_real, p.ncells)
    orc.run(sine_problem(orc, dims, b), z, seed=0, n_steps=1000)
    assert np.max(np.abs(ref - z)) > 1e-3  # the dispersion moves the trajectory by far more than 1e-4
    states = []
    for name, kind in ENGINES:
        g = disp_grid(pkg, dims, b, engine=_engine(pkg, name), kind=kind, disp=0.3)
        g.reset(seed=0, n_real=n_real)
        g.advance(1000)
        s = state_of(g, n_real)
        assert float(np.max(np.abs(s.double().cpu().numpy() - ref))) <= 1e-4, (name, kind)
        states.append(s)
        g.close()
    for s in states[1:]:
        assert torch.equal(s, states[0])


def test_dispersion_b1_rod_and_periodic_slab(pkg, orc):
    """The full b = 1 rod (generic plane-pipelined kernel with axes) and a periodic slab through
    the streaming engine, against the oracle and the plain engine."""
    dims, n_real = ROD_DIMS[1], 2
    g = disp_grid(pkg, dims, 1, engine=pkg.ENGINE_RESIDENT, dt=2e-15)
    g.reset(seed=4, n_real=n_real)
    g.advance(300)
    p = disp_problem(orc, dims, 1, dt=2e-15)
    ref = orc.uniform_state(n_real, p.ncells)
    orc.run(p, ref, seed=4, n_steps=300)
    assert float(np.max(np.abs(state_of(g, n_real).double().cpu().numpy() - ref))) <= 1e-4
    g.close()
    dims = (40, 45, 6)
    a = disp_grid(pkg, dims, 1, engine=pkg.ENGINE_STREAM, periodic=0b011, dt=2e-15, disp=0.3)
    c = disp_grid(pkg, dims, 1, engine=pkg.ENGINE_PLAIN, periodic=0b011, dt=2e-15, disp=0.3)
    for x in (a, c):
        x.reset(seed=6, n_real=1)
        x.advance(200)
    assert torch.equal(state_of(a, 1), state_of(c, 1))
    a.close()
    c.close()


def test_dispersion_batch_equals_job_alone(pkg):
    dims, b = ROD_DIMS[4], 4
    jobs = [disp_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT, disp=d) for d in (0.3, 0.0)]
    for i, j in enumerate(jobs):
        j.reset(seed=8 + i, n_real=5)
    pkg.run_batch(jobs, 500)
    for i, d in enumerate((0.3, 0.0)):
        alone = disp_grid(pkg, dims, b, engine=pkg.ENGINE_RESIDENT, disp=d)
        alone.reset(seed=8 + i, n_real=5)
        alone.advance(500)
        assert torch.equal(state_of(jobs[i], 5), state_of(alone, 5)), d
        alone.close()
    for j in jobs:
        j.close()


def test_dispersion_adjoint_matches_oracle_gradient(pkg, orc):
    dims, n_real, step0, n_steps = (1, 2, 3), 16, 130, 640
    g = disp_grid(pkg, dims, 4, engine=pkg.ENGINE_RESIDENT, disp=0.3)
    g.reset(seed=0, n_real=n_real)
    m0 = random_unit_state(n_real, 6, seed=5, cone=0.6).astype(np.float32)
    g.set_state(m0, step0)
    target = 0.5 * np.cos(2 * np.pi * np.arange(g.n_samples) / (g.n_samples - 1))
    L, grad = g.loss_grad(n_steps, target, objective=0, ckpt_every=256)
    p = disp_problem(orc, dims, 4, disp=0.3)
    Lo, go, _ = orc.loss_grad(p, m0.astype(np.float64), target=target, scale=(1.0, 1.0, 1.0),
                              seed=0, step0=step0, n_steps=n_steps, sample_every=g.sample_every)
    assert L == pytest.approx(Lo, rel=1e-3)
    for k in range(3):
        assert grad[k] == pytest.approx(go[k], rel=1e-2, abs=1e-3 * np.abs(go).max()), (k, grad, go)
    g.close()


def test_protocol_runner_matches_oracle_statistics(pkg, orc):
    """The paper-protocol runner end to end at b = 8 (sinusoid, 5-degree dispersion, delta
    rescaling, autotuned launch) on a fast cycle: +-500 Oe at 250 Oe/ns with alpha = 1, 64
    realisations.  Its rescaled area and coercive field against the oracle's loops of the same
    realisations, within 3 combined standard errors."""
    from paper_1912_00310_gb300 import protocol as P
    n_real, kw = 64, dict(H_max=500.0, rate=250.0, alpha=1.0, sample_dH=5.0)
    r = P.run(8, n_real, seed=4, **kw)
    assert r["steps"] == 400000 and r["b"] == 8
    dims, _ = P.level_grid(8)
    p = orc.material_problem(*dims, a0=M["a0"], b=8, A0=M["A0"], K0=M["K0"], Ms=M["Ms"], alpha=1.0,
                             T=M["T"], dt=P.DT_BY_B[8], mode=2, Tc=M["Tc"], H_start_Oe=500.0,
                             rate_Oe_per_ns=250.0, shape=1, disp=math.radians(5.0))
    every = orc.sample_interval(5.0, 250.0, P.DT_BY_B[8])
    ns = p.period // every + 1
    ref = orc.uniform_state(n_real, p.ncells)
    s, _ = orc.run(p, ref, seed=4, n_steps=p.period, sample_every=every, n_samples=ns)
    s[:, 0] = 1.0
    H = np.array([orc.field_Oe(p, k * every) for k in range(ns)])
    o = orc.loop_stats(H, s, (ns - 1) // 2)
    f = orc.m_rescale(2, r["zeta"], M["delta"]) / r["zeta"]
    se = math.hypot(o["area_se"], r["area_se_Oe"])
    assert abs(o["area"] - r["area_Oe"]) <= 3 * se, (o["area"], r["area_Oe"], se)
    assert r["area0_Oe"] == pytest.approx(r["area_Oe"] * f, rel=1e-9)
    se = math.hypot(o["Hc_se"], r["Hc_se_Oe"])
    assert abs(o["Hc"] - r["Hc_Oe"]) <= 3 * se, (o["Hc"], r["Hc_Oe"], se)
    assert r["slp_W_per_g_at_alpha_0p1"] > 0


@pytest.mark.parametrize("dims,rods,disp,kind,cpt", [((10, 10, 10), 1, 0.3, 1, 0), ((12, 12, 12), 1, 0.3, 1, 0),
                                                     ((12, 12, 12), 1, 0.0, 1, 0), (ROD_DIMS[4], 3, 0.3, 1, 0),
                                                     (ROD_DIMS[4], 2, 0.3, 1, 2), (ROD_DIMS[4], 1, 0.0, 1, 4),
                                                     (ROD_DIMS[4], 3, 0.3, 3, 0), (ROD_DIMS[2], 1, 0.3, 3, 0),
                                                     (ROD_DIMS[8], 5, 0.3, 3, 0)])
def test_twophase_variants_bitwise_with_plain(pkg, dims, rods, disp, kind, cpt):
    """The two-phase kernel with two and four cells per thread (1000- and 1728-cell grids, and the
    b = 4 rod's compile-time instances), with several rods per CTA, and the row kernel of the
    b = 2, 4, 8 rods, under the sinusoid, with and without dispersed axes: bitwise equal to the
    plain engine."""
    n_real, outs = 5, []
    for eng, kd in ((pkg.ENGINE_RESIDENT, kind), (pkg.ENGINE_PLAIN, 0)):
        g = sine_grid(pkg, dims, 4, engine=eng, kind=kd)
        if rods > 1 and kd:
            g.set_tuning(pkg.TUNE_RODS_PER_CTA, rods)
        if cpt and kd:
            g.set_tuning(pkg.TUNE_CELLS_PER_THREAD, cpt)
        g.set_axis_dispersion(disp)
        g.reset(seed=12, n_real=n_real)
        g.advance(60)
        outs.append(state_of(g, n_real))
        g.close()
    assert torch.equal(outs[0], outs[1])
    assert float((torch.linalg.norm(outs[0], dim=-1) - 1).abs().max()) < 1e-6


def test_held_field_samples_and_time_average(pkg, orc):
    """A held (zero) field with sample columns (the equilibrium runs behind Eq. 12): the b = 8 rod
    at 310 K, 64 realisations, 20k steps sampled every 100: the early samples equal the oracle's
    within 1e-4 (trajectory parity), and the time average of |m_z| after the burn-in lies within
    three combined standard errors of the oracle's."""
    from paper_1912_00310_gb300 import equilibrium as E
    n_real, steps, every = 64, 20000, 100
    g = E.make_grid(8, 310.0, sample_every=every)
    g.set_held_samples(steps // every + 1)
    assert g.n_samples == steps // every + 1 and g.steps_per_loop == 0
    g.reset(seed=5, n_real=n_real)
    S = torch.zeros((n_real, g.n_samples), device="cuda")
    g.advance(steps, S)
    g.sync(120)
    gs = S.double().cpu().numpy()[:, 1:]
    p = orc.material_problem(1, 3, 7, a0=M["a0"], b=8, A0=M["A0"], K0=M["K0"], Ms=M["Ms"], alpha=M["alpha"],
                             T=310.0, dt=20e-15, mode=1, Tc=M["Tc"], H_start_Oe=0.0, H_turn_Oe=0.0,
                             rate_Oe_per_ns=0.0)
    ref = orc.uniform_state(n_real, 21)
    rs, _ = orc.run(p, ref, seed=5, n_steps=steps, sample_every=every, n_samples=g.n_samples)
    rs = rs[:, 1:]
    assert np.abs(gs[:, :5] - rs[:, :5]).max() <= 1e-4  # 500 steps
    k0 = 50  # burn-in: the first 5000 steps
    a, b = np.abs(gs[:, k0:]).mean(1), np.abs(rs[:, k0:]).mean(1)
    se = math.hypot(a.std(ddof=1), b.std(ddof=1)) / math.sqrt(n_real)
    assert abs(a.mean() - b.mean()) <= 3 * se, (a.mean(), b.mean(), se)
    assert 0.3 < a.mean() < 1.0
    with pytest.raises(pkg.LLGError):
        swept = E.make_grid(8, 310.0)
        swept.set_sweep(H_start=100.0, H_turn=-100.0, rate=1000.0, dt=20e-15, sample_dH=1.0)
        swept.set_held_samples(10)
    g.close()


def test_resumable_protocol_run_equals_uninterrupted(pkg, tmp_path):
    """A level's loops run in chunks, the ensemble saved to a checkpoint and restored between
    calls (protocol.run_resumable), give bitwise the observables of one uninterrupted run: the
    noise and the field depend on the absolute step only."""
    from paper_1912_00310_gb300 import protocol as P
    kw = dict(rate=10.0, dt=20e-15)  # b = 8: a cycle of 1e7 steps, a sample every 5000; it switches
    ck = str(tmp_path / "b8.npz")
    r1 = P.run_resumable(8, 64, 3, ck, max_chunks=2, chunk=1 << 18, **kw)
    assert r1["unfinished"] and r1["step"] == 2 << 18
    with pytest.raises(ValueError):
        P.run_resumable(8, 32, 3, ck, max_chunks=1, chunk=1 << 18, **kw)  # another ensemble
    r2 = P.run_resumable(8, 64, 3, ck, chunk=1 << 18, **kw)
    assert not r2.get("unfinished") and r2["samples_finite"]
    assert not (tmp_path / "b8.npz").exists()
    ref = P.run(8, 64, 3, tune=False, **kw)
    assert math.isfinite(ref["Hc_Oe"]) and ref["area_Oe"] > 0
    for k in ("Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe", "area0_Oe", "Hc_down_Oe", "Hc_up_Oe"):
        same = r2[k] == ref[k] or (math.isnan(r2[k]) and math.isnan(ref[k]))
        assert same, (k, r2[k], ref[k])
