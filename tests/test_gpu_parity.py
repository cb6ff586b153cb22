"""GPU parity of the CUDA engines against the FP64 oracle, through the C ABI.

Tolerances: trajectories max |dm| <= 1e-4 over the first 1000 steps (FP32 kernels against the FP64
oracle on the same seeds); single-step noise checks at 2e-6; loop statistics (coercive field,
area) within 3 combined standard errors over 64 realisations.  Engines are compared bitwise with
each other (they share the arithmetic and the summation order).
"""
import math

import numpy as np
import pytest

from workloads import CONFIGS, MAGNETITE as M, ROD_DIMS, DT_BY_B, random_unit_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    assert torch.cuda.is_available()
    return P


def make_grid(pkg, dims, b, dt, *, engine=None, alpha=None, T=None, K0=None, A0=None, mode=1,
              H_start=1500.0, H_turn=-1500.0, rate=1000.0, sample_dH=1.0, kind=0, rods=0):
    g = pkg.Grid(*dims, a0=M["a0"], b=b)
    g.set_material(A0=M["A0"] if A0 is None else A0, Ms=M["Ms"], K0=M["K0"] if K0 is None else K0,
                   alpha=M["alpha"] if alpha is None else alpha, T=M["T"] if T is None else T)
    g.set_scaling(mode=mode, Tc=M["Tc"])
    g.set_sweep(H_start=H_start, H_turn=H_turn, rate=rate, dt=dt, sample_dH=sample_dH)
    if engine is not None:
        g.set_engine(engine)
    if kind:
        g.set_tuning(pkg.TUNE_ROD_KIND, kind)
    if rods:
        g.set_tuning(pkg.TUNE_RODS_PER_CTA, rods)
    return g


def oracle_problem(orc, dims, b, dt, *, alpha=None, T=None, K0=None, A0=None, mode=1,
                   H_start=1500.0, H_turn=-1500.0, rate=1000.0):
    return orc.material_problem(*dims, a0=M["a0"], b=b, A0=M["A0"] if A0 is None else A0,
                                K0=M["K0"] if K0 is None else K0, Ms=M["Ms"],
                                alpha=M["alpha"] if alpha is None else alpha,
                                T=M["T"] if T is None else T, dt=dt, mode=mode, Tc=M["Tc"],
                                H_start_Oe=H_start, H_turn_Oe=H_turn, rate_Oe_per_ns=rate)


def state_of(g, n_real):
    out = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    g.get_state(out)
    g.sync(300.0)
    return out


def test_noise_keys_single_step(pkg, orc):
    """A=0, K=0, H=0: one step from +z moves each cell by its own thermal field only."""
    dims, b, dt = (1, 2, 3), 4, 10e-15
    kw = dict(A0=0.0, K0=0.0, mode=0, H_start=0.0, H_turn=0.0, rate=0.0)
    for engine in (pkg.ENGINE_RESIDENT, pkg.ENGINE_PLAIN):
        g = make_grid(pkg, dims, b, dt, engine=engine, **kw)
        g.reset(seed=7, n_real=3, real_offset=5)
        g.advance(1)
        gpu = state_of(g, 3).double().cpu().numpy()
        ref = orc.uniform_state(3, 6)
        orc.run(oracle_problem(orc, dims, b, dt, **kw), ref, seed=7, real0=5, n_steps=1)
        assert np.max(np.abs(gpu - ref)) < 2e-6
        assert np.max(np.abs(ref - orc.uniform_state(3, 6))) > 1e-3  # noise acted
        g.close()


TRAJ_CASES = [
    # (dims, b, engine, kind, n_real, label)
    ((1, 2, 3), 4, "plain", 0, 3, "tiny grid, plain"),
    ((1, 2, 3), 4, "resident", 1, 3, "tiny grid, two-phase"),
    ((1, 2, 3), 4, "resident", 2, 3, "tiny grid, pipelined nx=1"),
    (ROD_DIMS[4], 4, "resident", 1, 4, "b=4 rod, two-phase"),
    (ROD_DIMS[4], 4, "resident", 2, 4, "b=4 rod, pipelined nx=2"),
    (ROD_DIMS[4], 4, "plain", 0, 4, "b=4 rod, plain"),
    (ROD_DIMS[8], 8, "resident", 1, 5, "b=8 rod, two-phase"),
    ((3, 5, 7), 4, "resident", 2, 2, "3x5x7, pipelined merged"),
    (ROD_DIMS[1], 1, "resident", 0, 2, "b=1 rod, pipelined (auto)"),
]


@pytest.mark.parametrize("dims,b,engine,kind,n_real,label", TRAJ_CASES, ids=[c[-1] for c in TRAJ_CASES])
def test_trajectory_parity_first_1000_steps(pkg, orc, dims, b, engine, kind, n_real, label):
    dt = DT_BY_B[b]
    eng = pkg.ENGINE_PLAIN if engine == "plain" else pkg.ENGINE_RESIDENT
    g = make_grid(pkg, dims, b, dt, engine=eng, kind=kind)
    g.reset(seed=0, n_real=n_real)
    p = oracle_problem(orc, dims, b, dt)
    ref = orc.uniform_state(n_real, g.ncells)
    done = 0
    worst = 0.0
    for upto in (10, 100, 1000):
        g.advance(upto - done)
        orc.run(p, ref, seed=0, step0=done, n_steps=upto - done)
        done = upto
        gpu = state_of(g, n_real).double().cpu().numpy()
        err = float(np.max(np.abs(gpu - ref)))
        worst = max(worst, err)
        assert err <= 1e-4, (label, upto, err)
        assert np.max(np.abs(np.linalg.norm(gpu, axis=-1) - 1.0)) < 1e-6
    assert g.step == 1000
    g.close()


@pytest.mark.parametrize("dims,b,n_real", [(ROD_DIMS[4], 4, 6), (ROD_DIMS[2], 2, 3), (ROD_DIMS[1], 1, 2),
                                            (ROD_DIMS[8], 8, 37)])
def test_engines_bitwise_equal(pkg, dims, b, n_real):
    """Plain engine, two-phase, plane-pipelined and (b = 2, 4, 8) row kernels: bitwise-equal states
    and samples; 37 b = 8 rods leave a partial last CTA of the row kernel (32 rods per CTA)."""
    dt = DT_BY_B[b]
    outs = []
    for eng, kind in ((pkg.ENGINE_PLAIN, 0), (pkg.ENGINE_RESIDENT, 1), (pkg.ENGINE_RESIDENT, 2),
                      (pkg.ENGINE_RESIDENT, 3)):
        if kind == 1 and b == 1:
            continue  # the b = 1 rod does not fit the two-phase kernel
        if kind == 3 and b == 1:
            continue  # the row kernel serves the b = 2, 4, 8 rods
        g = make_grid(pkg, dims, b, dt, engine=eng, kind=kind)
        g.reset(seed=3, n_real=n_real, real_offset=11)
        S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
        g.advance(3 * g.sample_every + 17, S)
        outs.append((state_of(g, n_real), S[:, :4].clone()))
        g.close()
    for st, sm in outs[1:]:
        assert torch.equal(st, outs[0][0])
        assert torch.equal(sm[:, 1:4], outs[0][1][:, 1:4])


@pytest.mark.parametrize("dims", [ROD_DIMS[1], (8, 40, 30)])
def test_b1_kernel_variants_bitwise_equal(pkg, dims):
    """Rods with 8 x planes: the kernels specialised for the plane count (and, for the 8x24x56
    rod, for the whole shape) and the runtime-size kernel, with 2, 3 and 4 rows per thread, give
    bitwise-equal states and samples over several sample intervals."""
    b, dt, n_real = 1, 2e-15, 3
    outs = []
    for generic in (0, 1):
        for rows in (2, 3, 4):
            g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=10000.0)
            g.set_tuning(pkg.TUNE_GENERIC_KERNEL, generic)
            g.set_tuning(pkg.TUNE_ROWS_PER_THREAD, rows)
            g.reset(seed=5, n_real=n_real)
            S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
            g.advance(2 * g.sample_every + 13, S)
            g.advance(g.sample_every - 13, S)
            outs.append((state_of(g, n_real), S[:, :4].clone()))
            g.close()
    assert not torch.isnan(outs[0][1][:, 1:4]).any()
    for st, sm in outs[1:]:
        assert torch.equal(st, outs[0][0])
        assert torch.equal(sm[:, 1:4], outs[0][1][:, 1:4])


@pytest.mark.parametrize("n_real,steps", [(160, 2 * 50 + 7), (2 * 152 + 5, 50), (155, 3), (3 * 152 + 1, 7)])
def test_balanced_schedule_is_bitwise_equal(pkg, n_real, steps):
    """More b = 1 rods than one wave: the balanced schedule (rods split between CTAs at step
    boundaries, hand-off through global memory) gives the same states and samples as one rod
    per CTA."""
    dims, b, dt = ROD_DIMS[1], 1, 2e-15
    outs = []
    for balance in (0, 1):
        g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=1e5, sample_dH=1.0)
        g.set_tuning(pkg.TUNE_BALANCE, balance)
        g.reset(seed=8, n_real=n_real)
        assert g.sample_every == 5
        S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
        g.advance(steps, S)
        g.advance(steps, S)
        outs.append((state_of(g, n_real), S.clone()))
        g.close()
    assert torch.equal(outs[0][0], outs[1][0])
    k = (2 * steps) // 5
    assert not torch.isnan(outs[0][1][:, 1:k + 1]).any()
    assert torch.equal(outs[0][1][:, 1:k + 1], outs[1][1][:, 1:k + 1])


def test_samples_match_oracle(pkg, orc):
    """A short loop (+-5 Oe at 1000 Oe/ns, 1 Oe spacing): every sample against the oracle."""
    dims, b, dt, n_real = ROD_DIMS[4], 4, 10e-15, 4
    kw = dict(H_start=5.0, H_turn=-5.0, rate=1000.0)
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, **kw)
    S = torch.zeros((n_real, g.n_samples), device="cuda")
    g.run_loops(seed=0, n_real=n_real, samples=S, stats=False)
    g.sync(60)
    p = oracle_problem(orc, dims, b, dt, **kw)
    ref = orc.uniform_state(n_real, g.ncells)
    every = g.sample_every
    ns = g.n_samples
    s_ref, _ = orc.run(p, ref, seed=0, n_steps=g.steps_per_loop, sample_every=every, n_samples=ns)
    s_ref[:, 0] = 1.0
    assert ns == 21 and every == 100
    assert np.max(np.abs(S.double().cpu().numpy() - s_ref)) < 1e-4
    g.close()


def _loop_stats_both(pkg, orc, dims, b, dt, n_real, sample_dH, **kw):
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, sample_dH=sample_dH, **kw)
    S = np.zeros((n_real, g.n_samples), dtype=np.float32)
    st = g.run_loops(seed=0, n_real=n_real, samples=S)
    p = oracle_problem(orc, dims, b, dt, **kw)
    ref = orc.uniform_state(n_real, g.ncells)
    s_ref, _ = orc.run(p, ref, seed=0, n_steps=g.steps_per_loop, sample_every=g.sample_every,
                       n_samples=g.n_samples)
    s_ref[:, 0] = 1.0
    H = g.sample_fields()
    k_turn = (g.n_samples - 1) // 2
    o = orc.loop_stats(H, s_ref, k_turn)
    gpu = orc.loop_stats(H, S.astype(np.float64), k_turn)
    g.close()
    return st, o, gpu


def test_loop_statistics_parity(pkg, orc):
    """64 realisations of a full +-400 Oe loop at 250 Oe/ns (alpha = 1) on the b = 8 rod: the
    coercive field and area of the GPU ensemble lie within 3 combined standard errors of the
    oracle's (same seeds); the library's own statistics equal the oracle's statistics of the same
    samples."""
    st, o, gpu = _loop_stats_both(pkg, orc, ROD_DIMS[8], 8, 20e-15, 64, 2.0, alpha=1.0,
                                  H_start=400.0, H_turn=-400.0, rate=250.0)
    assert st["Hc_Oe"] == pytest.approx(gpu["Hc"], rel=1e-6)
    assert st["area_Oe"] == pytest.approx(gpu["area"], rel=1e-6)
    for key in ("Hc", "area"):
        se = math.hypot(o[key + "_se"], gpu[key + "_se"])
        assert abs(o[key] - gpu[key]) <= 3 * se, (key, o[key], gpu[key], se)
    assert 100 < gpu["Hc"] < 400


def test_rod_b4_full_loop_statistics(pkg, orc):
    """The b = 4 rod, 4 realisations, full +-1500 Oe loop at 1000 Oe/ns, 1 Oe sampling: the loop
    area and the ascending-branch crossing of the GPU ensemble within 3 combined standard errors
    of the oracle's.  (At this rate the descending branch has not crossed zero by -1500 Oe.)"""
    cfg = CONFIGS["rod_b4_4real"]
    st, o, gpu = _loop_stats_both(pkg, orc, cfg["dims"], 4, cfg["dt"], cfg["n_real"], 1.0,
                                  H_start=cfg["H_start"], H_turn=cfg["H_turn"], rate=cfg["rate"])
    se = math.hypot(o["area_se"], gpu["area_se"])
    assert abs(o["area"] - gpu["area"]) <= 3 * se, (o["area"], gpu["area"], se)
    assert st["area_Oe"] == pytest.approx(gpu["area"], rel=1e-6)


def test_full_size_b1_ensemble(pkg, orc):
    """The bench launch shape: 256 b = 1 rods (10752 cells each) in one persistent launch.
    Sampled realisations against the oracle after 1000 steps; |m| = 1 everywhere."""
    cfg = CONFIGS["rod_b1_256real"]
    dims, b, dt, n_real = cfg["dims"], 1, cfg["dt"], cfg["n_real"]
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=cfg["rate"])
    g.reset(seed=cfg["seed"], n_real=n_real)
    g.advance(1000)
    gpu = state_of(g, n_real)
    norms = torch.linalg.norm(gpu, dim=-1)
    assert float((norms - 1).abs().max()) < 1e-6
    p = oracle_problem(orc, dims, b, dt, rate=cfg["rate"])
    for r in (0, 97, 255):
        ref = orc.uniform_state(1, g.ncells)
        orc.run(p, ref, seed=cfg["seed"], real0=r, n_steps=1000)
        assert np.max(np.abs(gpu[r].double().cpu().numpy() - ref[0])) <= 1e-4, r
    g.close()


def test_checkpoint_resume_is_bitwise(pkg):
    dims, b, dt, n_real = ROD_DIMS[4], 4, 10e-15, 4
    g1 = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT)
    g1.reset(seed=1, n_real=n_real)
    g1.advance(1234)
    whole = state_of(g1, n_real)
    g2 = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT)
    g2.reset(seed=1, n_real=n_real)
    g2.advance(600)
    mid = state_of(g2, n_real).cpu().numpy()  # through host memory
    g3 = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_PLAIN)
    g3.reset(seed=1, n_real=n_real)
    g3.set_state(np.ascontiguousarray(mid), 600)
    g3.advance(634)
    assert torch.equal(state_of(g3, n_real), whole)
    for g in (g1, g2, g3):
        g.close()


def test_determinism_and_edge_sizes(pkg, orc):
    # a single macrospin (no neighbours) and an odd ensemble that leaves a ragged last CTA
    for dims, n_real in (((1, 1, 1), 3), (ROD_DIMS[4], 7)):
        runs = []
        for _ in range(2):
            g = make_grid(pkg, dims, 4, 10e-15, engine=pkg.ENGINE_RESIDENT, kind=1, rods=2)
            g.reset(seed=9, n_real=n_real)
            g.advance(500)
            runs.append(state_of(g, n_real))
            g.close()
        assert torch.equal(runs[0], runs[1])
        p = oracle_problem(orc, dims, 4, 10e-15)
        ref = orc.uniform_state(n_real, int(np.prod(dims)))
        orc.run(p, ref, seed=9, n_steps=500)
        assert np.max(np.abs(runs[0].double().cpu().numpy() - ref)) <= 1e-4


def test_nonfinite_state_is_reported(pkg):
    dims, b, dt = ROD_DIMS[4], 4, 10e-15
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT)
    g.reset(seed=0, n_real=2)
    m = random_unit_state(2, g.ncells, seed=0).astype(np.float32)
    m[1, 5, :] = np.nan
    g.set_state(m, 0)
    S = torch.zeros((2, g.n_samples), device="cuda")
    g.advance(g.sample_every, S)
    with pytest.raises(pkg.LLGError) as e:
        g.sync(60)
    assert e.value.status == 4
    assert math.isfinite(float(S[0, 1])) and math.isnan(float(S[1, 1]))
    g.close()


def test_sync_timeout_then_recovery(pkg):
    dims, b, dt = ROD_DIMS[1], 1, 2e-15
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=100.0)
    g.reset(seed=0, n_real=152)
    g.advance(20000)
    with pytest.raises(pkg.LLGError) as e:
        g.sync(1e-4)
    assert e.value.status == 5
    g.sync(600)
    g.close()


def test_handoff_wait_runs_out_then_recovery(pkg):
    """The one device-side wait (a CTA of the balanced schedule waiting for the CTA that runs the
    first part of a rod it finishes) is bounded: with the hand-offs withheld on purpose and a 1 ms
    limit, every waiting CTA gives up, the launch ends, and llg_sync reports ETIMEOUT.  The same
    context then runs normally, bitwise equal to one rod per CTA."""
    dims, b, dt, n_real, steps = ROD_DIMS[1], 1, 2e-15, 160, 20
    g = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=1e5, sample_dH=1.0)
    g.set_tuning(pkg.TUNE_HANDOFF_TIMEOUT_MS, 1)
    g.set_tuning(pkg.TUNE_WITHHOLD_HANDOFF, 1)
    g.reset(seed=3, n_real=n_real)
    g.advance(steps)
    with pytest.raises(pkg.LLGError) as e:
        g.sync(120)
    assert e.value.status == 5 and "hand-off" in str(e.value)
    g.set_tuning(pkg.TUNE_WITHHOLD_HANDOFF, 0)
    g.reset(seed=3, n_real=n_real)
    g.advance(steps)
    g.sync(120)
    ref = make_grid(pkg, dims, b, dt, engine=pkg.ENGINE_RESIDENT, rate=1e5, sample_dH=1.0)
    ref.set_tuning(pkg.TUNE_BALANCE, 0)
    ref.reset(seed=3, n_real=n_real)
    ref.advance(steps)
    assert torch.equal(state_of(g, n_real), state_of(ref, n_real))
    g.close()
    ref.close()


def test_run_loops_host_and_device_buffers_agree(pkg):
    dims, b, dt, n_real = ROD_DIMS[8], 8, 20e-15, 3
    kw = dict(H_start=500.0, H_turn=-500.0, rate=1000.0)
    g = make_grid(pkg, dims, b, dt, **kw)
    Sd = torch.zeros((n_real, g.n_samples), device="cuda")
    Sh = np.zeros((n_real, g.n_samples), dtype=np.float32)
    a = g.run_loops(seed=2, n_real=n_real, samples=Sd)
    bb = g.run_loops(seed=2, n_real=n_real, samples=Sh)
    assert np.array_equal(Sd.cpu().numpy(), Sh)
    for k in a:
        assert np.isclose(a[k], bb[k], rtol=0, atol=0, equal_nan=True), k
    assert np.all(Sh[:, 0] == 1.0)
    g.close()
