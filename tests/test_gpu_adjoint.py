"""GPU pathwise adjoint (llg_loop_area_grad) against the FP64 forward-mode oracle gradient and
against central finite differences with common random numbers, within 1e-2 relative."""
import numpy as np
import pytest

from workloads import CONFIGS, MAGNETITE as M, ROD_DIMS, random_unit_state

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    return P


def grid(pkg, dims, scale=(1.0, 1.0, 1.0), alpha=None, b=4, dt=10e-15):
    g = pkg.Grid(*dims, a0=M["a0"], b=b)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=alpha or M["alpha"], T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"], scale=scale)
    g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=1000.0, dt=dt, sample_dH=1.0)
    return g


def target_for(g):
    return 0.92 + 0.05 * np.cos(np.arange(g.n_samples) / 7.0)


def oracle_grad(orc, dims, m0, scale, step0, n_steps, target, alpha=None, seed=0, b=4, dt=10e-15):
    p = orc.material_problem(*dims, a0=M["a0"], b=b, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=alpha or M["alpha"], T=M["T"], dt=dt, mode=1, Tc=M["Tc"],
                             H_start_Oe=1500.0, H_turn_Oe=-1500.0, rate_Oe_per_ns=1000.0)
    return orc.loss_grad(p, m0, target=target, scale=scale, seed=seed, step0=step0,
                         n_steps=n_steps, sample_every=orc.sample_interval(1.0, 1000.0, dt))


@pytest.mark.parametrize("scale,alpha", [((1.0, 1.0, 1.0), None), ((1.25, 0.8, 1.1), 0.5)])
def test_adjoint_matches_oracle_gradient_tiny_grid(pkg, orc, scale, alpha):
    dims, n_real, step0, n_steps = (1, 2, 3), 16, 300, 2000
    g = grid(pkg, dims, scale, alpha)
    g.reset(seed=0, n_real=n_real)
    m0 = random_unit_state(n_real, 6, seed=21, cone=0.6)
    g.set_state(m0.astype(np.float32), step0)
    target = target_for(g)
    L, grad = g.loss_grad(n_steps, target, objective=0, ckpt_every=512)  # 4 segments, last ragged
    Lo, go, _ = oracle_grad(orc, dims, m0.astype(np.float32).astype(np.float64), scale, step0,
                            n_steps, target, alpha)
    assert L == pytest.approx(Lo, rel=1e-3)
    for k in range(3):
        assert grad[k] == pytest.approx(go[k], rel=1e-2, abs=1e-3 * np.abs(go).max()), (k, grad, go)
    assert g.step == step0  # the ensemble was not advanced
    g.close()


def test_adjoint_matches_fp64_central_differences(pkg, orc):
    """The GPU adjoint gradient against central differences of the FP64 oracle's forward loss
    with common random numbers (the same thermal normals at s +- h e_k, h = 1e-4, so the
    difference quotient's truncation and rounding errors are far below the tolerance): within
    1e-2 relative for every component, with no absolute floor.  The b = 4 rod, 8 realisations
    from +z, a 3000-step window."""
    dims, n_real, n_steps, seed = ROD_DIMS[4], 8, 3000, 4
    g = grid(pkg, dims)
    target = target_for(g)
    g.reset(seed=seed, n_real=n_real)
    L, grad = g.loss_grad(n_steps, target, 0, 256)
    p = orc.material_problem(*dims, a0=M["a0"], b=4, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=10e-15, mode=1, Tc=M["Tc"],
                             H_start_Oe=1500.0, H_turn_Oe=-1500.0, rate_Oe_per_ns=1000.0)
    every, K = 100, n_steps // 100

    def loss(scale):
        m = orc.uniform_state(n_real, g.ncells)
        s, _ = orc.run(orc.scaled_problem(p, scale), m, seed=seed, n_steps=n_steps, sample_every=every,
                       n_samples=K + 1)
        mbar = s[:, 1:].mean(0)
        return float(np.mean((mbar - target[1:K + 1]) ** 2))

    assert L == pytest.approx(loss((1.0, 1.0, 1.0)), rel=1e-3)
    h = 1e-4
    for k in range(3):
        sp, sm = np.ones(3), np.ones(3)
        sp[k] += h
        sm[k] -= h
        fd = (loss(tuple(sp)) - loss(tuple(sm))) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-2), (k, grad[k], fd)
    g.close()


def test_adjoint_matches_central_differences(pkg):
    """Central differences of the GPU forward loss (same noise at +-h), FP32, h = 1e-2: the whole
    GPU path on its own, within 1e-2 relative with no absolute floor.  On this case the FP32
    difference quotient agrees with the adjoint to 3e-3 at h = 1e-2 (truncation) and to 3e-4 at
    h = 3e-3; below h = 1e-3 FP32 rounding of the forward loss dominates (1.5e-2 on the smallest
    component, dL/ds_K)."""
    dims, n_real, n_steps = ROD_DIMS[4], 8, 3000
    g = grid(pkg, dims)
    target = target_for(g)
    base = np.array([1.0, 1.0, 1.0])
    g.reset(seed=4, n_real=n_real)
    _, grad = g.loss_grad(n_steps, target, 0, 256)
    for k in range(3):
        h = 1e-2
        vals = []
        for sgn in (1, -1):
            s = base.copy()
            s[k] += sgn * h
            g.set_scaling(mode=1, Tc=M["Tc"], scale=tuple(s))
            g.reset(seed=4, n_real=n_real)
            vals.append(g.loss_grad(n_steps, target, 0, 256)[0])
        fd = (vals[0] - vals[1]) / (2 * h)
        assert grad[k] == pytest.approx(fd, rel=1e-2), (k, grad[k], fd)
        g.set_scaling(mode=1, Tc=M["Tc"], scale=tuple(base))
    g.close()


def test_adjoint_full_rod_vs_oracle(pkg, orc):
    """The b = 4 rod (168 cells), 4 realisations from +z, a 3000-step window: GPU adjoint vs the
    FP64 forward-mode gradient; and the area objective against the oracle's forward loss."""
    dims, n_real, n_steps = ROD_DIMS[4], 4, 3000
    g = grid(pkg, dims)
    g.reset(seed=0, n_real=n_real)
    target = target_for(g)
    L, grad = g.loss_grad(n_steps, target, 0, 512)
    m0 = orc.uniform_state(n_real, g.ncells)
    Lo, go, _ = oracle_grad(orc, dims, m0, (1.0, 1.0, 1.0), 0, n_steps, target)
    assert L == pytest.approx(Lo, rel=1e-3)
    assert np.allclose(grad, go, rtol=1e-2, atol=1e-3 * np.abs(go).max()), (grad, go)
    g.close()


def test_calibration_workload_launch_shape(pkg):
    """The calibration workload: b = 4 rod, 64 realisations, 20k-step window at 1000 Oe/ns,
    checkpoints every 512 steps; finite gradient, loss equal to a plain forward run's, and the
    autograd wrapper returning the same gradient."""
    cfg = CONFIGS["adjoint_b4"]
    g = grid(pkg, cfg["dims"])
    g.reset(seed=cfg["seed"], n_real=cfg["n_real"])
    target = target_for(g)
    L, grad = g.loss_grad(cfg["window_steps"], target, 0, cfg["ckpt_every"])
    assert np.all(np.isfinite(grad)) and np.isfinite(L)
    S = torch.zeros((cfg["n_real"], g.n_samples), device="cuda")
    g.reset(seed=cfg["seed"], n_real=cfg["n_real"])
    g.advance(cfg["window_steps"], S)
    g.sync(120)
    mbar = S[:, 1:cfg["window_steps"] // 100 + 1].double().mean(0).cpu().numpy()
    Lf = float(np.mean((mbar - target[1:len(mbar) + 1]) ** 2))
    assert L == pytest.approx(Lf, rel=1e-6)
    import paper_1912_00310_gb300 as P
    s = torch.tensor([1.0, 1.0, 1.0], dtype=torch.float64, requires_grad=True)
    loss = P.loop_loss(s, g, seed=cfg["seed"], n_real=cfg["n_real"], n_steps=cfg["window_steps"],
                       target=target, ckpt_every=cfg["ckpt_every"], Tc=M["Tc"])
    loss.backward()
    assert float(loss) == pytest.approx(L, rel=1e-12)
    assert np.allclose(s.grad.numpy(), grad, rtol=1e-12)
    g.close()


@pytest.mark.parametrize("ckpt_every,disp", [(512, 0.0), (300, 0.3)])
def test_stored_window_equals_segment_by_segment(pkg, ckpt_every, disp):
    """The two reverse schedules (every segment recomputed at once into a stored window, or one
    segment at a time) compute the same FP32 states: bitwise-equal loss, and gradients that differ
    only by how the parameter partial sums are grouped (FP32 blocks of 64 steps that a segment
    boundary splits, FP64 across blocks), with a ragged last segment and in the dispersed-axis
    mode."""
    dims, n_real, n_steps = ROD_DIMS[4], 6, 2000
    out = []
    for budget in (16384, 0):
        g = grid(pkg, dims)
        g.set_axis_dispersion(disp)
        g.set_tuning(pkg.TUNE_ADJOINT_STATE_MB, budget)
        g.reset(seed=9, n_real=n_real)
        g.advance(150)
        out.append(g.loss_grad(n_steps, target_for(g), 0, ckpt_every))
        assert g.step == 150
        g.close()
    assert out[0][0] == out[1][0]
    # measured on the calibration workload: the two schedules agree bitwise with aligned segments,
    # and regrouping the FP32 block sums moves the gradient by at most 2e-8 relative (against a
    # per-step FP64 accumulation)
    assert np.allclose(out[0][1], out[1][1], rtol=1e-7, atol=0)


@pytest.mark.parametrize("disp,shape", [(0.0, 0), (0.3, 1)])
def test_tangent_method_matches_adjoint_and_oracle(pkg, orc, disp, shape):
    """The forward-mode method (LLG_TUNE_GRAD_METHOD 1): the same loss as the adjoint, bitwise (its
    primal is the forward run's arithmetic), and a gradient within 1e-2 of the FP64 forward-mode
    oracle gradient with no absolute floor and within 1e-4 of the reverse-mode adjoint (the two
    FP32 methods differ only in rounding); with dispersed axes under the sinusoid too."""
    dims, n_real, n_steps = ROD_DIMS[4], 8, 3000
    g = grid(pkg, dims)
    if shape == 1:
        g.set_sweep(H_start=1500.0, H_turn=0.0, rate=1000.0, dt=10e-15, sample_dH=1.0, shape=1)
    g.set_axis_dispersion(disp)
    target = target_for(g)
    out = {}
    for method in (0, 1):
        g.set_tuning(pkg.TUNE_GRAD_METHOD, method)
        g.reset(seed=4, n_real=n_real)
        out[method] = g.loss_grad(n_steps, target, 0, 256)
        assert g.step == 0
    assert out[0][0] == out[1][0]
    assert np.allclose(out[1][1], out[0][1], rtol=1e-4, atol=0), (out[0][1], out[1][1])
    if shape == 0 and disp == 0.0:
        m0 = orc.uniform_state(n_real, g.ncells)
        Lo, go, _ = oracle_grad(orc, dims, m0, (1.0, 1.0, 1.0), 0, n_steps, target, seed=4)
        assert out[1][0] == pytest.approx(Lo, rel=1e-3)
        for k in range(3):
            assert out[1][1][k] == pytest.approx(go[k], rel=1e-2), (k, out[1][1], go)
    g.close()


def test_tangent_method_b2_rod_vs_oracle(pkg, orc):
    """The b = 2 rod (4 x 12 x 28 = 1344 cells, beyond the adjoint's one cell per thread): the
    tangent method (two cells per thread) against the FP64 forward-mode oracle gradient, within
    1e-2 relative with no absolute floor, and its loss against the oracle's."""
    dims, n_real, n_steps, dt = ROD_DIMS[2], 8, 3000, 5e-15
    g = grid(pkg, dims, b=2, dt=dt)
    g.set_tuning(pkg.TUNE_GRAD_METHOD, 1)
    g.reset(seed=4, n_real=n_real)
    target = target_for(g)
    L, grad = g.loss_grad(n_steps, target, 0, 256)
    assert g.step == 0
    m0 = orc.uniform_state(n_real, g.ncells)
    Lo, go, _ = oracle_grad(orc, dims, m0, (1.0, 1.0, 1.0), 0, n_steps, target, seed=4, b=2, dt=dt)
    assert L == pytest.approx(Lo, rel=1e-3)
    for k in range(3):
        assert grad[k] == pytest.approx(go[k], rel=1e-2), (k, grad, go)
    g.set_tuning(pkg.TUNE_GRAD_METHOD, 0)
    with pytest.raises(pkg.LLGError):
        g.loss_grad(n_steps, target, 0, 256)  # the adjoint stops at 1024 cells
    g.close()


def test_gradient_methods_long_period_sweep(pkg, orc):
    """A triangle sweep whose period exceeds 2^31 steps (500 -> -500 Oe at 0.05 Oe/ns, 10 fs) runs
    the gradient kernels' instances with the 64-bit sweep phase: the adjoint and the tangent method
    agree with the FP64 forward-mode oracle gradient within 1e-2 and with each other within 1e-3."""
    dims, n_real, n_steps, dt = (1, 2, 3), 16, 12000, 10e-15
    g = pkg.Grid(*dims, a0=M["a0"], b=4)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=0.5, T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=500.0, H_turn=-500.0, rate=0.05, dt=dt, sample_dH=2e-3)
    assert g.steps_per_loop >= 2 ** 31
    target = 0.92 + 0.05 * np.cos(np.arange(g.n_samples) / 7.0)
    out = {}
    for method in (0, 1):
        g.set_tuning(pkg.TUNE_GRAD_METHOD, method)
        g.reset(seed=9, n_real=n_real)
        out[method] = g.loss_grad(n_steps, target, 0, 4096)
    assert out[0][0] == out[1][0]
    p = orc.material_problem(*dims, a0=M["a0"], b=4, A0=M["A0"], K0=M["K0"], Ms=M["Ms"], alpha=0.5,
                             T=M["T"], dt=dt, mode=1, Tc=M["Tc"], H_start_Oe=500.0, H_turn_Oe=-500.0,
                             rate_Oe_per_ns=0.05)
    Lo, go, _ = orc.loss_grad(p, orc.uniform_state(n_real, g.ncells), target=target, seed=9, step0=0,
                              n_steps=n_steps, sample_every=orc.sample_interval(2e-3, 0.05, dt))
    assert out[1][0] == pytest.approx(Lo, rel=1e-3)
    for method in (0, 1):
        for k in range(3):
            assert out[method][1][k] == pytest.approx(go[k], rel=1e-2, abs=1e-3 * np.abs(go).max()), \
                (method, k, out[method][1], go)
    assert np.allclose(out[1][1], out[0][1], rtol=1e-3, atol=1e-4 * np.abs(go).max())
    g.close()
