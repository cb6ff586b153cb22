"""The batching layer (uneven jobs in one graph launch) and the autotuner, through the C ABI.

A batch must give every job exactly the state and samples it gets when run alone (the engines
share the arithmetic), advance each job by min(max_steps, steps left in its loop), and leave jobs
in the batch independent; the autotuner must pick a launch shape without advancing the ensemble.
"""
import numpy as np
import pytest

from workloads import MAGNETITE as M, ROD_DIMS, DT_BY_B

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    return P


def job(pkg, b, rate, alpha, n_real, seed, sample_dH=2.0):
    g = pkg.Grid(*ROD_DIMS[b], a0=M["a0"], b=b)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=alpha, T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=rate, dt=DT_BY_B[b], sample_dH=sample_dH)
    g.set_engine(pkg.ENGINE_RESIDENT)
    g.reset(seed=seed, n_real=n_real)
    return g


def state(g, n_real):
    out = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    g.get_state(out)
    g.sync(600)
    return out


SPECS = [(1, 1e4, 0.1, 2), (2, 1e4, 0.5, 3), (4, 1e5, 1.0, 5), (8, 1e5, 0.05, 7), (4, 1e5, 0.1, 1)]


def test_batch_equals_jobs_run_alone(pkg):
    W = 700
    grids = [job(pkg, b, r, a, n, seed=10 + i) for i, (b, r, a, n) in enumerate(SPECS)]
    samples = [torch.full((n, g.n_samples), float("nan"), device="cuda")
               for g, (_, _, _, n) in zip(grids, SPECS)]
    done = pkg.run_batch(grids, W, samples)
    done2 = pkg.run_batch(grids, W, samples)
    for i, (g, (b, r, a, n)) in enumerate(zip(grids, SPECS)):
        assert done[i] == min(W, g.steps_per_loop) and done2[i] == min(W, g.steps_per_loop - done[i])
        alone = job(pkg, b, r, a, n, seed=10 + i)
        S = torch.full((n, alone.n_samples), float("nan"), device="cuda")
        alone.advance(done[i] + done2[i], S)
        assert torch.equal(state(g, n), state(alone, n)), (b, r, a)
        k = (done[i] + done2[i]) // g.sample_every
        assert torch.equal(samples[i][:, 1:k + 1], S[:, 1:k + 1])
        assert g.step == done[i] + done2[i]
        alone.close()
    for g in grids:
        g.close()


def test_batch_stops_jobs_at_loop_end(pkg):
    g = job(pkg, 8, 1e6, 1.0, 2, seed=1, sample_dH=20.0)  # a loop of 300 steps at 20 fs
    assert g.steps_per_loop == 300
    h = job(pkg, 4, 1e5, 0.1, 2, seed=2)
    d = pkg.run_batch([g, h], 250)
    assert d == [250, 250]
    d = pkg.run_batch([g, h], 250)
    assert d == [50, 250]
    d = pkg.run_batch([g, h], 250)
    assert d[0] == 0 and g.step == 300
    g.close()
    h.close()


def test_autotune_keeps_the_ensemble(pkg):
    for b, n in ((1, 160), (4, 64)):
        g = job(pkg, b, 1e4, 0.1, n, seed=3)
        g.advance(10)
        before = state(g, n).clone()
        rate = g.autotune(trial_steps=40)
        assert rate > 1e9
        assert g.step == 10
        assert torch.equal(state(g, n), before)
        ref = job(pkg, b, 1e4, 0.1, n, seed=3)
        ref.advance(60)
        g.advance(50)
        assert torch.equal(state(g, n), state(ref, n))  # the tuned shape computes the same
        g.close()
        ref.close()


def test_autotune_cache_follows_the_sweep(pkg):
    """Two b = 4 ensembles of the same size, one swept within 2^31 steps and one whose sweep
    phase needs 64 bits (the +-1500 Oe loop at 0.1 Oe/ns): the second autotune does not reuse the
    first's launch shape (the row kernel takes only 32-bit sweeps), and its ensemble then
    advances bitwise like the plain engine's."""
    n_real = 64
    a = job(pkg, 4, 1000.0, 0.1, n_real, 0)
    a.autotune(trial_steps=200)
    b = job(pkg, 4, 0.1, 0.1, n_real, 0)
    assert b.steps_per_loop >= 2 ** 31
    b.autotune(trial_steps=200)
    b.advance(300)
    c = job(pkg, 4, 0.1, 0.1, n_real, 0)
    c.set_engine(pkg.ENGINE_PLAIN)
    c.advance(300)
    sb, sc = state(b, n_real), state(c, n_real)
    assert torch.isfinite(sb).all()
    assert torch.equal(sb, sc)
    for g in (a, b, c):
        g.close()
