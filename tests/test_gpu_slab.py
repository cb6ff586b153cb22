"""GPU parity of the streaming (HBM slab) engine against the FP64 oracle and the plain engine.

The streaming kernel shares the arithmetic and neighbour order of the plain engine, so the two
give bitwise-equal states; against the oracle, trajectories stay within 1e-4 over the first 1000
steps.  Samples use a different (two-pass) reduction order and are compared within 1e-6.
"""
import numpy as np
import pytest

from workloads import CONFIGS, MAGNETITE as M

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    return P


def make(pkg, dims, periodic, engine, rate=1000.0, H_start=1500.0, H_turn=-1500.0):
    g = pkg.Grid(*dims, a0=M["a0"], b=1, periodic=periodic)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=H_start, H_turn=H_turn, rate=rate, dt=2e-15, sample_dH=1.0)
    g.set_engine(engine)
    return g


def state(g, n_real):
    out = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    g.get_state(out)
    g.sync(600)
    return out


@pytest.mark.parametrize("dims,periodic,n_real,steps", [
    ((20, 12, 5), 0b011, 2, 1000),   # periodic x, y: every tile wraps
    ((20, 12, 5), 0b000, 2, 1000),   # free faces everywhere
    ((70, 260, 3), 0b011, 1, 400),   # several tiles in x and y, ragged tile widths
    ((9, 7, 1), 0b001, 3, 1000),     # one plane, periodic x only
])
def test_slab_matches_oracle_and_plain(pkg, orc, dims, periodic, n_real, steps):
    g = make(pkg, dims, periodic, pkg.ENGINE_STREAM)
    assert g.engine == pkg.ENGINE_STREAM
    g.reset(seed=2, n_real=n_real, real_offset=3)
    g.advance(steps // 2)
    g.advance(steps - steps // 2)
    got = state(g, n_real)
    gp = make(pkg, dims, periodic, pkg.ENGINE_PLAIN)
    gp.reset(seed=2, n_real=n_real, real_offset=3)
    gp.advance(steps)
    assert torch.equal(got, state(gp, n_real))
    p = orc.material_problem(*dims, a0=M["a0"], b=1, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=2e-15, mode=1, Tc=M["Tc"],
                             H_start_Oe=1500.0, H_turn_Oe=-1500.0, rate_Oe_per_ns=1000.0,
                             periodic=periodic)
    ref = orc.uniform_state(n_real, g.ncells)
    orc.run(p, ref, seed=2, real0=3, n_steps=steps)
    assert np.max(np.abs(got.double().cpu().numpy() - ref)) <= 1e-4
    g.close()
    gp.close()


def test_slab_samples(pkg):
    dims, periodic, n_real = (33, 17, 4), 0b011, 2
    outs = []
    for eng in (pkg.ENGINE_STREAM, pkg.ENGINE_PLAIN):
        g = make(pkg, dims, periodic, eng, rate=1e5)
        g.reset(seed=1, n_real=n_real)
        S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
        g.advance(3 * g.sample_every + 2, S)
        outs.append(S[:, 1:4].clone())
        g.close()
    assert not torch.isnan(outs[0]).any()
    assert float((outs[0] - outs[1]).abs().max()) <= 1e-6


def test_full_slab_launch_shape(pkg):
    """The 512x512x56 periodic slab (14.7M cells): bitwise equal to the plain engine over 20
    steps, unit norms everywhere."""
    cfg = CONFIGS["slab_512x512x56"]
    dims, periodic = cfg["dims"], cfg["periodic"]
    g = make(pkg, dims, periodic, pkg.ENGINE_STREAM, rate=cfg["rate"])
    g.reset(seed=cfg["seed"], n_real=1)
    g.advance(20)
    got = state(g, 1)
    gp = make(pkg, dims, periodic, pkg.ENGINE_PLAIN, rate=cfg["rate"])
    gp.reset(seed=cfg["seed"], n_real=1)
    gp.advance(20)
    assert torch.equal(got, state(gp, 1))
    assert float((torch.linalg.norm(got, dim=-1) - 1).abs().max()) < 1e-6
    assert float(got[..., 2].min()) < 0.999  # the noise acted
    g.close()
    gp.close()
