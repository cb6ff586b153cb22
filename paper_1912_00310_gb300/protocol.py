"""The paper's own hysteresis protocol (arXiv:1912.00310, material and field-sweep paragraphs,
Fig. 2c): magnetite rods of 8 x 24 x 56 a0 at T = 310 K with a 5 degree dispersion of the easy
axis, driven by a sinusoidal field of amplitude 500 Oe at a sweep rate SR = 4 H_max f of
2.5 Oe/ns, coarse-grained at level b with the delta-rescaling of Eq. 13 (delta = 0.511), and
the single-block limit b = 22 (the whole rod as one prism of volume 10752 a0^3).

The paper prints the rescaled loop areas 495, 488, 443, 432 and 472 Oe for b = 1, 2, 4, 8, 22
(the text accompanying Fig. 2c), and for the SR/alpha invariance of Fig. 4 (loops at several
sweep-rate and damping pairs with SR/alpha = 2.5 Oe/ns) a mean area of 171.3 +- 2.8 Oe at b = 4
and 149.4 Oe at b = 8.  `run` computes one level's ensemble of loops on the GPU through the
library's C ABI and returns its observables next to the printed area.

    python -m paper_1912_00310_gb300.protocol --b 8 4 22 --n-real 256
    python -m paper_1912_00310_gb300.protocol --b 4 8 --rates 2.5 5 10 25 --sr-over-alpha 2.5
    python -m paper_1912_00310_gb300.protocol --b 1 --n-real 152 --rate 5 --alpha 0.2 \
        --checkpoint b1.npz --max-seconds 2800      # repeat until the loop is complete

Differences from the paper's runs: the time step grows with b (2, 5, 10, 20, 20 fs for
b = 1, 2, 4, 8, 22; the paper quotes 1 fs), the loop is the first cycle from m = +z at +H_max,
and the axis dispersion is uniform over the solid angle of the 5 degree cone.
"""
import argparse
import json
import math
import time

import numpy as np

from . import ENGINE_AUTO, Grid, loop_stats, specific_loss_power

MAGNETITE = dict(a0=0.839e-9, A0=0.98e-11, Ms=480e3, K0=10e3, alpha=0.1, T=310.0, Tc=858.0,
                 delta=0.511, rho=5170.0)  # rho: density (kg/m^3) of the specific loss power
ROD_CELLS = (8, 24, 56)                     # the rod in cells of a0
BLOCK_B = 22                                # the single-block level
DT_BY_B = {1: 2e-15, 2: 5e-15, 4: 10e-15, 8: 20e-15, BLOCK_B: 20e-15}
PAPER_AREA_OE = {1: 495.0, 2: 488.0, 4: 443.0, 8: 432.0, BLOCK_B: 472.0}
PAPER_AREA_SR_ALPHA_2P5_OE = {4: 171.3, 8: 149.4}  # Fig. 4 text, SR/alpha = 2.5 Oe/ns


def level_grid(b: int):
    """Cells and cell-volume override of level b: the rod cut into (8/b)(24/b)(56/b) cubes of
    edge b a0, or at b = 22 one prism of the rod's whole volume."""
    if b == BLOCK_B:
        return (1, 1, 1), math.prod(ROD_CELLS) * MAGNETITE["a0"] ** 3
    if any(n % b for n in ROD_CELLS):
        raise ValueError(f"b = {b} does not divide the 8 x 24 x 56 rod")
    return tuple(n // b for n in ROD_CELLS), 0.0


def make_grid(b: int, *, H_max=500.0, rate=2.5, dt=None, alpha=None, disp_deg=5.0, mode=2,
              sample_dH=1.0, device=None, stream=None, engine=ENGINE_AUTO):
    M = MAGNETITE
    dims, volume = level_grid(b)
    g = Grid(*dims, a0=M["a0"], b=b, device=device, stream=stream)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"] if alpha is None else alpha,
                   T=M["T"])
    g.set_scaling(mode=mode, Tc=M["Tc"], delta=M["delta"])
    g.set_sweep(H_start=H_max, H_turn=-H_max, rate=rate, dt=dt or DT_BY_B[b], sample_dH=sample_dH,
                shape=1)
    if volume:
        g.set_cell_volume(volume)
    g.set_axis_dispersion(math.radians(disp_deg))
    g.set_engine(engine)
    return g


def specific_loss_power_W_per_g(area_Oe: float, f_Hz: float) -> float:
    """Specific loss power of magnetite (W/g) for a loop of area S (Oe) at frequency f (the
    SR/alpha paragraph), computed by the library (llg_specific_loss_power)."""
    return specific_loss_power(f_Hz, MAGNETITE["Ms"], area_Oe, MAGNETITE["rho"])


def _observables(g, b: int, n_real: int, seed: int, seconds: float, st: dict, paper: dict, kw: dict) -> dict:
    """A level's loop observables next to the printed area (the fields of `run`)."""
    out = dict(b=b, n_real=n_real, seed=seed, cells=g.ncells, steps=g.steps_per_loop,
               dt_s=kw.get("dt") or DT_BY_B[b], seconds=seconds,
               cell_steps_per_s=g.ncells * n_real * g.steps_per_loop / seconds)
    out.update(st)
    out["rate_Oe_per_ns"] = kw.get("rate", 2.5)
    out["alpha"] = MAGNETITE["alpha"] if kw.get("alpha") is None else kw["alpha"]
    # the loss power at the frequency whose SR, at the run's SR/alpha, has alpha = 0.1
    rate0 = out["rate_Oe_per_ns"] * MAGNETITE["alpha"] / out["alpha"]
    out["slp_W_per_g_at_alpha_0p1"] = specific_loss_power_W_per_g(
        out["area0_Oe"], rate0 * 1e9 / (4.0 * kw.get("H_max", 500.0)))
    out["paper_area0_Oe"] = paper.get(b)
    if out["paper_area0_Oe"]:
        out["area0_over_paper"] = out["area0_Oe"] / out["paper_area0_Oe"]
    return out


def run(b: int, n_real: int, seed: int = 0, *, tune=True, paper=PAPER_AREA_OE, **kw) -> dict:
    """One loop per realisation at level b; the loop observables (jackknife standard errors)
    with the rescaled area beside the paper's."""
    g = make_grid(b, **kw)
    try:
        if tune:
            g.reset(seed=seed, n_real=n_real)
            g.autotune(trial_steps=2000)
        S = np.zeros((n_real, g.n_samples), dtype=np.float32)
        t0 = time.perf_counter()
        st = g.run_loops(seed=seed, n_real=n_real, samples=S)
        return _observables(g, b, n_real, seed, time.perf_counter() - t0, st, paper, kw)
    finally:
        g.close()


def run_resumable(b: int, n_real: int, seed: int, checkpoint: str, *, max_seconds: float = float("inf"),
                  max_chunks=None, chunk: int = 1 << 21, paper=PAPER_AREA_OE, **kw) -> dict:
    """The loops of `run` advanced in chunks of `chunk` steps until the loop ends or the time
    (max_seconds) or chunk (max_chunks) budget of this call runs out.  An unfinished ensemble's
    state, its samples so far and its step go to `checkpoint` (.npz), and a call with the same
    arguments resumes from there; the noise and the field are functions of the absolute step, so
    the resumed loops are bitwise those of one uninterrupted run.  Returns the observables of
    `run` once the loop is complete (and removes the checkpoint), else {"unfinished": True, ...}.
    The sample buffer lives in device memory (a torch tensor)."""
    import os

    import torch

    g = make_grid(b, **kw)
    try:
        g.reset(seed=seed, n_real=n_real)
        total, every = g.steps_per_loop, g.sample_every
        dev = torch.device("cuda", g.device)
        S = torch.zeros((n_real, g.n_samples), dtype=torch.float32, device=dev)
        meta = json.dumps(dict(b=b, n_real=n_real, seed=seed, steps=total, n_samples=g.n_samples,
                               **{k: kw[k] for k in sorted(kw) if k != "device"}), sort_keys=True)
        step, spent = 0, 0.0
        if os.path.exists(checkpoint):
            d = np.load(checkpoint)
            if str(d["meta"]) != meta:
                raise ValueError(f"{checkpoint} holds another run ({d['meta']})")
            step, spent = int(d["step"]), float(d["seconds"])
            g.set_state(torch.from_numpy(d["m"]).to(dev), step)
            S.copy_(torch.from_numpy(d["S"]).to(dev))
        else:
            S[:, 0] = 1.0  # sample 0: the saturated start, as llg_run_loops writes it
        t0, chunks = time.perf_counter(), 0
        while step < total and time.perf_counter() - t0 < max_seconds and (max_chunks is None or chunks < max_chunks):
            n = min(chunk, total - step)
            g.advance(n, S)
            g.sync(0.0)
            step += n
            chunks += 1
        spent += time.perf_counter() - t0
        if step < total:
            m = torch.empty((n_real, g.ncells, 3), dtype=torch.float32, device=dev)
            g.get_state(m)
            g.sync(0.0)
            tmp = checkpoint + ".tmp.npz"
            np.savez(tmp, m=m.cpu().numpy(), S=S.cpu().numpy(), step=step, seconds=spent, meta=meta)
            os.replace(tmp, checkpoint)
            return dict(b=b, unfinished=True, step=step, steps=total, seconds=spent, checkpoint=checkpoint)
        Sh = S.cpu().numpy()
        st = loop_stats(Sh, g.sample_fields(), (total // 2) // every, mode=kw.get("mode", 2),
                        zeta=g.coefficients()["zeta"], delta=MAGNETITE["delta"])
        st.pop("mean", None)
        out = _observables(g, b, n_real, seed, spent, st, paper, kw)
        out["samples_finite"] = bool(np.isfinite(Sh).all())
        if os.path.exists(checkpoint):
            os.remove(checkpoint)
        return out
    finally:
        g.close()


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--b", type=int, nargs="+", default=[8, 4, BLOCK_B])
    ap.add_argument("--n-real", type=int, default=256)
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--rate", type=float, default=2.5, help="sweep rate SR = 4 H_max f (Oe/ns)")
    ap.add_argument("--rates", type=float, nargs="+", default=None,
                    help="several sweep rates, each with alpha = rate / --sr-over-alpha")
    ap.add_argument("--sr-over-alpha", type=float, default=None)
    ap.add_argument("--h-max", type=float, default=500.0)
    ap.add_argument("--alpha", type=float, default=None)
    ap.add_argument("--disp-deg", type=float, default=5.0)
    ap.add_argument("--dt", type=float, default=None, help="time step (s); default by level b")
    ap.add_argument("--checkpoint", default=None,
                    help="run one level and rate in resumable chunks, saving the unfinished ensemble here")
    ap.add_argument("--max-seconds", type=float, default=float("inf"),
                    help="with --checkpoint: stepping time of this call")
    a = ap.parse_args(argv)
    pairs = [(a.rate, a.alpha)]
    paper = PAPER_AREA_OE
    if a.rates:
        if not a.sr_over_alpha:
            ap.error("--rates needs --sr-over-alpha")
        pairs = [(r, r / a.sr_over_alpha) for r in a.rates]
        paper = PAPER_AREA_SR_ALPHA_2P5_OE if a.sr_over_alpha == 2.5 else {}
    if a.checkpoint:
        if len(a.b) != 1 or len(pairs) != 1:
            ap.error("--checkpoint takes one level and one rate")
        rate, alpha = pairs[0]
        r = run_resumable(a.b[0], a.n_real, a.seed, a.checkpoint, max_seconds=a.max_seconds, paper=paper,
                          H_max=a.h_max, rate=rate, alpha=alpha, disp_deg=a.disp_deg, dt=a.dt)
        print(json.dumps(r), flush=True)
        return
    for b in a.b:
        for rate, alpha in pairs:
            r = run(b, a.n_real, a.seed, paper=paper, H_max=a.h_max, rate=rate, alpha=alpha,
                    disp_deg=a.disp_deg, dt=a.dt)
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
