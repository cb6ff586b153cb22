"""The C ABI without a GPU: the library loads, exports every function include/llg.h declares,
the binding declares them all, and the host-side logic (parameter setup, sweep bookkeeping,
loop observables) agrees with the oracle."""
import os
import re

import numpy as np
import pytest

from helpers import ROOT


def declared_functions():
    text = open(os.path.join(ROOT, "include", "llg.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(llg_[a-z_0-9]+)\s*\(", text)))


@pytest.fixture(scope="module")
def pkg():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as P
    return P


def test_library_exports_every_declared_symbol(pkg):
    lib = pkg.library()
    names = declared_functions()
    assert len(names) >= 20
    for n in names:
        assert hasattr(lib, n), n
    from paper_1912_00310_gb300 import _lib
    assert sorted(_lib.SIGNATURES) == names


def test_built_for_sm103a_only():
    from paper_1912_00310_gb300 import build
    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def _grid(pkg, b=4, dims=(2, 6, 14)):
    from workloads import MAGNETITE as M
    g = pkg.Grid(*dims, a0=M["a0"], b=b)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    return g


def test_coefficients_match_oracle(pkg, orc):
    from workloads import MAGNETITE as M
    for b, dims, dt in ((1, (8, 24, 56), 2e-15), (4, (2, 6, 14), 10e-15), (8, (1, 3, 7), 20e-15)):
        g = _grid(pkg, b, dims)
        g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=1000.0, dt=dt, sample_dH=1.0)
        c = g.coefficients()
        p = orc.material_problem(*dims, a0=M["a0"], b=b, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                                 alpha=M["alpha"], T=M["T"], dt=dt, mode=1, Tc=M["Tc"],
                                 H_start_Oe=1500.0, H_turn_Oe=-1500.0, rate_Oe_per_ns=1000.0)
        oc = orc.coefficients(p)
        for k in ("c_ex", "c_an", "sigma", "g1", "ag1", "g0"):
            assert c[k] == pytest.approx(oc[k], rel=1e-12), (b, k)
        assert c["zeta"] == pytest.approx(orc.zeta(b, M["T"], M["Tc"]), rel=1e-14)
        assert g.steps_per_loop == 2 * p.n_half
        assert g.sample_every == orc.sample_interval(1.0, 1000.0, dt)
        assert g.n_samples == 6001
        H = g.sample_fields()
        every = g.sample_every
        for k in (0, 1, 1500, 3000, 4500, 6000):
            assert H[k] == pytest.approx(orc.field_Oe(p, k * every), abs=1e-9)
        g.close()


def test_sinusoid_and_block_volume_match_oracle(pkg, orc):
    from workloads import MAGNETITE as M, ROD_DIMS
    b, dt = 4, 10e-15
    g = _grid(pkg, b)
    g.set_sweep(H_start=500.0, H_turn=0.0, rate=1000.0, dt=dt, sample_dH=1.0, shape=1)
    p = orc.material_problem(*ROD_DIMS[b], a0=M["a0"], b=b, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=dt, H_start_Oe=500.0,
                             rate_Oe_per_ns=1000.0, shape=1)
    assert g.steps_per_loop == p.period == 200000
    assert g.n_samples == 2001
    H = g.sample_fields()
    for k in (0, 1, 250, 500, 999, 1000, 1500, 2000):
        assert H[k] == pytest.approx(orc.field_Oe(p, k * g.sample_every), abs=1e-9)
    V = 10752 * M["a0"] ** 3
    g.set_cell_volume(V)
    q = orc.Problem(*ROD_DIMS[b], a=p.a, A=p.A, K=p.K, Ms=p.Ms, alpha=p.alpha, T=p.T, dt=dt, volume=V)
    assert g.coefficients()["sigma"] == pytest.approx(orc.coefficients(q)["sigma"], rel=1e-12)
    g.close()


def test_sweep_validation(pkg):
    g = _grid(pkg)
    with pytest.raises(pkg.LLGError) as e:
        g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=1000.0, dt=10e-15, sample_dH=0.333)
    assert e.value.status == 1
    with pytest.raises(pkg.LLGError) as e:  # a sinusoid period of 4 H_max / (rate dt) = 5 steps
        g.set_sweep(H_start=1.25, H_turn=0.0, rate=1e5, dt=10e-15, sample_dH=1.0, shape=1)
    assert e.value.status == 1
    with pytest.raises(pkg.LLGError) as e:
        g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=1000.0, dt=10e-15, shape=2)
    assert e.value.status == 1
    with pytest.raises(pkg.LLGError):
        g.set_cell_volume(-1.0)
    with pytest.raises(pkg.LLGError) as e:
        g.set_axis_dispersion(-0.1)
    assert e.value.status == 1
    g.set_axis_dispersion(0.0872664626)
    with pytest.raises(pkg.LLGError):
        g.set_material(A0=1e-11, Ms=4.8e5, K0=1e4, alpha=0.1, T=310, u=(0.1, 0, 1))
    with pytest.raises(pkg.LLGError):
        g.set_scaling(mode=3)
    g.close()


def test_loop_stats_match_oracle(pkg, orc):
    rng = np.random.default_rng(1)
    n_half, R = 300, 16
    H = np.concatenate([np.linspace(300, -300, n_half + 1), np.linspace(-300, 300, n_half + 1)[1:]])
    k = np.arange(len(H))
    hcs = rng.normal(80.0, 8.0, size=R)
    S = np.stack([np.where(k <= n_half, np.tanh((H + h) / 30.0), np.tanh((H - h) / 30.0))
                  for h in hcs]).astype(np.float32)
    mine = pkg.loop_stats(S, H, n_half, mode=2, zeta=0.72902, delta=0.511)
    ref = orc.loop_stats(H, S.astype(np.float64), n_half)
    for key in ("Hc", "Hc_se", "area", "area_se", "Hc_down", "Hc_up"):
        assert mine[key + "_Oe"] == pytest.approx(ref[key], rel=1e-10), key
    f = orc.m_rescale(2, 0.72902, 0.511)
    assert mine["area0_Oe"] == pytest.approx(ref["area"] * f / 0.72902, rel=1e-10)
    assert mine["Hc0_Oe"] == pytest.approx(ref["Hc"] / 0.72902, rel=1e-10)
    # one realisation: that loop's own observables and no standard errors
    one = pkg.loop_stats(S[:1], H, n_half, mode=1, zeta=1.0)
    ref1 = orc.loop_stats(H, S[:1].astype(np.float64), n_half)
    for key in ("Hc", "area", "Hc_down", "Hc_up"):
        assert one[key + "_Oe"] == pytest.approx(ref1[key], rel=1e-10), key
    assert np.isnan(one["Hc_se_Oe"]) and np.isnan(one["area_se_Oe"])
    with pytest.raises(pkg.LLGError, match="llg_loop_stats_host"):
        pkg.loop_stats(S, H, len(H), mode=1)  # the turning point past the last sample


def test_gk_flow_matches_oracle(pkg, orc):
    for args in ((2 * np.pi * 0.3613, 4.4e-5, 1.8e-5, 22.0), (2.0, 0.05, 0.08, 5.5), (1.0, 0.0, 0.0, 1.0)):
        mine, ref = pkg.gk_flow(*args), orc.gk_flow(*args)
        for k in ("Tstar", "h", "g", "zeta"):
            assert mine[k] == pytest.approx(ref[k], rel=1e-12, abs=1e-300), (args, k)
    with pytest.raises(pkg.LLGError):
        pkg.gk_flow(1.0, 0.0, 0.0, 0.5)


def test_specific_loss_power_matches_oracle(pkg, orc):
    # the library's formula against the oracle's (whose energy per cycle is pinned by the energy
    # balance of Eq. 1 in test_oracle_loops.py); rho in kg/m^3 against g/cm^3
    for f, Ms, S in ((125e3, 480e3, 171.3), (1e5, 3e5, 12.5), (0.0, 480e3, 400.0)):
        assert pkg.specific_loss_power(f, Ms, S, 5170.0) == pytest.approx(
            orc.specific_loss_power(f, Ms, S, 5.17), rel=1e-12, abs=1e-300)
    assert pkg.specific_loss_power(125e3, 480e3, 171.3, 5170.0) == pytest.approx(198.8, abs=0.05)
    with pytest.raises(pkg.LLGError):
        pkg.specific_loss_power(1e5, 0.0, 100.0, 5170.0)


def test_loop_stats_from_sums_equal_host_statistics(pkg):
    """The three-call distributed form over one process reproduces llg_loop_stats_host, and a
    split of the realisations into two parts, combined by adding the parts' sums, gives the same
    observables (what two processes exchange)."""
    from paper_1912_00310_gb300 import ensemble
    rng = np.random.default_rng(5)
    n_half, R = 200, 24
    H = np.concatenate([np.linspace(250, -250, n_half + 1), np.linspace(-250, 250, n_half + 1)[1:]])
    k = np.arange(len(H))
    S = np.stack([np.where(k <= n_half, np.tanh((H + h) / 25.0), np.tanh((H - h) / 25.0))
                  for h in rng.normal(70.0, 9.0, size=R)]).astype(np.float32)
    S += rng.normal(0, 0.02, size=S.shape).astype(np.float32)
    ref = pkg.loop_stats(S, H, n_half, mode=2, zeta=0.72902, delta=0.511)
    one = ensemble.loop_stats(S, H, n_half, mode=2, zeta=0.72902, delta=0.511)
    for key in ("Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe", "area0_Oe", "Hc0_Oe"):
        assert one[key] == pytest.approx(ref[key], rel=1e-12), key
    assert one["n_real"] == R
    # two parts, sums added by hand
    import ctypes as C
    L = pkg.library()
    dp = lambda a: a.ctypes.data_as(C.POINTER(C.c_double))
    parts = (S[:10], S[10:])
    sums = []
    for part in parts:
        s1 = np.zeros(len(H))
        assert L.llg_loop_moments(part.ctypes.data, part.shape[0], len(H), dp(s1), None) == 0
        sums.append(s1)
    total = sums[0] + sums[1]
    jk = np.zeros(4)
    for part in parts:
        t = np.zeros(4)
        part = np.ascontiguousarray(part)
        assert L.llg_loop_jackknife_terms(part.ctypes.data, part.shape[0], len(H), dp(total), R, dp(H),
                                          n_half, dp(t)) == 0
        jk += t
    st = pkg.LoopStats()
    assert L.llg_loop_stats_from_sums(dp(total), R, len(H), dp(H), n_half, dp(jk), 2, 0.72902, 0.511,
                                      C.byref(st), None) == 0
    d = st.as_dict()
    for key in ("Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe"):
        assert d[key] == pytest.approx(ref[key], rel=1e-10), key


def test_level_temperature_and_held_samples(pkg, orc):
    """T(b) = T0 / (b zeta(b, T0)) (Eq. 12) from the library's map equals the oracle's closed
    form; T(1) = T0; a held field takes a sample count, a swept one refuses it."""
    from paper_1912_00310_gb300 import equilibrium as E
    from workloads import MAGNETITE as M
    assert E.level_temperature(1) == pytest.approx(310.0, rel=1e-15)
    for b in (2, 4, 8):
        assert E.level_temperature(b) == pytest.approx(310.0 / (b * orc.zeta(b, 310.0, M["Tc"])), rel=1e-12)
    g = E.make_grid(4, 310.0, sample_every=50)
    assert g.n_samples == 1
    g.set_held_samples(21)
    assert g.n_samples == 21 and g.sample_every == 50
    g.close()


def test_default_device_is_the_current_cuda_device(pkg, monkeypatch):
    """A grid or peak measurement without an explicit device goes on the caller's current CUDA
    device (one rank per GPU), and on device 0 without CUDA."""
    import torch
    import paper_1912_00310_gb300 as P
    monkeypatch.setattr(torch.cuda, "is_available", lambda: False)
    assert P._current_device() == 0
    monkeypatch.setattr(torch.cuda, "is_available", lambda: True)
    monkeypatch.setattr(torch.cuda, "current_device", lambda: 3)
    assert P._current_device() == 3


def test_tuning_keys_round_trip_and_ranges(pkg):
    """Every tuning key reads back what was set, and each key's documented range is enforced
    (EINVAL), on the host and without a GPU."""
    g = _grid(pkg)
    good = {pkg.TUNE_ROD_KIND: 3, pkg.TUNE_RODS_PER_CTA: 8, pkg.TUNE_CHUNK_STEPS: 4096,
            pkg.TUNE_ROWS_PER_THREAD: 4, pkg.TUNE_GENERIC_KERNEL: 1, pkg.TUNE_BALANCE: 0,
            pkg.TUNE_ADJOINT_STATE_MB: 1024, pkg.TUNE_CELLS_PER_THREAD: 2, pkg.TUNE_GRAD_METHOD: 1,
            pkg.TUNE_HANDOFF_TIMEOUT_MS: 250, pkg.TUNE_WITHHOLD_HANDOFF: 1}
    for key, value in good.items():
        g.set_tuning(key, value)
        assert g.tuning(key) == value, key
    bad = [(pkg.TUNE_ROD_KIND, 4), (pkg.TUNE_ROWS_PER_THREAD, 5), (pkg.TUNE_CELLS_PER_THREAD, 3),
           (pkg.TUNE_GRAD_METHOD, 2), (pkg.TUNE_HANDOFF_TIMEOUT_MS, 0),
           (pkg.TUNE_HANDOFF_TIMEOUT_MS, 3600001), (pkg.TUNE_CHUNK_STEPS, (1 << 30) + 1),
           (pkg.TUNE_ADJOINT_STATE_MB, (1 << 22) + 1), (pkg.TUNE_RODS_PER_CTA, 4097),
           (pkg.TUNE_ROD_KIND, -1), (999, 1)]
    for key, value in bad:
        with pytest.raises(pkg.LLGError) as e:
            g.set_tuning(key, value)
        assert e.value.status == 1, (key, value)
        if key in good:
            assert g.tuning(key) == good[key]  # a refused value leaves the setting
    g.close()


def test_binding_constants_match_the_header():
    """The binding's tuning keys, engines and status codes are the header's."""
    from paper_1912_00310_gb300 import _lib
    text = open(os.path.join(ROOT, "include", "llg.h")).read()
    tune = {m.group(1): int(m.group(2)) for m in re.finditer(r"#define LLG_TUNE_(\w+) (\d+)", text)}
    assert tune and all(getattr(_lib, "TUNE_" + k) == v for k, v in tune.items()), tune
    enums = {m.group(1): int(m.group(2)) for m in re.finditer(r"\b(LLG_\w+) = (\d+)", text)}
    for name in ("AUTO", "RESIDENT", "PLAIN", "STREAM"):
        assert getattr(_lib, "ENGINE_" + name) == enums["LLG_ENGINE_" + name]
    for code, name in _lib.STATUS.items():
        assert enums[name] == code, name


def test_binding_signatures_match_the_header_prototypes():
    """Every prototype of the header has a ctypes signature in the binding with the same number of
    arguments, and the binding declares nothing the header does not."""
    from paper_1912_00310_gb300 import _lib
    text = re.sub(r"/\*.*?\*/", "", open(os.path.join(ROOT, "include", "llg.h")).read(), flags=re.S)
    protos = {}
    for m in re.finditer(r"\b(llg_\w+)\s*\(([^;{]*?)\)\s*;", text):
        args = m.group(2).strip()
        protos[m.group(1)] = 0 if args in ("", "void") else args.count(",") + 1
    assert set(protos) == set(_lib.SIGNATURES), set(protos) ^ set(_lib.SIGNATURES)
    for name, (_, argtypes) in _lib.SIGNATURES.items():
        assert len(argtypes) == protos[name], name
