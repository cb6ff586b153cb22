"""Pins of the coarse-graining map (Eqs. 8-13) and the printed material numbers."""
import math

import pytest

from helpers import read_golden
from workloads import MAGNETITE, ROD_DIMS


def golden():
    return {r[0]: (float(r[1]), int(r[2])) for r in read_golden("paper_constants.txt")}


def round_sig(x, d):
    return float(f"{x:.{d}g}")


def test_printed_zeta(orc):
    g = golden()
    M = MAGNETITE
    t = M["T"] / M["Tc"]
    assert round_sig(t, 4) == g["t_310K"][0]
    for b in (2, 4, 8, 22):
        val, digits = g[f"zeta_{b}"]
        assert round(orc.zeta(b, M["T"], M["Tc"]), 4) == pytest.approx(val, abs=1e-12), b
    assert orc.zeta(1, M["T"], M["Tc"]) == pytest.approx(1.0, abs=1e-15)
    # zeta -> 1 - t as b -> infinity, and zeta = 1 at T = 0 for every b
    assert orc.zeta(1e12, M["T"], M["Tc"]) == pytest.approx(1 - t, rel=1e-9)
    assert orc.zeta(4, 0.0, M["Tc"]) == 1.0


def test_exchange_constant_and_tc(orc):
    g = golden()
    M = MAGNETITE
    J = M["a0"] * M["A0"]
    assert round_sig(J, 4) == pytest.approx(g["J_eff_J"][0], rel=1e-12)
    # Tc = 1.44 J_eff / kB prints as 858 K at three digits
    assert round_sig(1.44 * J / orc.KB, 3) == g["Tc_K"][0]


def test_printed_exchange_lengths(orc):
    g = golden()
    M = MAGNETITE
    assert round(orc.exchange_length(1.0, M["A0"], M["Ms"]) * 1e9, 2) == g["lex_0_nm"][0]
    for b in (2, 4, 8, 22):
        # The printed l_ex,b follow from the printed four-digit zeta(b) (l_ex,4 from the
        # unrounded zeta = 0.72902 is 7.0251 nm, which would print as 7.03).
        z_printed = g[f"zeta_{b}"][0]
        lex = orc.exchange_length(z_printed, M["A0"], M["Ms"]) * 1e9
        assert round(lex, 2) == g[f"lex_{b}_nm"][0], b
        z = orc.zeta(b, M["T"], M["Tc"])
        assert abs(orc.exchange_length(z, M["A0"], M["Ms"]) * 1e9 - g[f"lex_{b}_nm"][0]) < 0.01
    assert round(8 * M["a0"] * 1e9, 3) == g["a8_nm"][0]


def test_cell_counts():
    g = golden()
    n1 = math.prod(ROD_DIMS[1])
    assert n1 == g["cells_b1"][0]
    assert math.prod(ROD_DIMS[2]) == g["cells_b2"][0]
    for b, dims in ROD_DIMS.items():
        assert math.prod(dims) * b ** 3 == n1  # rod volume fixed at 10752 a0^3


def test_m_rescale_modes(orc):
    z = 0.72902
    assert orc.m_rescale(0, z, 0.511) == 1.0
    assert orc.m_rescale(1, z, 0.511) == pytest.approx(z)  # Eq. 11
    # Eq. 13 reduces to Eq. 11 at delta = 1 and to no rescale at delta = 0
    assert orc.m_rescale(2, z, 1.0) == pytest.approx(z)
    assert orc.m_rescale(2, z, 0.0) == pytest.approx(1.0)
    assert orc.m_rescale(2, z, 0.511) == pytest.approx(0.511 * z + 0.489)


def test_material_problem_scaling(orc):
    M = MAGNETITE
    p = orc.material_problem(2, 6, 14, a0=M["a0"], b=4, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=1e-14, mode=1, Tc=M["Tc"])
    z = orc.zeta(4, M["T"], M["Tc"])
    assert p.A == pytest.approx(z * M["A0"])            # Eq. 8
    assert p.K == pytest.approx(z ** 3 * M["K0"])       # Eq. 9
    assert p.a == pytest.approx(4 * M["a0"])
    # the b = 4 anisotropy field 2K/(mu0 Ms) is 161.44 Oe at Tc = 858 K
    c = orc.coefficients(p)
    assert c["c_an"] / orc.OE == pytest.approx(161.44, abs=0.01)
    q = orc.material_problem(2, 6, 14, a0=M["a0"], b=4, A0=M["A0"], K0=M["K0"], Ms=M["Ms"],
                             alpha=M["alpha"], T=M["T"], dt=1e-14, mode=0, Tc=M["Tc"])
    assert q.A == M["A0"] and q.K == M["K0"]


def test_specific_loss_power_formula(orc):
    # SLP = f mu0 (1000/4pi) Ms S / rho with S = 171.3 Oe, f = 125 kHz, rho = 5.17 g/cm^3.
    # The printed formula evaluates to 198.8 W/g; the paper prints 207 W/g +-10%, which the
    # recomputed value sits inside (a documented discrepancy, not a pin of the oracle).
    slp = orc.specific_loss_power(125e3, 480e3, 171.3, 5.17)
    assert slp == pytest.approx(198.8, abs=0.1)
    assert abs(slp - 207.0) / 207.0 < 0.10


# ---- the Grinstein-Koch flow (Eqs. 4-7) against its closed forms --------------------------------
@pytest.mark.parametrize("t", [0.1, 0.3613, 0.6])
def test_gk_flow_without_field_and_anisotropy_is_the_closed_form(orc, t):
    """With h = g = 0, F = T*/2pi and the flow integrates in closed form: with u = T*/2pi,
    du/dl = u (u - 1), so u(l) = 1 / (1 + K e^l), K = (1 - u0)/u0, and
    zeta = exp(-integral u) = u0 / b + 1 - u0: the analytic zeta of Eq. 11 with t = u0."""
    for b in (2, 4, 8, 22):
        r = orc.gk_flow(2 * math.pi * t, 0.0, 0.0, b)
        assert r["zeta"] == pytest.approx(t / b + 1 - t, rel=1e-12), b
        K = (1 - t) / t
        assert r["Tstar"] == pytest.approx(2 * math.pi / (1 + K * b), rel=1e-12), b
        assert r["h"] == 0.0 and r["g"] == 0.0


def test_gk_flow_invariants_give_eqs_8_to_10(orc):
    """For any h and g: d/dl [T* zeta e^l] = 0, d/dl [g e^(-2l) zeta^(-2)] = 0 and h = h0 e^(2l).
    With T* = k_B T Lambda / A and Lambda = 2 pi / (b a0) the first gives A(b) = zeta A0 (Eq. 8),
    the second K(b) = zeta^3 K0 (Eq. 9) and the third H(b) = zeta H0 (Eq. 10)."""
    T0, h0, g0 = 2 * math.pi * 0.45, 0.05, 0.08
    for b in (2, 5.5, 22):
        r = orc.gk_flow(T0, h0, g0, b)
        assert r["Tstar"] * r["zeta"] * b == pytest.approx(T0, rel=1e-10)
        assert r["g"] == pytest.approx(g0 * b * b * r["zeta"] ** 2, rel=1e-10)
        assert r["h"] == pytest.approx(h0 * b * b, rel=1e-10)
        # the h and g terms lower F, so zeta lies above the h = g = 0 closed form
        assert r["zeta"] > 0.45 / b + 1 - 0.45


def test_gk_flow_for_magnetite_matches_the_printed_zeta(orc):
    """The paper's claim that for magnetite h and g are so small that the numerical flow is
    practically indistinguishable from the analytic zeta: with the reading t = T/Tc
    (T*0 = 2 pi t) and the field at its 500 Oe amplitude, the flow stays within 0.1% of the
    analytic zeta up to b = 22 (h grows as b^2: 0.021 at b = 22) and within 5e-4 of the four
    printed values."""
    M = MAGNETITE
    red = orc.reduced_parameters(T=M["T"], A=M["A0"], K=M["K0"], Ms=M["Ms"], H_Oe=500.0,
                                 a=M["a0"])
    assert red["h"] < 1e-4 and red["g"] < 1e-4
    t = M["T"] / M["Tc"]
    g = golden()
    for b in (2, 4, 8, 22):
        r = orc.gk_flow(2 * math.pi * t, red["h"], red["g"], b)
        assert 0 < r["zeta"] / orc.zeta(b, M["T"], M["Tc"]) - 1 < 1e-3, b
        assert r["zeta"] == pytest.approx(g[f"zeta_{b}"][0], abs=5e-4), b
    # the physical reduced temperature k_B T Lambda0 / A0 instead corresponds to
    # t' = k_B T / (a0 A0) = 0.52, which does not give the printed values
    tp = red["Tstar"] / (2 * math.pi)
    assert tp == pytest.approx(0.5206, abs=1e-4)
    assert round(orc.gk_flow(red["Tstar"], red["h"], red["g"], 4)["zeta"], 4) != g["zeta_4"][0]


def test_protocol_levels_and_loss_power():
    """The protocol runner's host-side pieces: the rod cut at each level (the printed cell counts),
    the b = 22 block's volume, and the specific loss power formula on the printed S = 171.3 Oe."""
    from paper_1912_00310_gb300 import protocol as P
    assert P.level_grid(1) == ((8, 24, 56), 0.0)
    assert P.level_grid(2)[0] == (4, 12, 28) and P.level_grid(8)[0] == (1, 3, 7)
    dims, V = P.level_grid(22)
    assert dims == (1, 1, 1) and V == pytest.approx(10752 * MAGNETITE["a0"] ** 3, rel=1e-12)
    with pytest.raises(ValueError):
        P.level_grid(3)
    # f mu0 (1000/4pi) Ms S / rho at 125 kHz: 198.8 W/g for the printed area (R13)
    assert P.specific_loss_power_W_per_g(171.3, 125e3) == pytest.approx(198.8, abs=0.05)
    # a resumable run takes one level and one rate (refused before any device work)
    for argv in (["--b", "1", "4", "--checkpoint", "x.npz"],
                 ["--b", "4", "--rates", "2.5", "5", "--sr-over-alpha", "2.5", "--checkpoint", "x.npz"]):
        with pytest.raises(SystemExit):
            P.main(argv)
