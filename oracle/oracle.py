"""Python view of the FP64 CPU oracle (``llg_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` use this module.  The product package never imports it, and it imports nothing from
the product package.

The C file holds the arithmetic (Eq. 1 LLG right-hand side, the effective field, the Heun step,
Philox4x32-10 + Box-Muller, the coarse-graining map of Eqs. 8-13 and the loop observables).  This
module only marshals numpy arrays and applies the parameter map of Eqs. 8-9 (A(b) = zeta A0,
K(b) = zeta^3 K0) to build a simulation-level problem.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import math
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "llg_oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lib = None
_lock = threading.Lock()


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (plain -O2, no fast-math) into oracle/liboracle.so."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(
            ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-Wall", "-o", tmp, _SRC,
             "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Problem(C.Structure):
    _fields_ = [("nx", C.c_int), ("ny", C.c_int), ("nz", C.c_int), ("periodic", C.c_uint),
                ("a", C.c_double), ("volume", C.c_double), ("A", C.c_double), ("K", C.c_double),
                ("Ms", C.c_double), ("alpha", C.c_double), ("T", C.c_double), ("u", C.c_double * 3),
                ("dt", C.c_double), ("H_start_Oe", C.c_double), ("H_turn_Oe", C.c_double),
                ("n_half", C.c_int64), ("shape", C.c_int), ("period", C.c_int64),
                ("disp", C.c_double)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            L = C.CDLL(build())
            dp = C.POINTER(C.c_double)
            u32p = C.POINTER(C.c_uint32)
            L.orc_philox4x32_10.argtypes = [u32p, u32p, u32p]
            L.orc_uniform24.argtypes = [C.c_uint32]
            L.orc_uniform24.restype = C.c_double
            L.orc_thermal_normals.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_uint64, dp]
            L.orc_zeta.argtypes = [C.c_double] * 3
            L.orc_zeta.restype = C.c_double
            L.orc_easy_axis.argtypes = [C.c_void_p, C.c_uint32, C.c_uint32, C.c_uint32, dp]
            L.orc_gk_flow.argtypes = [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, dp]
            L.orc_exchange_length.argtypes = [C.c_double] * 3
            L.orc_exchange_length.restype = C.c_double
            L.orc_m_rescale.argtypes = [C.c_int, C.c_double, C.c_double]
            L.orc_m_rescale.restype = C.c_double
            L.orc_coefficients.argtypes = [C.POINTER(_Problem), dp]
            L.orc_field_Oe.argtypes = [C.POINTER(_Problem), C.c_int64]
            L.orc_field_Oe.restype = C.c_double
            L.orc_run.argtypes = [C.POINTER(_Problem), C.c_uint32, C.c_int, C.c_uint32, C.c_int64,
                                  C.c_int64, dp, C.c_int64, C.c_int64, dp, dp, C.c_int64, C.c_int]
            L.orc_run.restype = C.c_int
            L.orc_energy.argtypes = [C.POINTER(_Problem), dp, C.c_double]
            L.orc_energy.restype = C.c_double
            L.orc_coercive_field.argtypes = [dp, dp, C.c_int64, C.c_int64, dp, dp]
            L.orc_coercive_field.restype = C.c_double
            L.orc_loop_area.argtypes = [dp, dp, C.c_int64]
            L.orc_loop_area.restype = C.c_double
            L.orc_loop_stats.argtypes = [dp, dp, C.c_int, C.c_int64, C.c_int64, dp, dp]
            L.orc_loss_grad.argtypes = [C.POINTER(_Problem), dp, C.c_uint32, C.c_int, C.c_uint32,
                                        C.c_int64, C.c_int64, dp, C.c_int64, dp, dp, dp, C.c_int]
            L.orc_loss_grad.restype = C.c_int64
            L.orc_specific_loss_power.argtypes = [C.c_double] * 4
            L.orc_specific_loss_power.restype = C.c_double
            _lib = L
    return _lib


def _dp(a: np.ndarray):
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(C.POINTER(C.c_double))


# ------------------------------------------------------------------------------------------------
# Physical constants used by the oracle's Python-side parameter map (same values as the C file).
MU0 = 4e-7 * math.pi
GAMMA_E = 1.76e11
KB = 1.380649e-23
OE = 1000.0 / (4.0 * math.pi)


def philox4x32_10(ctr, key) -> np.ndarray:
    c = (C.c_uint32 * 4)(*[int(v) & 0xFFFFFFFF for v in ctr])
    k = (C.c_uint32 * 2)(*[int(v) & 0xFFFFFFFF for v in key])
    o = (C.c_uint32 * 4)()
    lib().orc_philox4x32_10(c, k, o)
    return np.array(list(o), dtype=np.uint32)


def uniform24(x: int) -> float:
    return lib().orc_uniform24(int(x) & 0xFFFFFFFF)


def thermal_normals(seed: int, real: int, cell: int, step: int) -> np.ndarray:
    out = np.zeros(3)
    lib().orc_thermal_normals(seed & 0xFFFFFFFF, real & 0xFFFFFFFF, cell & 0xFFFFFFFF, step, _dp(out))
    return out


def easy_axes(p: Problem, seed: int, n_real: int, real0: int = 0) -> np.ndarray:
    """Easy axis of every cell of every realisation, [n_real][ncells][3]."""
    pc = p._c()
    out = np.zeros((n_real, p.ncells, 3))
    L = lib()
    for r in range(n_real):
        for i in range(p.ncells):
            L.orc_easy_axis(C.byref(pc), seed & 0xFFFFFFFF, (real0 + r) & 0xFFFFFFFF, i,
                            _dp(out[r, i]))
    return out


def gk_flow(Tstar0: float, h0: float, g0: float, b: float, n: int = 4000) -> dict:
    """Grinstein-Koch flow (Eqs. 4-7) from l = 0 to ln b: reduced temperature T*, field h and
    anisotropy g at level b and the magnetisation factor zeta."""
    out = np.zeros(4)
    lib().orc_gk_flow(Tstar0, h0, g0, b, int(n), _dp(out))
    return dict(zip(["Tstar", "h", "g", "zeta"], out.tolist()))


def reduced_parameters(*, T, A, K, Ms, H_Oe, a):
    """Eqs. 4-5: T* = k_B T Lambda / A, h = mu0 Ms H / (A Lambda^2) (H in Oe converted to A/m),
    g = K / (A Lambda^2), with the cut-off Lambda = 2 pi / a of cells of edge a."""
    lam = 2.0 * math.pi / a
    return dict(Tstar=KB * T * lam / A, h=MU0 * Ms * H_Oe * OE / (A * lam * lam),
                g=K / (A * lam * lam))


def zeta(b: float, T: float, Tc: float) -> float:
    """Eq. 11's coarse-graining factor zeta(b) = t/b + 1 - t, t = T/Tc."""
    return lib().orc_zeta(b, T, Tc)


def exchange_length(z: float, A0: float, Ms: float) -> float:
    return lib().orc_exchange_length(z, A0, Ms)


def m_rescale(mode: int, z: float, delta: float) -> float:
    return lib().orc_m_rescale(mode, z, delta)


@dataclasses.dataclass
class Problem:
    """A simulation-level problem: grid, already-scaled material, time step and field sweep."""
    nx: int
    ny: int
    nz: int
    a: float
    A: float
    K: float
    Ms: float
    alpha: float
    T: float
    dt: float
    H_start_Oe: float = 0.0
    H_turn_Oe: float = 0.0
    n_half: int = 0
    u: tuple = (0.0, 0.0, 1.0)
    periodic: int = 0
    volume: float | None = None
    shape: int = 0     # 0 triangle, 1 sinusoid of amplitude H_start
    period: int = 0    # sinusoid: steps per cycle
    disp: float = 0.0  # easy-axis dispersion: cone half-angle about z (rad), 0 = the axis u

    @property
    def ncells(self) -> int:
        return self.nx * self.ny * self.nz

    def _c(self) -> _Problem:
        p = _Problem()
        p.nx, p.ny, p.nz, p.periodic = self.nx, self.ny, self.nz, self.periodic
        p.a = self.a
        p.volume = self.volume if self.volume is not None else self.a ** 3
        p.A, p.K, p.Ms, p.alpha, p.T = self.A, self.K, self.Ms, self.alpha, self.T
        for i in range(3):
            p.u[i] = self.u[i]
        p.dt = self.dt
        p.H_start_Oe, p.H_turn_Oe, p.n_half = self.H_start_Oe, self.H_turn_Oe, int(self.n_half)
        p.shape, p.period = int(self.shape), int(self.period)
        p.disp = float(self.disp)
        return p


def material_problem(nx, ny, nz, *, a0, b, A0, K0, Ms, alpha, T, dt, mode=1, Tc=858.0,
                     scale=(1.0, 1.0, 1.0), H_start_Oe=0.0, H_turn_Oe=0.0, rate_Oe_per_ns=0.0,
                     periodic=0, u=(0.0, 0.0, 1.0), shape=0, volume=None, disp=0.0) -> Problem:
    """Level-b problem from the unscaled material.  mode 0: A0, K0 unchanged (Fig. 2a);
    modes 1 and 2: A(b) = zeta A0 (Eq. 8), K(b) = zeta^3 K0 (Eq. 9).  scale = (s_K, s_alpha, s_Ms)
    multiplies K(b), alpha and Ms.  shape 0: the sweep is a triangle H_start -> H_turn -> H_start
    at the given rate (Oe/ns).  shape 1: the sinusoid of amplitude H_max = H_start whose sweep
    rate SR = 4 H_max f is the given rate, so a cycle is 4 H_max / (rate dt) steps.  volume
    replaces (b a0)^3 in the thermal field (the single-block limit).  disp (rad) spreads each
    cell's easy axis uniformly over the cone of that half-angle about z."""
    z = zeta(b, T, Tc) if mode in (1, 2) else 1.0
    A = z * A0
    K = z ** 3 * K0 * scale[0]
    period = 0
    if shape == 1:
        period = sweep_steps(4.0 * H_start_Oe, 0.0, rate_Oe_per_ns, dt)
        n_half = period // 2
    else:
        n_half = sweep_steps(H_start_Oe, H_turn_Oe, rate_Oe_per_ns, dt)
    return Problem(nx, ny, nz, a=b * a0, A=A, K=K, Ms=Ms * scale[2], alpha=alpha * scale[1], T=T,
                   dt=dt, H_start_Oe=H_start_Oe, H_turn_Oe=H_turn_Oe, n_half=n_half, u=u,
                   periodic=periodic, shape=shape, period=period, volume=volume, disp=disp)


def sweep_steps(H_start_Oe, H_turn_Oe, rate_Oe_per_ns, dt) -> int:
    """Steps from H_start to H_turn at rate (Oe/ns) and step dt (s); 0 for a constant field."""
    if rate_Oe_per_ns == 0.0 or H_start_Oe == H_turn_Oe:
        return 0
    per_step = rate_Oe_per_ns * 1e9 * dt
    n = abs(H_start_Oe - H_turn_Oe) / per_step
    if abs(n - round(n)) > 1e-6 * max(1.0, n):
        raise ValueError("sweep span is not a whole number of steps")
    return int(round(n))


def sample_interval(sample_dH_Oe, rate_Oe_per_ns, dt) -> int:
    per_step = rate_Oe_per_ns * 1e9 * dt
    n = sample_dH_Oe / per_step
    if abs(n - round(n)) > 1e-6 * max(1.0, n):
        raise ValueError("sample spacing is not a whole number of steps")
    return int(round(n))


def coefficients(p: Problem) -> dict:
    out = np.zeros(6)
    pc = p._c()
    lib().orc_coefficients(C.byref(pc), _dp(out))
    return dict(zip(["g0", "g1", "ag1", "c_ex", "c_an", "sigma"], out.tolist()))


def field_Oe(p: Problem, n: int) -> float:
    pc = p._c()
    return lib().orc_field_Oe(C.byref(pc), int(n))


def uniform_state(n_real: int, ncells: int, direction=(0.0, 0.0, 1.0)) -> np.ndarray:
    d = np.asarray(direction, dtype=np.float64)
    d = d / np.linalg.norm(d)
    return np.ascontiguousarray(np.broadcast_to(d, (n_real, ncells, 3)).copy())


def run(p: Problem, m_state: np.ndarray, *, seed: int = 0, real0: int = 0, step0: int = 0,
        n_steps: int, sample_every: int = 0, n_samples: int = 0, samples: np.ndarray | None = None,
        timeavg_burn_in: int | None = None, threads: int | None = None):
    """Advance m_state [n_real][ncells][3] (float64, modified in place) by n_steps Heun steps.
    Returns (samples, timeavg) where samples [n_real][n_samples] holds the cell-averaged m_z after
    every step index that is a multiple of sample_every, and timeavg [n_real] the mean cell-averaged
    m_z over the steps >= timeavg_burn_in of this call (None when not asked for)."""
    assert m_state.dtype == np.float64 and m_state.flags.c_contiguous
    n_real = m_state.shape[0]
    assert m_state.shape[1] == p.ncells and m_state.shape[2] == 3
    if sample_every and samples is None:
        samples = np.full((n_real, n_samples), np.nan)
    tav = np.zeros(n_real) if timeavg_burn_in is not None else None
    pc = p._c()
    nt = threads or os.cpu_count() or 1
    lib().orc_run(C.byref(pc), seed & 0xFFFFFFFF, n_real, real0 & 0xFFFFFFFF, int(step0), int(n_steps),
                  _dp(m_state), int(sample_every), int(n_samples),
                  _dp(samples) if samples is not None else None,
                  _dp(tav) if tav is not None else None,
                  int(timeavg_burn_in or 0), int(nt))
    return samples, tav


def energy(p: Problem, m: np.ndarray, H_Oe: float) -> float:
    m = np.ascontiguousarray(m, dtype=np.float64)
    pc = p._c()
    return lib().orc_energy(C.byref(pc), _dp(m), float(H_Oe))


def loop_stats(H: np.ndarray, samples: np.ndarray, k_turn: int) -> dict:
    """Mean loop, coercive field (Hc, with descending / ascending crossings) and loop area, with
    delete-one jackknife standard errors over realisations."""
    H = np.ascontiguousarray(H, dtype=np.float64)
    S = np.ascontiguousarray(samples, dtype=np.float64)
    n_real, n = S.shape
    out = np.zeros(6)
    mean = np.zeros(n)
    lib().orc_loop_stats(_dp(H), _dp(S), n_real, n, int(k_turn), _dp(out), _dp(mean))
    return dict(Hc=out[0], Hc_se=out[1], area=out[2], area_se=out[3], Hc_down=out[4], Hc_up=out[5],
                mean=mean)


def coercive_field(H, m, k_turn):
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    d = C.c_double()
    u = C.c_double()
    hc = lib().orc_coercive_field(_dp(H), _dp(m), len(H), int(k_turn), C.byref(d), C.byref(u))
    return hc, d.value, u.value


def loop_area(H, m) -> float:
    H = np.ascontiguousarray(H, dtype=np.float64)
    m = np.ascontiguousarray(m, dtype=np.float64)
    return lib().orc_loop_area(_dp(H), _dp(m), len(H))


def specific_loss_power(f_hz, Ms, S_Oe, rho_g_cm3) -> float:
    return lib().orc_specific_loss_power(f_hz, Ms, S_Oe, rho_g_cm3)


def loss_grad(p: Problem, m0: np.ndarray, *, target: np.ndarray, scale=(1.0, 1.0, 1.0), seed=0,
              real0=0, step0=0, n_steps: int, sample_every: int, threads=None):
    """Loss L = mean_k (mbar_k - target[k])^2 over the samples of the window and its forward-mode
    gradient with respect to (s_K, s_alpha, s_Ms) (pathwise: the thermal normals fixed).
    p is the problem at scale (1, 1, 1); target is indexed by the global sample number.
    Returns (L, grad[3], mbar[K])."""
    m0 = np.ascontiguousarray(m0, dtype=np.float64)
    target = np.ascontiguousarray(target, dtype=np.float64)
    n_real = m0.shape[0]
    k_first = step0 // sample_every + 1
    k_last = (step0 + n_steps) // sample_every
    out = np.zeros(4)
    mean = np.zeros(max(1, k_last - k_first + 1))
    sc = np.ascontiguousarray(scale, dtype=np.float64)
    pc = p._c()
    lib().orc_loss_grad(C.byref(pc), _dp(sc), seed & 0xFFFFFFFF, n_real, real0 & 0xFFFFFFFF,
                        int(step0), int(n_steps), _dp(m0), int(sample_every), _dp(target), _dp(out),
                        _dp(mean), int(threads or os.cpu_count() or 1))
    return out[0], out[1:4].copy(), mean[:max(0, k_last - k_first + 1)]


def scaled_problem(p: Problem, scale) -> Problem:
    """The problem with K, alpha and Ms multiplied by (s_K, s_alpha, s_Ms)."""
    return dataclasses.replace(p, K=p.K * scale[0], alpha=p.alpha * scale[1], Ms=p.Ms * scale[2])
