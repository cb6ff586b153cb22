"""GB300-native stochastic-LLG hysteresis-loop library (arXiv:1912.00310, coarse-grained
micromagnetic loops).  Python view of the C ABI in include/llg.h.

PyTorch supplies device memory and streams; every step of the integration runs in libllg.so.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import (COEFF_NAMES, ENGINE_AUTO, ENGINE_PLAIN, ENGINE_RESIDENT, ENGINE_STREAM,
                   TUNE_ADJOINT_STATE_MB, TUNE_BALANCE, TUNE_CHUNK_STEPS, TUNE_GENERIC_KERNEL,
                   TUNE_HANDOFF_TIMEOUT_MS, TUNE_ROD_KIND, TUNE_RODS_PER_CTA, TUNE_ROWS_PER_THREAD,
                   TUNE_WITHHOLD_HANDOFF, TUNE_CELLS_PER_THREAD, TUNE_GRAD_METHOD, LLGError, LoopStats)

__all__ = ["Grid", "run_batch", "loop_loss", "LLGError", "LoopStats", "loop_stats", "gk_flow",
           "specific_loss_power", "measure_alu_peak", "ENGINE_AUTO", "ENGINE_RESIDENT",
           "ENGINE_PLAIN", "ENGINE_STREAM", "TUNE_ROD_KIND", "TUNE_RODS_PER_CTA", "TUNE_CHUNK_STEPS",
           "TUNE_ROWS_PER_THREAD", "TUNE_GENERIC_KERNEL", "TUNE_BALANCE", "TUNE_ADJOINT_STATE_MB",
           "TUNE_HANDOFF_TIMEOUT_MS", "TUNE_WITHHOLD_HANDOFF", "TUNE_CELLS_PER_THREAD", "TUNE_GRAD_METHOD", "library"]


def library():
    """The loaded libllg.so (raises ImportError if it has not been built)."""
    return _lib.load()


def _ptr(x) -> int:
    """Address of a torch tensor (device or host) or a numpy array."""
    if isinstance(x, np.ndarray):
        assert x.flags.c_contiguous
        return x.ctypes.data
    assert x.is_contiguous()
    return x.data_ptr()


def _current_stream(device: int):
    import torch
    if not torch.cuda.is_available():
        return None
    return C.c_void_p(torch.cuda.current_stream(device).cuda_stream)


def _current_device() -> int:
    """The caller's current CUDA device (torch's), 0 without one: a process that drives one GPU
    of several (one rank per GPU) gets its contexts, streams and buffers on the same device."""
    import torch
    return torch.cuda.current_device() if torch.cuda.is_available() else 0


class Grid:
    """One grid of nx*ny*nz cubic cells of edge b*a0 (context of the C ABI), on `device` (default:
    the current CUDA device) and `stream` (default: that device's current torch stream)."""

    def __init__(self, nx: int, ny: int, nz: int, *, a0: float, b: int = 1, periodic: int = 0,
                 device: int | None = None, stream=None):
        L = _lib.load()
        self._L = L
        if device is None:
            device = _current_device()
        h = C.c_void_p()
        st = stream if stream is not None else _current_stream(device)
        _lib.check(L.llg_create_grid(C.byref(h), nx, ny, nz, a0, b, periodic, device, st))
        self._h = h
        self.dims = (nx, ny, nz)
        self.device = device

    def close(self):
        if getattr(self, "_h", None):
            self._L.llg_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # ---- setup -------------------------------------------------------------------------
    def set_stream(self, stream):
        _lib.check(self._L.llg_set_stream(self._h, stream))

    def set_material(self, *, A0, Ms, K0, alpha, T, u=(0.0, 0.0, 1.0)):
        uu = (C.c_double * 3)(*u)
        _lib.check(self._L.llg_set_material(self._h, A0, Ms, K0, uu, alpha, T))
        return self

    def set_scaling(self, mode=1, Tc=858.0, delta=0.511, scale=(1.0, 1.0, 1.0)):
        s = (C.c_double * 3)(*scale)
        _lib.check(self._L.llg_set_scaling(self._h, mode, Tc, delta, s))
        return self

    def set_sweep(self, *, H_start, H_turn, rate, dt, sample_dH=1.0, shape=0):
        _lib.check(self._L.llg_set_sweep(self._h, H_start, H_turn, rate, dt, sample_dH, shape))
        return self

    def set_axis_dispersion(self, half_angle_rad: float):
        """Per-cell easy axes uniform over the cone of this half-angle about z (0: axis z)."""
        _lib.check(self._L.llg_set_axis_dispersion(self._h, half_angle_rad))
        return self

    def get_axes(self, out):
        """Copy the ensemble's easy axes [n_real][ncells][3] into out (host or device)."""
        _lib.check(self._L.llg_get_axes(self._h, C.c_void_p(_ptr(out))))
        return out

    def set_held_samples(self, n_samples: int):
        """Sample columns of a held (rate 0) field: sample k after step k * sample_every."""
        _lib.check(self._L.llg_set_held_samples(self._h, int(n_samples)))
        return self

    def set_cell_volume(self, volume_m3: float):
        _lib.check(self._L.llg_set_cell_volume(self._h, volume_m3))
        return self

    def set_engine(self, engine: int):
        _lib.check(self._L.llg_set_engine(self._h, engine))
        return self

    def set_tuning(self, key: int, value: int):
        _lib.check(self._L.llg_set_tuning(self._h, key, int(value)))
        return self

    _TUNE_NAMES = {"kind": TUNE_ROD_KIND, "rods_per_cta": TUNE_RODS_PER_CTA, "chunk_steps": TUNE_CHUNK_STEPS,
                   "rows_per_thread": TUNE_ROWS_PER_THREAD, "cells_per_thread": TUNE_CELLS_PER_THREAD}

    def tuning(self, key) -> int:
        """Current value of a tuning key (an LLG_TUNE_* number or one of kind, rods_per_cta,
        chunk_steps, rows_per_thread, cells_per_thread)."""
        k = self._TUNE_NAMES.get(key, key)
        v = C.c_int64()
        _lib.check(self._L.llg_get_tuning(self._h, int(k), C.byref(v)))
        return v.value

    # ---- queries -----------------------------------------------------------------------
    @property
    def ncells(self) -> int:
        return self._L.llg_num_cells(self._h)

    @property
    def n_samples(self) -> int:
        return self._L.llg_num_samples(self._h)

    @property
    def steps_per_loop(self) -> int:
        return self._L.llg_steps_per_loop(self._h)

    @property
    def sample_every(self) -> int:
        return self._L.llg_sample_every(self._h)

    @property
    def step(self) -> int:
        return self._L.llg_current_step(self._h)

    @property
    def engine(self) -> int:
        return self._L.llg_active_engine(self._h)

    def coefficients(self) -> dict:
        out = (C.c_double * len(COEFF_NAMES))()
        _lib.check(self._L.llg_get_coefficients(self._h, out))
        return dict(zip(COEFF_NAMES, list(out)))

    def sample_fields(self) -> np.ndarray:
        H = np.zeros(self.n_samples)
        _lib.check(self._L.llg_sample_fields(self._h, H.ctypes.data_as(C.POINTER(C.c_double))))
        return H

    # ---- ensemble ----------------------------------------------------------------------
    def reset(self, seed: int, n_real: int, real_offset: int = 0):
        _lib.check(self._L.llg_reset(self._h, seed, n_real, real_offset))

    def advance(self, n_steps: int, samples=None):
        """samples: device tensor float32 [n_real][n_samples] or None."""
        _lib.check(self._L.llg_advance(self._h, int(n_steps),
                                       C.c_void_p(_ptr(samples)) if samples is not None else None))

    def run_loops(self, seed: int, n_real: int, samples, real_offset: int = 0, stats=True):
        """One full loop per realisation into samples (device tensor or host array, float32
        [n_real][n_samples]); returns the loop observables when stats is true."""
        st = LoopStats()
        _lib.check(self._L.llg_run_loops(self._h, seed, n_real, real_offset,
                                         C.c_void_p(_ptr(samples)),
                                         C.byref(st) if stats else None))
        return st.as_dict() if stats else None

    def get_state(self, out):
        step = C.c_int64()
        _lib.check(self._L.llg_get_state(self._h, C.c_void_p(_ptr(out)), C.byref(step)))
        return step.value

    def set_state(self, m, step: int):
        _lib.check(self._L.llg_set_state(self._h, C.c_void_p(_ptr(m)), int(step)))

    def sync(self, timeout_s: float = 0.0):
        _lib.check(self._L.llg_sync(self._h, timeout_s))

    def loss_grad(self, n_steps: int, target=None, objective: int = 0, ckpt_every: int = 512):
        """Loss of the window's mean loop and its pathwise gradient with respect to
        (s_K, s_alpha, s_Ms); returns (L, grad[3]).  target: host array indexed by the global
        sample number (objective 0)."""
        L = C.c_double()
        g = (C.c_double * 3)()
        tp = None
        if target is not None:
            t = np.ascontiguousarray(target, dtype=np.float64)
            tp = t.ctypes.data_as(C.POINTER(C.c_double))
        _lib.check(self._L.llg_loop_area_grad(self._h, int(n_steps), int(objective), tp,
                                              int(ckpt_every), C.byref(L), g))
        return L.value, np.array(list(g))

    def autotune(self, trial_steps: int = 200) -> float:
        rate = C.c_double()
        _lib.check(self._L.llg_autotune(self._h, int(trial_steps), C.byref(rate)))
        return rate.value


def run_batch(grids, max_steps: int, samples=None):
    """Advance every grid's ensemble by min(max_steps, steps left in its loop) in one launch
    (a CUDA graph with one node per grid); returns the steps each grid advanced."""
    L = _lib.load()
    n = len(grids)
    hs = (C.c_void_p * n)(*[g._h.value for g in grids])
    sp = None
    if samples is not None:
        sp = (C.c_void_p * n)(*[_ptr(s) if s is not None else None for s in samples])
    done = (C.c_int64 * n)()
    _lib.check(L.llg_run_batch(hs, n, int(max_steps), sp, done))
    return list(done)


def _loop_loss_function():
    import torch

    class LoopLoss(torch.autograd.Function):
        """L(s_K, s_alpha, s_Ms) of a grid's loop window with its pathwise gradient:
        forward sets the scale factors on the grid, restarts its ensemble (seed, n_real) and
        evaluates the loss; backward returns grad_output times dL/ds."""

        @staticmethod
        def forward(ctx, scales, grid, seed, n_real, n_steps, target, objective, ckpt_every,
                    mode, Tc, delta):
            s = tuple(float(v) for v in scales.detach().cpu().tolist())
            grid.set_scaling(mode=mode, Tc=Tc, delta=delta, scale=s)
            grid.reset(seed, n_real)
            L, g = grid.loss_grad(n_steps, target, objective, ckpt_every)
            ctx.save_for_backward(torch.tensor(g, dtype=scales.dtype, device=scales.device))
            return torch.tensor(L, dtype=scales.dtype, device=scales.device)

        @staticmethod
        def backward(ctx, gout):
            (g,) = ctx.saved_tensors
            return (gout * g,) + (None,) * 10

    return LoopLoss


def loop_loss(scales, grid, *, seed, n_real, n_steps, target=None, objective=0, ckpt_every=512,
              mode=1, Tc=858.0, delta=0.511):
    """Differentiable loop loss (torch autograd) of the calibration scale factors."""
    return _loop_loss_function().apply(scales, grid, seed, n_real, n_steps, target, objective,
                                       ckpt_every, mode, Tc, delta)


def gk_flow(Tstar0: float, h0: float, g0: float, b: float, n_steps: int = 4000) -> dict:
    """The Grinstein-Koch flow (Eqs. 4-7) from l = 0 to ln b: {Tstar, h, g, zeta}."""
    out = (C.c_double * 4)()
    _lib.check(_lib.load().llg_gk_flow(Tstar0, h0, g0, b, int(n_steps), out))
    return dict(zip(["Tstar", "h", "g", "zeta"], list(out)))


def specific_loss_power(f_hz: float, Ms: float, area_Oe: float, rho_kg_m3: float) -> float:
    """Specific loss power (W/g) of a loop of area area_Oe at frequency f_hz:
    f mu0 Ms (1000/4 pi) area / rho (the SR/alpha paragraph's heating figure)."""
    out = C.c_double()
    _lib.check(_lib.load().llg_specific_loss_power(f_hz, Ms, area_Oe, rho_kg_m3, C.byref(out)))
    return out.value


def measure_alu_peak(device: int | None = None) -> dict:
    """Measured 32-bit lane issue rates of the GPU (llg_measure_alu_peak; default: the current
    CUDA device)."""
    out = (C.c_double * 4)()
    _lib.check(_lib.load().llg_measure_alu_peak(_current_device() if device is None else device, out))
    return dict(ffma_lane_ops_per_s=out[0], ffma_sm_mhz=out[1], int_lane_ops_per_s=out[2],
                int_sm_mhz=out[3])


def loop_stats(samples: np.ndarray, H: np.ndarray, k_turn: int, mode=1, zeta=1.0, delta=0.511):
    """Host loop observables of float32 samples [n_real][n_samples] (library implementation)."""
    L = _lib.load()
    s = np.ascontiguousarray(samples, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.float64)
    out = LoopStats()
    mean = np.zeros(s.shape[1])
    _lib.check(L.llg_loop_stats_host(s.ctypes.data, s.shape[0], s.shape[1],
                                     H.ctypes.data_as(C.POINTER(C.c_double)), int(k_turn), mode,
                                     zeta, delta, C.byref(out),
                                     mean.ctypes.data_as(C.POINTER(C.c_double))))
    d = out.as_dict()
    d["mean"] = mean
    return d
