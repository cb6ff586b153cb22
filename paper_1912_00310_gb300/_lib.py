"""ctypes binding of libllg.so (include/llg.h): argument marshalling only.

Every step of the path runs in the CUDA library.  If libllg.so is missing the import fails
loudly; there is no CPU fallback.
"""
from __future__ import annotations

import ctypes as C
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libllg.so")

# names and order of llg_get_coefficients
COEFF_NAMES = ("zeta", "A", "K", "Ms", "alpha", "a", "V", "g0", "g1", "ag1", "c_ex", "c_an",
               "sigma", "H_start_Am", "slope_Am", "m_rescale")

STATUS = {0: "LLG_OK", 1: "LLG_EINVAL", 2: "LLG_ENOMEM", 3: "LLG_ECUDA", 4: "LLG_ENONFINITE",
          5: "LLG_ETIMEOUT", 6: "LLG_EUNSUPPORTED"}

ENGINE_AUTO, ENGINE_RESIDENT, ENGINE_PLAIN, ENGINE_STREAM = 0, 1, 2, 3
TUNE_ROD_KIND, TUNE_RODS_PER_CTA, TUNE_CHUNK_STEPS, TUNE_ROWS_PER_THREAD = 1, 2, 3, 4
TUNE_GENERIC_KERNEL, TUNE_BALANCE, TUNE_ADJOINT_STATE_MB = 5, 6, 7
TUNE_HANDOFF_TIMEOUT_MS, TUNE_WITHHOLD_HANDOFF, TUNE_CELLS_PER_THREAD, TUNE_GRAD_METHOD = 8, 9, 10, 11


class LoopStats(C.Structure):
    _fields_ = [(n, C.c_double) for n in (
        "Hc_Oe", "Hc_se_Oe", "area_Oe", "area_se_Oe", "Hc_down_Oe", "Hc_up_Oe", "zeta",
        "m_rescale", "Hc0_Oe", "area0_Oe")]

    def as_dict(self) -> dict:
        return {n: getattr(self, n) for n, _ in self._fields_}


class LLGError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


# Exported symbols and their signatures: (restype, argtypes)
_vp, _dp, _fp, _i64 = C.c_void_p, C.POINTER(C.c_double), C.c_void_p, C.c_int64
SIGNATURES = {
    "llg_create_grid": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, C.c_int, C.c_int, C.c_double,
                                  C.c_int, C.c_uint, C.c_int, _vp]),
    "llg_destroy": (None, [_vp]),
    "llg_last_error": (C.c_char_p, []),
    "llg_set_stream": (C.c_int, [_vp, _vp]),
    "llg_set_material": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, _dp, C.c_double,
                                   C.c_double]),
    "llg_set_scaling": (C.c_int, [_vp, C.c_int, C.c_double, C.c_double, _dp]),
    "llg_set_sweep": (C.c_int, [_vp, C.c_double, C.c_double, C.c_double, C.c_double, C.c_double,
                                C.c_int]),
    "llg_set_engine": (C.c_int, [_vp, C.c_int]),
    "llg_set_cell_volume": (C.c_int, [_vp, C.c_double]),
    "llg_set_held_samples": (C.c_int, [_vp, _i64]),
    "llg_set_axis_dispersion": (C.c_int, [_vp, C.c_double]),
    "llg_gk_flow": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, C.c_int64, _vp]),
    "llg_get_axes": (C.c_int, [_vp, _vp]),
    "llg_set_tuning": (C.c_int, [_vp, C.c_int, _i64]),
    "llg_get_tuning": (C.c_int, [_vp, C.c_int, C.POINTER(C.c_int64)]),
    "llg_reset": (C.c_int, [_vp, C.c_uint32, C.c_int, C.c_uint32]),
    "llg_advance": (C.c_int, [_vp, _i64, _fp]),
    "llg_run_loops": (C.c_int, [_vp, C.c_uint32, C.c_int, C.c_uint32, _fp, C.POINTER(LoopStats)]),
    "llg_get_state": (C.c_int, [_vp, _fp, C.POINTER(C.c_int64)]),
    "llg_set_state": (C.c_int, [_vp, _fp, _i64]),
    "llg_sync": (C.c_int, [_vp, C.c_double]),
    "llg_num_cells": (_i64, [_vp]),
    "llg_num_samples": (_i64, [_vp]),
    "llg_steps_per_loop": (_i64, [_vp]),
    "llg_sample_every": (_i64, [_vp]),
    "llg_current_step": (_i64, [_vp]),
    "llg_active_engine": (C.c_int, [_vp]),
    "llg_get_coefficients": (C.c_int, [_vp, _dp]),
    "llg_sample_fields": (C.c_int, [_vp, _dp]),
    "llg_run_batch": (C.c_int, [C.POINTER(C.c_void_p), C.c_int, _i64, C.POINTER(C.c_void_p),
                                C.POINTER(C.c_int64)]),
    "llg_loop_area_grad": (C.c_int, [_vp, _i64, C.c_int, _dp, _i64, _dp, _dp]),
    "llg_autotune": (C.c_int, [_vp, _i64, C.POINTER(C.c_double)]),
    "llg_plain_advance_noalloc": (C.c_int, [_vp, _fp, C.c_int, C.c_uint32, C.c_uint32, _i64, _i64,
                                            _fp, _vp, C.POINTER(C.c_int)]),
    "llg_loop_stats_host": (C.c_int, [_fp, C.c_int, _i64, _dp, _i64, C.c_int, C.c_double,
                                      C.c_double, C.POINTER(LoopStats), _dp]),
    "llg_loop_moments": (C.c_int, [_fp, C.c_int, _i64, _dp, _dp]),
    "llg_loop_jackknife_terms": (C.c_int, [_fp, C.c_int, _i64, _dp, C.c_int, _dp, _i64, _dp]),
    "llg_loop_stats_from_sums": (C.c_int, [_dp, C.c_int, _i64, _dp, _i64, _dp, C.c_int, C.c_double,
                                           C.c_double, C.POINTER(LoopStats), _dp]),
    "llg_specific_loss_power": (C.c_int, [C.c_double, C.c_double, C.c_double, C.c_double, _dp]),
    "llg_measure_alu_peak": (C.c_int, [C.c_int, _dp]),
}

_lib = None


def load():
    """Load libllg.so and declare the ABI.  Raises ImportError when it has not been built."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "`python -c 'import __graft_entry__ as g; g.build()'`")
        lib = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def check(status: int):
    if status != 0:
        raise LLGError(status, load().llg_last_error().decode(errors="replace"))
