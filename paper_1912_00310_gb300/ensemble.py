"""Ensembles split over processes (one per GPU): the loop observables of all realisations from
two small all-reduces (torch.distributed is the transport; the arithmetic is the library's).

Realisations are independent (the loop paragraph of arXiv:1912.00310 averages 88-250 of them per
loop), so each process runs its own share with disjoint noise keys and only the per-sample sums
and the four jackknife sums cross processes.
"""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib
from ._lib import LoopStats


def _dp(a: np.ndarray):
    return a.ctypes.data_as(C.POINTER(C.c_double))


def _allreduce_sum(values: np.ndarray, group=None) -> np.ndarray:
    """Sum of a float64 host array over the processes of the default (or given) group; the
    array itself when torch.distributed is not initialised."""
    import torch
    import torch.distributed as dist
    if not (dist.is_available() and dist.is_initialized()):
        return values
    backend = dist.get_backend(group)
    dev = "cuda" if backend == "nccl" else "cpu"
    t = torch.from_numpy(np.ascontiguousarray(values, dtype=np.float64)).to(dev)
    dist.all_reduce(t, op=dist.ReduceOp.SUM, group=group)
    return t.cpu().numpy()


def sample_moments(samples: np.ndarray, group=None):
    """(n_total, per-sample sum, per-sample sum of squares) of m_z over the realisations of every
    process; samples: this process's float32 host array [n_local][n_samples]."""
    L = _lib.load()
    s = np.ascontiguousarray(samples, dtype=np.float32)
    n_local, n = s.shape
    buf = np.zeros(2 * n + 1)
    _lib.check(L.llg_loop_moments(s.ctypes.data if n_local else None, n_local, n, _dp(buf[:n]),
                                  _dp(buf[n:2 * n])))
    buf[2 * n] = n_local
    tot = _allreduce_sum(buf, group)
    return int(round(tot[2 * n])), tot[:n], tot[n:2 * n]


def loop_stats(samples: np.ndarray, H: np.ndarray, k_turn: int, mode=1, zeta=1.0, delta=0.511,
               group=None) -> dict:
    """Loop observables (coercive field, area, jackknife standard errors, rescaled values) of the
    ensemble formed by every process's samples; over one process this equals
    llg_loop_stats_host.  Also returns the mean loop and its per-sample standard error."""
    L = _lib.load()
    s = np.ascontiguousarray(samples, dtype=np.float32)
    H = np.ascontiguousarray(H, dtype=np.float64)
    n_local, n = s.shape
    n_total, s1, s2 = sample_moments(s, group)
    jk = np.zeros(4)
    if n_total > 1:
        _lib.check(L.llg_loop_jackknife_terms(s.ctypes.data if n_local else None, n_local, n,
                                              _dp(s1), n_total, _dp(H), int(k_turn), _dp(jk)))
        jk = _allreduce_sum(jk, group)
    out = LoopStats()
    mean = np.zeros(n)
    _lib.check(L.llg_loop_stats_from_sums(_dp(s1), n_total, n, _dp(H), int(k_turn),
                                          _dp(jk) if n_total > 1 else None, mode, zeta, delta,
                                          C.byref(out), _dp(mean)))
    d = out.as_dict()
    d["n_real"] = n_total
    d["mean"] = mean
    if n_total > 1:
        var = np.maximum(0.0, s2 - s1 * s1 / n_total) / (n_total - 1)
        d["mean_se"] = np.sqrt(var / n_total)
    return d
