"""The allocation-free advance (llg_plain_advance_noalloc), called through the C ABI.

It serves callers that cannot allocate device memory (inside stream capture, under a foreign
allocator, in loops that cannot take an allocation's synchronisation).  It runs the same kernels
with the same arithmetic as the regular plain engine (llg_reset + llg_advance), only with its
scratch in a fixed library array, so two calls in a row must reproduce that engine on the same
seeds bitwise, samples included (stricter than the 1e-4 trajectory tolerance of the other parity
tests).  A request beyond the fixed scratch, and buffers that are not device memory of the
context's device, must be refused before anything is launched.  This file is collected last on
purpose.
"""
import ctypes as C

import numpy as np
import pytest

from workloads import MAGNETITE as M, ROD_DIMS

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def _grid(pkg, engine):
    g = pkg.Grid(*ROD_DIMS[4], a0=M["a0"], b=4)
    g.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    g.set_scaling(mode=1, Tc=M["Tc"])
    g.set_sweep(H_start=1500.0, H_turn=-1500.0, rate=1000.0, dt=10e-15, sample_dH=1.0)
    g.set_engine(engine)
    return g


def test_noalloc_matches_regular_plain_engine_over_two_calls():
    from paper_1912_00310_gb300 import build
    build.build()
    import paper_1912_00310_gb300 as pkg
    L = pkg.library()
    n_real, seed, off = 6, 4, 9
    first, second = 250, 180

    ref = _grid(pkg, pkg.ENGINE_PLAIN)
    ref.reset(seed=seed, n_real=n_real, real_offset=off)
    S_ref = torch.full((n_real, ref.n_samples), float("nan"), device="cuda")
    ref.advance(first, S_ref)
    ref.advance(second, S_ref)
    m_ref = torch.empty((n_real, ref.ncells, 3), dtype=torch.float32, device="cuda")
    ref.get_state(m_ref)
    ref.sync(120)

    g = _grid(pkg, pkg.ENGINE_PLAIN)  # host-side parameters only
    m = torch.zeros((n_real, g.ncells, 3), dtype=torch.float32, device="cuda")
    m[..., 2] = 1.0  # the +z start of llg_reset
    S = torch.full((n_real, g.n_samples), float("nan"), device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    status = C.c_int(-1)
    for step0, n in ((0, first), (first, second)):
        rc = L.llg_plain_advance_noalloc(g._h, C.c_void_p(m.data_ptr()), n_real, seed, off, step0,
                                         n, C.c_void_p(S.data_ptr()), stream, C.byref(status))
        assert rc == 0, L.llg_last_error()
        assert status.value == 0
    torch.cuda.synchronize()
    assert torch.equal(m, m_ref)  # same kernels, same arithmetic: bitwise
    k = (first + second) // g.sample_every
    assert k == 4
    assert not torch.isnan(S[:, 1:k + 1]).any()
    assert torch.equal(S[:, 1:k + 1], S_ref[:, 1:k + 1])
    assert np.allclose(np.linalg.norm(m.cpu().numpy(), axis=-1), 1.0, atol=1e-6)

    # a host buffer in place of device memory: refused, the device state untouched
    m_before = m.clone()
    host = np.zeros((n_real, g.ncells, 3), dtype=np.float32)
    rc = L.llg_plain_advance_noalloc(g._h, C.c_void_p(host.ctypes.data), n_real, seed, off, 0, 1,
                                     None, stream, None)
    assert rc == 1
    assert b"device memory" in L.llg_last_error()
    rc = L.llg_plain_advance_noalloc(g._h, C.c_void_p(m.data_ptr()), n_real, seed, off, 0, 1,
                                     C.c_void_p(host.ctypes.data), stream, None)
    assert rc == 1
    torch.cuda.synchronize()
    assert torch.equal(m, m_before)

    # beyond the fixed scratch: refused with a clear message, nothing launched
    big = pkg.Grid(64, 64, 64, a0=M["a0"], b=1)
    big.set_material(A0=M["A0"], Ms=M["Ms"], K0=M["K0"], alpha=M["alpha"], T=M["T"])
    big.set_sweep(H_start=0.0, H_turn=0.0, rate=0.0, dt=2e-15, sample_dH=1.0)
    rc = L.llg_plain_advance_noalloc(big._h, C.c_void_p(m.data_ptr()), 2, 0, 0, 0, 1, None,
                                     stream, None)
    assert rc == 1
    assert b"allocation-free scratch" in L.llg_last_error()
    for x in (ref, g, big):
        x.close()
