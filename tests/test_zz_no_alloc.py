"""mhd_diagnostics_static: the allocation-free diagnostics entry point.

It exists for callers that cannot call cudaMalloc (device memory already
owned by another allocator, or a loop that must avoid the implicit
synchronisation of allocation).  It must give the same answer as the
context-based mhd_diagnostics, on consecutive calls that reuse its static
device scratch.  This file is collected last on purpose.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

from paper_2402_05240_gb300 import inputs as I  # noqa: E402


@pytest.fixture(scope="module")
def mhd():
    from paper_2402_05240_gb300 import build
    build.build()
    from paper_2402_05240_gb300 import mhd as m
    return m


def test_static_diagnostics_match_context_version_on_consecutive_calls(mhd):
    n = (40, 28, 21)
    sim = mhd.Sim(*n)
    states = [I.turbulent_box(I.Box(*n), seed_v=s, seed_b=s + 1, kmax=4) for s in (101, 203)]
    for U0 in states:  # two calls in a row share (and overwrite) the static scratch
        U = torch.from_numpy(U0).cuda()
        ref_div, ref_tot = sim.diagnostics(U)
        m = ctypes.c_double(0)
        tot = (ctypes.c_double * 8)()
        code = mhd.LIB.mhd_diagnostics_static(ctypes.byref(sim.cfg), ctypes.c_void_p(U.data_ptr()),
                                              ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                              ctypes.byref(m), tot)
        assert code == mhd.MHD_OK
        assert abs(m.value - ref_div) <= 1e-12 * max(abs(ref_div), 1e-300)
        np.testing.assert_allclose(list(tot), ref_tot, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref_tot)))
    sim.close()


def _static_call(mhd, cfg, U):
    m = ctypes.c_double(0)
    tot = (ctypes.c_double * 8)()
    code = mhd.LIB.mhd_diagnostics_static(ctypes.byref(cfg), ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(m), tot)
    return code, m.value, list(tot)


def test_static_diagnostics_at_its_largest_grid(mhd):
    """512^3 cells (131072 partial blocks) fill the static scratch exactly;
    two calls in a row on different states match the context version."""
    n = 512
    N = n ** 3
    sim = mhd.Sim(n, n, n, precision="fp32_bulk")  # the smaller workspace; the diagnostics are FP64 either way
    gen = torch.Generator(device="cuda")
    U = torch.empty(8, n, n, n, dtype=torch.float64, device="cuda")
    for seed in (11, 12):
        gen.manual_seed(seed)
        U.uniform_(0.5, 1.5, generator=gen)
        U[1:4] -= 1.0  # momenta of both signs
        U[5:8] -= 1.0  # face fields of both signs, div B of order 1 / dx
        ref_div, ref_tot = sim.diagnostics(U)
        code, div, tot = _static_call(mhd, sim.cfg, U)
        assert code == mhd.MHD_OK
        assert abs(div - ref_div) <= 1e-12 * abs(ref_div)
        np.testing.assert_allclose(tot, ref_tot, rtol=1e-12, atol=1e-12 * np.max(np.abs(ref_tot)))
        # the sums also agree with torch's own FP64 sums of the fields
        np.testing.assert_allclose(tot, U.reshape(8, N).sum(dim=1).cpu().numpy(), rtol=1e-10,
                                   atol=1e-10 * N)
    sim.close()
    del U
    torch.cuda.empty_cache()


def test_static_diagnostics_rejects_grids_beyond_its_scratch(mhd):
    big = mhd.mhd_config(1024, 1024, 1024, 1e-3, 1e-3, 1e-3, 5 / 3, 0.4, 1, 0, 1e-20, 1e-20)
    U = torch.zeros(8, dtype=torch.float64, device="cuda")  # never read: the size check comes first
    m = ctypes.c_double(0)
    tot = (ctypes.c_double * 8)()
    code = mhd.LIB.mhd_diagnostics_static(ctypes.byref(big), ctypes.c_void_p(U.data_ptr()),
                                          ctypes.c_void_p(torch.cuda.current_stream().cuda_stream),
                                          ctypes.byref(m), tot)
    assert code == mhd.MHD_ERR_TOO_LARGE
    # the binding refuses the undersized buffer before the library sees it
    with pytest.raises(ValueError):
        mhd.mhd_diagnostics_static(big, U)
