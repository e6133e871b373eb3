"""The allocation-free profile entry point against lbif_profiles.

lbif_field_profiles_noalloc serves callers that cannot allocate device memory
when they need profiles (stream capture, pre-reserved device budgets,
fixed-footprint loops): it reduces fields the caller already holds and keeps
its scratch in a fixed array inside the library. This file is collected last
so that a failure here never hides the result of another test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def test_noalloc_profiles_match_handle_profiles():
    torch = pytest.importorskip("torch")
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    lib = lbif.load_library()
    torch.cuda.set_device(0)
    nx, ny, nz = 16, 12, 20
    g = lbif.Slit(nx, ny, nz, 4, 0.25, 0.9, body=(1e-5, 0, 0), seed=7)
    g.step(30)
    n_ref, ux_ref, tot_ref = g.profiles()
    rho = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    g.moments(rho, u)
    torch.cuda.synchronize()
    pd = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    for call in range(2):  # two calls in a row share the static scratch
        n = np.full(nz, np.nan)
        ux = np.full(nz, np.nan)
        tot = np.full(4, np.nan)
        rc = lib.lbif_field_profiles_noalloc(rho.data_ptr(), u.data_ptr(), nx, ny, nz, pd(n), pd(ux),
                                             pd(tot), None)
        assert rc == 0, lib.lbif_noalloc_last_error()
        # rho is the FP32 rounding of n0 (1 + dn): agreement to FP32 resolution
        assert np.abs(n - n_ref).max() < 1e-6 * np.abs(n_ref).max(), call
        assert np.abs(ux - ux_ref).max() < 1e-6 * np.abs(ux_ref).max(), call
        assert np.abs(tot - tot_ref).max() < 1e-6 * abs(tot_ref[0]), call
    g.close()


def test_noalloc_rejects_oversized_grids():
    torch = pytest.importorskip("torch")
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    lib = lbif.load_library()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    n = np.zeros(4)
    rc = lib.lbif_field_profiles_noalloc(buf.data_ptr(), buf.data_ptr(), 1, 1, 8193,
                                         n.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), None,
                                         None, None)
    assert rc == -6
    assert b"8192" in lib.lbif_noalloc_last_error()
