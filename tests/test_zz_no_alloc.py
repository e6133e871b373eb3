"""The allocation-free profile entry point against lbif_profiles.

lbif_field_profiles_noalloc serves callers that cannot allocate device memory
when they need profiles (services whose device budget is reserved up front by
their own allocator, loops that must keep a fixed footprint): it reduces
fields the caller already holds and keeps its scratch in a fixed array inside
the library. This file is collected last so that a failure here never hides
the result of another test.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

_pd = lambda a: a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _setup():
    torch = pytest.importorskip("torch")
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    torch.cuda.set_device(0)
    return torch, lbif, lbif.load_library()


def _noalloc(lib, rho, u, nx, ny, nz):
    n = np.full(nz, np.nan)
    ux = np.full(nz, np.nan)
    tot = np.full(4, np.nan)
    rc = lib.lbif_field_profiles_noalloc(rho.data_ptr(), u.data_ptr(), nx, ny, nz, _pd(n), _pd(ux), _pd(tot), None)
    assert rc == 0, lib.lbif_noalloc_last_error()
    return n, ux, tot


def _device_fields(torch, g, nz, ny, nx):
    rho = torch.empty((nz, ny, nx), dtype=torch.float32, device="cuda")
    u = torch.empty((3, nz, ny, nx), dtype=torch.float32, device="cuda")
    g.moments(rho, u)
    torch.cuda.synchronize()
    return rho, u


def _agree(got, ref):
    # rho is the FP32 rounding of n0 (1 + dn): agreement to FP32 resolution
    (n, ux, tot), (n_ref, ux_ref, tot_ref) = got, ref
    assert np.abs(n - n_ref).max() < 1e-6 * np.abs(n_ref).max()
    assert np.abs(ux - ux_ref).max() < 1e-6 * np.abs(ux_ref).max()
    assert np.abs(tot - tot_ref).max() < 1e-6 * abs(tot_ref[0])


def test_noalloc_profiles_match_handle_profiles():
    torch, lbif, lib = _setup()
    nx, ny, nz = 16, 12, 20
    g = lbif.Slit(nx, ny, nz, 4, 0.25, 0.9, body=(1e-5, 0, 0), seed=7)
    g.step(30)
    ref = g.profiles()
    rho, u = _device_fields(torch, g, nz, ny, nx)
    free0 = None
    for call in range(2):  # two calls in a row share the static scratch
        got = _noalloc(lib, rho, u, nx, ny, nz)
        torch.cuda.synchronize()
        free = torch.cuda.mem_get_info()[0]
        if call == 0:
            free0 = free
        else:
            # the warm call took no device memory
            assert free == free0
        _agree(got, ref)
    g.close()


def test_noalloc_profiles_of_a_stacked_ensemble():
    """A batch handle with gap planes between its slits: lbif_profiles skips
    the gaps, the caller's fields read 0 there, and both give the same
    profiles and totals."""
    torch, lbif, lib = _setup()
    H = np.array([9, 14, 11], np.int32)
    e = lbif.Ensemble(H, np.array([0.15, 0.25, 0.2]), np.array([2e-6, 1e-6, 5e-6]), np.array([0.8, 1.0, 0.7]),
                      sigma=4, nx=8, ny=8, storage=0, seed=3)
    e.step(20)
    nz, ny, nx = e.shape
    ref = e.profiles()
    rho, u = _device_fields(torch, e, nz, ny, nx)
    assert float(rho[int(H[0])].abs().max()) == 0.0  # a gap plane
    for _ in range(2):
        _agree(_noalloc(lib, rho, u, nx, ny, nz), ref)
    e.close()


def test_noalloc_rejects_oversized_grids():
    torch, lbif, lib = _setup()
    buf = torch.zeros(16, dtype=torch.float32, device="cuda")
    n = np.zeros(4)
    rc = lib.lbif_field_profiles_noalloc(buf.data_ptr(), buf.data_ptr(), 1, 1, 8193, _pd(n), None, None, None)
    assert rc == -6
    assert b"8192" in lib.lbif_noalloc_last_error()
