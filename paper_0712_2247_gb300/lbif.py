"""Thin ctypes binding of the C ABI in ``include/lbif.h``.

Argument marshalling only: every step of the method runs in the CUDA kernels of
``liblbif.so``. There is no CPU fallback; loading fails loudly when the library
is missing or when no CUDA device is present at call time.
"""
from __future__ import annotations

import ctypes
import os
from typing import Optional, Sequence

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbif.so")

LBIF_OK = 0
ERRORS = {
    -1: "LBIF_ERR_ARG", -2: "LBIF_ERR_NOMEM", -3: "LBIF_ERR_CUDA", -4: "LBIF_ERR_DIVERGED",
    -5: "LBIF_ERR_TIMEOUT", -6: "LBIF_ERR_UNSUPPORTED", -7: "LBIF_ERR_IO",
}
STORE_F32, STORE_F16 = 0, 1

# every function the header declares, with (restype, argtypes)
_vp, _i32, _i64, _f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)


class Grid(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("nz", ctypes.c_int32)]


class Walls(ctypes.Structure):
    _fields_ = [("z", ctypes.c_int32)]


class Force(ctypes.Structure):
    _fields_ = [("body", ctypes.c_double * 3), ("hs", ctypes.c_int32), ("coupling", ctypes.c_int32),
                ("regularize", ctypes.c_int32), ("g2_form", ctypes.c_int32), ("tail", ctypes.c_int32),
                ("eps", ctypes.c_double), ("rcut", ctypes.c_double), ("c2", ctypes.c_int32),
                ("shifted", ctypes.c_int32)]


class Opts(ctypes.Structure):
    _fields_ = [("storage", ctypes.c_int32), ("seed", ctypes.c_uint64), ("noise", ctypes.c_double),
                ("stream", ctypes.c_void_p), ("inplace", ctypes.c_int32)]


SIGNATURES = {
    "lbif_create": (_i32, [ctypes.POINTER(_vp), Grid, _f64, _f64, _f64, Walls,
                           ctypes.POINTER(Force), ctypes.POINTER(Opts)]),
    "lbif_step": (_i32, [_vp, _i64]),
    "lbif_step_profiled": (_i32, [_vp, _i64, _pd, ctypes.POINTER(_i64), _i32]),
    "lbif_moments": (_i32, [_vp, _vp, _vp, _vp, _i32]),
    "lbif_forces": (_i32, [_vp, _vp, _i32]),
    "lbif_set_fields": (_i32, [_vp, _vp, _vp, _i32]),
    "lbif_profiles": (_i32, [_vp, _pd, _pd, _pd]),
    "lbif_residual": (_i32, [_vp, _pd, _pd, _pd]),
    "lbif_time": (_i32, [_vp, ctypes.POINTER(_i64)]),
    "lbif_status": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "lbif_save": (_i32, [_vp, ctypes.c_char_p]),
    "lbif_load": (_i32, [_vp, ctypes.c_char_p]),
    "lbif_batch_create": (_i32, [ctypes.POINTER(_vp), _i32, ctypes.POINTER(_i32), _pd, _pd, _pd, _f64,
                                 _i32, _i32, ctypes.POINTER(Force), ctypes.POINTER(Opts)]),
    "lbif_batch_info": (_i32, [_vp, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i64)]),
    "lbif_batch_seed": (_i32, [_vp, _vp, _vp, _i32]),
    "lbif_batch_run": (_i32, [_vp, _f64, _i64, _i32, _i32, ctypes.POINTER(_i64), _pd]),
    "lbif_batch_profiles": (_i32, [_vp, _pd, _pd, _i32]),
    "lbif_autotune": (_i32, [_vp, _i32, ctypes.POINTER(_i32), ctypes.POINTER(_i32), ctypes.POINTER(_i32)]),
    "lbif_set_fused": (_i32, [_vp, _i32]),
    "lbif_get_shapes": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "lbif_set_shapes": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "lbif_get_fused": (_i32, [_vp, ctypes.POINTER(_i32)]),
    "lbif_selftest_wait": (_i32, [_i64, ctypes.POINTER(_i32)]),
    "lbif_field_profiles_noalloc": (_i32, [_vp, _vp, _i32, _i32, _i32, _pd, _pd, _pd, _vp]),
    "lbif_noalloc_last_error": (ctypes.c_char_p, []),
    "lbif_destroy": (_i32, [_vp]),
    "lbif_last_error": (ctypes.c_char_p, [_vp]),
}

_lib = None


def load_library(path: str = LIB_PATH) -> ctypes.CDLL:
    """Load ``liblbif.so`` (built by ``paper_0712_2247_gb300.build``); raises if absent."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(path):
        raise RuntimeError(f"lbif: CUDA library {path} is missing; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class LbifError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


def _ptr(a, n: Optional[int] = None) -> Optional[int]:
    """Device pointer of a torch tensor or host pointer of a numpy array. The
    array must be contiguous float32 and, when n is given, hold exactly n
    elements (the library reads or writes that many); anything else raises
    here, before the library sees the pointer."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        if a.dtype != np.float32 or not a.flags.c_contiguous:
            raise TypeError("lbif: arrays must be contiguous float32")
        size, p = a.size, a.ctypes.data
    else:
        if str(getattr(a, "dtype", "")) != "torch.float32" or not a.is_contiguous():
            raise TypeError("lbif: tensors must be contiguous torch.float32")
        size, p = a.numel(), a.data_ptr()
    if n is not None and size != n:
        raise ValueError(f"lbif: array of {size} elements where {n} are needed")
    return p


def _on_device(*arrays) -> int:
    """1 when the given arrays are CUDA tensors, 0 when they are host arrays;
    host and device arrays in one call raise."""
    where = {0 if isinstance(a, np.ndarray) else int(a.is_cuda) for a in arrays if a is not None}
    if len(where) > 1:
        raise ValueError("lbif: host and device arrays mixed in one call")
    return where.pop() if where else 0


def selftest_wait(polls: int):
    """Run the bounded device wait on a barrier nothing completes; returns
    (return code, timed_out)."""
    lib = load_library()
    t = ctypes.c_int32(0)
    rc = lib.lbif_selftest_wait(int(polls), ctypes.byref(t))
    return rc, bool(t.value)


class Slit:
    """One slit (or periodic box) advanced on the GPU through the C ABI.

    Arrays are (nz, ny, nx) with x fastest; host arrays are numpy float32, device
    arrays are contiguous torch float32 CUDA tensors.
    """

    def __init__(self, nx: int, ny: int, nz: int, sigma: float, eta: float, tau: float, *,
                 periodic_z: bool = False, body: Sequence[float] = (0.0, 0.0, 0.0), hs: bool = True,
                 coupling: bool = True, regularize: bool = True, g2_form: int = 0,
                 tail: bool = False, eps: float = 1.0, rcut: float = 2.5, storage: int = STORE_F32,
                 seed: int = 0, noise: float = 1e-3, stream: Optional[int] = None, c2: bool = False,
                 inplace: bool = False, shifted: bool = False):
        self._lib = load_library()
        f = Force((ctypes.c_double * 3)(*[float(b) for b in body]), int(hs), int(coupling),
                  int(regularize), int(g2_form), int(tail), float(eps), float(rcut), int(c2), int(shifted))
        o = Opts(int(storage), int(seed) & 0xFFFFFFFFFFFFFFFF, float(noise), stream, int(inplace))
        h = _vp()
        rc = self._lib.lbif_create(ctypes.byref(h), Grid(nx, ny, nz), float(sigma), float(eta),
                                   float(tau), Walls(1 if periodic_z else 0), ctypes.byref(f),
                                   ctypes.byref(o))
        if rc != LBIF_OK:
            raise LbifError(rc, self._lib.lbif_last_error(None).decode())
        self._h = h
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self.sigma, self.eta, self.tau = sigma, eta, tau
        self.n0 = 6.0 * eta / (np.pi * sigma ** 3)

    # -- plumbing ---------------------------------------------------------
    def _check(self, rc: int, allow_diverged: bool = False):
        if rc != LBIF_OK and not (allow_diverged and rc == -4):
            raise LbifError(rc, self._lib.lbif_last_error(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            self._lib.lbif_destroy(self._h)
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

    # -- calls ------------------------------------------------------------
    def step(self, nsteps: int = 1):
        self._check(self._lib.lbif_step(self._h, int(nsteps)))

    KERNEL_CLASSES = ("moments", "ball_g2", "tail", "force", "collide_stream")

    def step_profiled(self, nsteps: int):
        """Advance nsteps and return ({class: total ms}, {class: launches})."""
        ms = (ctypes.c_double * 5)()
        nl = (ctypes.c_int64 * 5)()
        self._check(self._lib.lbif_step_profiled(self._h, int(nsteps), ms, nl, 5))
        return (dict(zip(self.KERNEL_CLASSES, ms[:])), dict(zip(self.KERNEL_CLASSES, nl[:])))

    def autotune(self, trials: int = 3):
        """Pick the fastest launch shapes on the current state; returns (ball CTA
        target, force tile-group edge, ball staging: 1 tensor-memory accelerator,
        0 plain loads). The state is unchanged and the results are bit-identical."""
        b, g, st = ctypes.c_int32(), ctypes.c_int32(), ctypes.c_int32()
        self._check(self._lib.lbif_autotune(self._h, int(trials), ctypes.byref(b), ctypes.byref(g),
                                            ctypes.byref(st)))
        return b.value, g.value, st.value

    def shapes(self) -> dict:
        """The launch shapes in use (see lbif_get_shapes)."""
        v = (_i32 * 5)()
        self._check(self._lib.lbif_get_shapes(self._h, v))
        return {"ball_ctas": v[0], "force_group": v[1], "ball_staging": "tma" if v[2] else "loads",
                "pull_lz": v[3], "pull_gathers": self.PULL_GATHERS[v[4]]}

    PULL_GATHERS = ("loads", "prefetch", "tma")

    def set_shapes(self, ball_ctas=0, force_group=0, ball_staging="loads", pull_lz=0, pull_gathers="loads"):
        """Set the launch shapes (see lbif_set_shapes); no shape changes the
        arithmetic."""
        v = (_i32 * 5)(int(ball_ctas), int(force_group), 1 if ball_staging == "tma" else 0, int(pull_lz),
                       self.PULL_GATHERS.index(pull_gathers))
        self._check(self._lib.lbif_set_shapes(self._h, v))

    def set_fused(self, on: bool):
        """Every step is one pull pass (collision, streaming and the next
        moments); on=True changes nothing, on=False raises LbifError (the
        two-pass step is retired)."""
        self._check(self._lib.lbif_set_fused(self._h, 1 if on else 0))

    @property
    def fused(self) -> bool:
        v = ctypes.c_int32()
        self._check(self._lib.lbif_get_fused(self._h, ctypes.byref(v)))
        return bool(v.value)

    def moments(self, rho=None, u=None, pressure=None, allow_diverged=False):
        """Fill caller-owned buffers; with no buffers, return numpy (rho, u) arrays."""
        if rho is None and u is None and pressure is None:
            rho = np.empty(self.shape, np.float32)
            u = np.empty((3,) + self.shape, np.float32)
            self._check(self._lib.lbif_moments(self._h, _ptr(rho), _ptr(u), None, 0), allow_diverged)
            return rho, u
        n = self.grid_nodes
        dev = _on_device(rho, u, pressure)
        self._check(self._lib.lbif_moments(self._h, _ptr(rho, n), _ptr(u, 3 * n), _ptr(pressure, n), dev),
                    allow_diverged)
        return rho, u, pressure

    def pressure(self) -> np.ndarray:
        p = np.empty(self.shape, np.float32)
        self._check(self._lib.lbif_moments(self._h, None, None, _ptr(p), 0))
        return p

    def forces(self, out=None) -> np.ndarray:
        """Total force density divided by n0, shape (3, nz, ny, nx)."""
        F = np.empty((3,) + self.shape, np.float32) if out is None else out
        self._check(self._lib.lbif_forces(self._h, _ptr(F, 3 * self.grid_nodes), _on_device(F)))
        return F

    def set_fields(self, rho, u=None):
        dev = _on_device(rho, u)
        self._check(self._lib.lbif_set_fields(self._h, _ptr(rho, self.grid_nodes), _ptr(u, 3 * self.grid_nodes), dev))

    @property
    def grid_nodes(self) -> int:
        """nx ny nz: the element count of one field array (an ensemble's gap
        planes included)."""
        nz, ny, nx = self.shape
        return nx * ny * nz

    def profiles(self, allow_diverged=False):
        nz = self.shape[0]
        n = np.empty(nz)
        ux = np.empty(nz)
        tot = np.empty(4)
        pd = lambda a: a.ctypes.data_as(_pd)
        self._check(self._lib.lbif_profiles(self._h, pd(n), pd(ux), pd(tot)), allow_diverged)
        return n, ux, tot

    def residual(self):
        r, m = ctypes.c_double(), ctypes.c_double()
        mom = (ctypes.c_double * 3)()
        self._check(self._lib.lbif_residual(self._h, ctypes.byref(r), ctypes.byref(m), mom))
        return r.value, m.value, np.array(mom[:])

    @property
    def t(self) -> int:
        v = ctypes.c_int64()
        self._check(self._lib.lbif_time(self._h, ctypes.byref(v)))
        return v.value

    def status(self) -> int:
        v = ctypes.c_int32()
        self._check(self._lib.lbif_status(self._h, ctypes.byref(v)))
        return v.value

    def save(self, path: str):
        self._check(self._lib.lbif_save(self._h, path.encode()))

    def load(self, path: str):
        self._check(self._lib.lbif_load(self._h, path.encode()))


class Ensemble(Slit):
    """Many slits (widths H, packing fractions eta, forces F along x, relaxation
    times tau) advanced together through the C ABI; one stacked grid on the GPU.
    The populations live in place by default: each slit's storage ring holds
    only its own planes (the two-buffer layout also stores the planes between
    the slits), which made 256 slits of 32 x 32 x H 20 % faster with FP16
    storage and 9 % with FP32; results are identical either way."""

    def __init__(self, H, eta, F, tau, sigma: float, nx: int = 32, ny: int = 32, *,
                 hs: bool = True, coupling: bool = True, regularize: bool = True,
                 g2_form: int = 0, storage: int = STORE_F16, seed: int = 0, noise: float = 1e-3,
                 stream: Optional[int] = None, inplace: bool = True):
        self._lib = load_library()
        H = np.ascontiguousarray(H, dtype=np.int32)
        eta = np.ascontiguousarray(eta, dtype=np.float64)
        F = np.ascontiguousarray(F, dtype=np.float64)
        tau = np.ascontiguousarray(tau, dtype=np.float64)
        n = len(H)
        assert len(eta) == len(F) == len(tau) == n
        f = Force((ctypes.c_double * 3)(0.0, 0.0, 0.0), int(hs), int(coupling), int(regularize),
                  int(g2_form), 0, 1.0, 2.5)
        o = Opts(int(storage), int(seed) & 0xFFFFFFFFFFFFFFFF, float(noise), stream, int(inplace))
        h = _vp()
        pd = lambda a: a.ctypes.data_as(_pd)
        rc = self._lib.lbif_batch_create(ctypes.byref(h), n, H.ctypes.data_as(ctypes.POINTER(_i32)),
                                         pd(eta), pd(F), pd(tau), float(sigma), int(nx), int(ny),
                                         ctypes.byref(f), ctypes.byref(o))
        if rc != LBIF_OK:
            raise LbifError(rc, self._lib.lbif_last_error(None).decode())
        self._h = h
        self.H, self.eta_s, self.F_s, self.tau_s = H, eta, F, tau
        self.nslits = n
        self.sigma = sigma
        self.n0_s = 6.0 * eta / (np.pi * sigma ** 3)
        zlo = np.zeros(n, np.int32)
        nodes = ctypes.c_int64()
        self._check(self._lib.lbif_batch_info(self._h, None, zlo.ctypes.data_as(ctypes.POINTER(_i32)),
                                              ctypes.byref(nodes)))
        self.zlo = zlo
        self.nodes = nodes.value
        nz = int(zlo[-1] + H[-1])
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz

    def seed(self, n_z, ux_z=None):
        """Set every slit to the equilibrium of profiles n_z[s, j], ux_z[s, j] (j < H[s])."""
        n_z = np.ascontiguousarray(n_z, dtype=np.float32)
        hmax = n_z.shape[1]
        ux = None if ux_z is None else np.ascontiguousarray(ux_z, dtype=np.float32)
        self._check(self._lib.lbif_batch_seed(self._h, n_z.ctypes.data,
                                              None if ux is None else ux.ctypes.data, hmax))

    def run(self, tol: float = 1e-8, max_steps: int = 100000, check_every: int = 100,
            patience: int = 0, return_residual: bool = False):
        """Run to steady state; returns steps taken per slit (-1: not within max_steps,
        -2: diverged, -3: stalled above tol for `patience` checks) [and the best residual]."""
        out = np.zeros(self.nslits, np.int64)
        res = np.zeros(self.nslits)
        self._check(self._lib.lbif_batch_run(self._h, float(tol), int(max_steps), int(check_every),
                                             int(patience), out.ctypes.data_as(ctypes.POINTER(_i64)),
                                             res.ctypes.data_as(_pd)))
        return (out, res) if return_residual else out

    def slit_profiles(self, hmax: Optional[int] = None):
        hmax = int(hmax or self.H.max())
        n = np.zeros((self.nslits, hmax))
        ux = np.zeros((self.nslits, hmax))
        pd = lambda a: a.ctypes.data_as(_pd)
        self._check(self._lib.lbif_batch_profiles(self._h, pd(n), pd(ux), hmax), True)
        return n, ux


