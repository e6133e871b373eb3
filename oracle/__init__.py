"""FP64 CPU oracle for the inhomogeneous hard-sphere lattice Boltzmann step.

TEST INFRASTRUCTURE ONLY: the test-suite, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` are the only callers. The CUDA product path
never imports this package, and this package never imports the product.

The arithmetic lives in ``lbif_oracle.c`` (plain FP64 loops, one per step of
the method as the paper orders it); this module only compiles it with gcc and
marshals numpy arrays through ctypes. ``mlp.py`` holds the numpy FP64 oracle of
the warm-start network.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "lbif_oracle.c")
_LIB = os.path.join(_HERE, "liblbif_oracle.so")
_lock = threading.Lock()
_lib = None

NV = 19


def build(force: bool = False) -> str:
    """Compile the oracle into ``oracle/liblbif_oracle.so`` (gcc, OpenMP)."""
    if not force and os.path.exists(_LIB) and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC):
        return _LIB
    tmp = _LIB + ".%d.tmp" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-std=c11", "-D_DEFAULT_SOURCE",
           "-o", tmp, _SRC, "-lm"]
    subprocess.check_call(cmd)
    os.replace(tmp, _LIB)
    return _LIB


_D = ctypes.POINTER(ctypes.c_double)
_I = ctypes.POINTER(ctypes.c_int)


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        build()
        lib = ctypes.CDLL(_LIB)
        vp = ctypes.c_void_p
        i32, f64, i64, u64 = ctypes.c_int, ctypes.c_double, ctypes.c_int64, ctypes.c_uint64
        sigs = {
            "or_lattice": (None, [_I, _D]),
            "or_sphere_rule": (None, [_D, _D]),
            "or_g2": (f64, [f64, i32]),
            "or_ball_count": (i32, [i32]),
            "or_threads": (i32, []),
            "or_set_threads": (None, [i32]),
            "or_coarse_density": (None, [i32, i32, i32, i32, i32, _D, _D]),
            "or_equilibrium": (None, [f64, _D, _D]),
            "or_collide_node": (None, [_D, _D, f64, _D]),
            "or_create": (vp, [i32, i32, i32, i32, i32, f64, f64, _D, i32, i32, i32, i32, i32,
                               f64, f64]),
            "or_destroy": (None, [vp]),
            "or_n0": (f64, [vp]),
            "or_time": (ctypes.c_long, [vp]),
            "or_init_noise": (None, [vp, u64, f64, i64]),
            "or_init_fields": (None, [vp, _D, _D, _D, _D]),
            "or_step": (None, [vp, ctypes.c_long]),
            "or_step_lagged": (None, [vp, ctypes.c_long]),
            "or_set_c2": (None, [vp, ctypes.c_int]),
            "or_c2_field": (None, [vp, _D]),
            "or_moments": (None, [vp, _D, _D, _D, _D, _D]),
            "or_forces": (None, [vp, _D, _D, _D, _D]),
            "or_profiles": (None, [vp, _D, _D]),
            "or_totals": (None, [vp, _D]),
            "or_hs_force_fields": (None, [i32, i32, i32, i32, i32, i32, i32, i32, _D, _D, _D,
                                          _D, _D, _D, _D, _D, _D]),
            "or_tail_force_field": (None, [i32, i32, i32, i32, i32, f64, f64, _D, _D, _D, _D]),
            "or_step_shifted": (i32, [vp, ctypes.c_long]),
            "or_get_pops": (None, [vp, _D]),
            "or_set_pops": (None, [vp, _D]),
        }
        for name, (res, args) in sigs.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_D)


def _f64(a, n=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if n is not None:
        assert a.size == n
    return a


# --------------------------------------------------------------------------
# tables and closures
# --------------------------------------------------------------------------
def lattice():
    """D3Q19 velocities (19,3) int and weights (19,)."""
    lib = _load()
    c = np.zeros(NV * 3, dtype=np.int32)
    w = np.zeros(NV)
    lib.or_lattice(c.ctypes.data_as(_I), _p(w))
    return c.reshape(NV, 3), w


def sphere_rule():
    """18-point sphere quadrature: unit directions (18,3) and weights (18,)."""
    lib = _load()
    d = np.zeros(18 * 3)
    w = np.zeros(18)
    lib.or_sphere_rule(_p(d), _p(w))
    return d.reshape(18, 3), w


def g2(eta: float, form: int = 0) -> float:
    return _load().or_g2(float(eta), int(form))


def ball_count(sigma: int) -> int:
    return _load().or_ball_count(int(sigma))


def threads() -> int:
    """Threads the oracle's parallel loops run on."""
    return _load().or_threads()


def set_threads(n: int) -> None:
    """Run the oracle's parallel loops on n threads from now on."""
    _load().or_set_threads(int(n))


def equilibrium(n: float, u) -> np.ndarray:
    u = _f64(u, 3)
    out = np.zeros(NV)
    _load().or_equilibrium(float(n), _p(u), _p(out))
    return out


def collide_node(f, F, tau: float) -> np.ndarray:
    f = _f64(f, NV)
    F = _f64(F, 3)
    out = np.zeros(NV)
    _load().or_collide_node(_p(f), _p(F), float(tau), _p(out))
    return out


def coarse_density(n: np.ndarray, sigma: int, zper: bool) -> np.ndarray:
    """Ball average of a (nz, ny, nx) field."""
    nz, ny, nx = n.shape
    a = _f64(n)
    out = np.zeros_like(a)
    _load().or_coarse_density(nx, ny, nz, int(zper), int(sigma), _p(a), _p(out))
    return out


def hs_force(n, sigma: int, zper: bool, u=None, coupling=True, regularize=True, g2form=0):
    """Hard-sphere force (3, nz, ny, nx), g2 field and collisional pressure of given fields."""
    nz, ny, nx = n.shape
    N = n.size
    a = _f64(n)
    if u is None:
        ux = uy = uz = None
    else:
        ux, uy, uz = (_f64(u[k], N) for k in range(3))
    F = np.zeros((3,) + n.shape)
    G = np.zeros(n.shape)
    pc = np.zeros(n.shape)
    _load().or_hs_force_fields(nx, ny, nz, int(zper), int(sigma), int(coupling), int(regularize),
                               int(g2form), _p(a), _p(ux), _p(uy), _p(uz), _p(F[0]), _p(F[1]),
                               _p(F[2]), _p(G), _p(pc))
    return F, G, pc


def tail_force(n, sigma: int, zper: bool, eps=1.0, rcut=2.5):
    nz, ny, nx = n.shape
    a = _f64(n)
    F = np.zeros((3,) + n.shape)
    _load().or_tail_force_field(nx, ny, nz, int(zper), int(sigma), float(eps), float(rcut),
                                _p(a), _p(F[0]), _p(F[1]), _p(F[2]))
    return F


# --------------------------------------------------------------------------
# time-stepping state
# --------------------------------------------------------------------------
class Oracle:
    """FP64 slit (or periodic box) advanced by the plain two-array scheme.

    Fields are returned with shape (nz, ny, nx), x fastest, matching the
    device layout idx = (z*ny + y)*nx + x.
    """

    def __init__(self, nx, ny, nz, sigma, eta, tau, *, zper=False, body=(0.0, 0.0, 0.0),
                 hs=True, coupling=True, regularize=True, g2form=0, tail=False, eps=1.0,
                 rcut=2.5, seed=None, noise=1e-3, offset=0, c2=False):
        lib = _load()
        b = _f64(body, 3)
        self._lib = lib
        self.shape = (nz, ny, nx)
        self.N = nx * ny * nz
        self._h = lib.or_create(nx, ny, nz, int(zper), int(sigma), float(eta), float(tau), _p(b),
                                int(hs), int(coupling), int(regularize), int(g2form), int(tail),
                                float(eps), float(rcut))
        if not self._h:
            raise ValueError("oracle: invalid parameters")
        if seed is not None:
            lib.or_init_noise(self._h, int(seed) & 0xFFFFFFFFFFFFFFFF, float(noise), int(offset))
        if c2:
            lib.or_set_c2(self._h, 1)

    def c2_field(self):
        """The energy source of Eq. C2eq (constant T) of the current state."""
        out = np.zeros(self.shape)
        self._lib.or_c2_field(self._h, _p(out))
        return out

    def close(self):
        if self._h:
            self._lib.or_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def n0(self) -> float:
        return self._lib.or_n0(self._h)

    @property
    def t(self) -> int:
        return self._lib.or_time(self._h)

    def init_fields(self, n, u=None):
        a = _f64(n, self.N)
        if u is None:
            ux = uy = uz = None
        else:
            ux, uy, uz = (_f64(u[k], self.N) for k in range(3))
        self._lib.or_init_fields(self._h, _p(a), _p(ux), _p(uy), _p(uz))

    def step(self, nsteps: int = 1, lagged: bool = False, shifted: bool = False):
        """Plain steps, steps of the lagged-force variant (the force of the
        previous step's moments drives the collision), or steps with the
        velocity-shifted second-order forcing (the force from the unshifted
        moments; the equilibrium at (j + F/2)/n)."""
        if shifted:
            if self._lib.or_step_shifted(self._h, int(nsteps)) != 0:
                raise ValueError("oracle: the shifted forcing does not add the energy source")
            return
        (self._lib.or_step_lagged if lagged else self._lib.or_step)(self._h, int(nsteps))

    def moments(self, pressure: bool = False):
        n = np.zeros(self.shape)
        u = np.zeros((3,) + self.shape)
        p = np.zeros(self.shape) if pressure else None
        self._lib.or_moments(self._h, _p(n), _p(u[0]), _p(u[1]), _p(u[2]), _p(p))
        return (n, u, p) if pressure else (n, u)

    def forces(self):
        F = np.zeros((3,) + self.shape)
        G = np.zeros(self.shape)
        self._lib.or_forces(self._h, _p(F[0]), _p(F[1]), _p(F[2]), _p(G))
        return F, G

    def profiles(self):
        nz = self.shape[0]
        a = np.zeros(nz)
        b = np.zeros(nz)
        self._lib.or_profiles(self._h, _p(a), _p(b))
        return a, b

    def totals(self):
        out = np.zeros(4)
        self._lib.or_totals(self._h, _p(out))
        return out

    def populations(self) -> np.ndarray:
        """Copy of the populations, shape (19, nz, ny, nx)."""
        f = np.zeros((NV,) + self.shape)
        self._lib.or_get_pops(self._h, _p(f))
        return f

    def set_populations(self, f):
        """Replace the populations (shape (19, nz, ny, nx)); the step count is kept."""
        self._lib.or_set_pops(self._h, _p(_f64(f, NV * self.N)))
