"""Host-side checks of the C-ABI library: it builds for sm_103a, loads, exports
every symbol that include/*.h declares, and rejects bad arguments before any
device work (no GPU needed for any of these)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    return lbif.load_library()


def _declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(lbif_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return sorted(names)


def test_headers_declare_the_boundary():
    names = _declared_symbols()
    for core in ("lbif_create", "lbif_step", "lbif_moments", "lbif_destroy"):
        assert core in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_0712_2247_gb300 import lbif

    import importlib

    declared = set(_declared_symbols())
    bound = set(lbif.SIGNATURES)
    for mod in ("batch", "mlp"):
        try:
            m = importlib.import_module("paper_0712_2247_gb300." + mod)
        except ImportError:
            continue
        bound |= set(getattr(m, "SIGNATURES", {}))
    assert declared <= bound, sorted(declared - bound)


def _create(lib, nx=8, ny=8, nz=8, sigma=4.0, eta=0.3, tau=1.0, zbc=0, storage=0, noise=1e-3, inplace=0):
    from paper_0712_2247_gb300 import lbif

    h = ctypes.c_void_p()
    f = lbif.Force((ctypes.c_double * 3)(0, 0, 0), 1, 1, 1, 0, 0, 1.0, 2.5)
    o = lbif.Opts(storage, 0, noise, None, inplace)
    rc = lib.lbif_create(ctypes.byref(h), lbif.Grid(nx, ny, nz), sigma, eta, tau, lbif.Walls(zbc),
                         ctypes.byref(f), ctypes.byref(o))
    return rc, h


@pytest.mark.parametrize("kw,code", [
    (dict(sigma=3.0), -6), (dict(sigma=4.5), -6), (dict(sigma=26.0), -6), (dict(sigma=0.0), -6),
    (dict(tau=0.5), -1), (dict(eta=0.0), -1), (dict(eta=1.0), -1), (dict(nx=0), -1),
    (dict(zbc=7), -1), (dict(storage=5), -1), (dict(noise=-1.0), -1),
    (dict(ny=-3), -1), (dict(nz=0), -1),
    # padded grid beyond 32-bit node indices: refused before any allocation
    (dict(nx=2048, ny=2048, nz=1024), -6),
    # in place: 19 x 253 M ring nodes exceed 32-bit element offsets
    (dict(nx=1024, ny=1024, nz=240, inplace=1), -6),
])
def test_create_rejects_bad_arguments(lib, kw, code):
    rc, h = _create(lib, **kw)
    assert rc == code
    assert not h.value
    msg = lib.lbif_last_error(None)
    assert msg and b"create" in msg


def test_null_handle_calls_fail_cleanly(lib):
    assert lib.lbif_step(None, 1) == -1
    assert lib.lbif_destroy(None) == -1
    assert lib.lbif_moments(None, None, None, None, 0) == -1
    assert lib.lbif_set_fused(None, 1) == -1
    t = ctypes.c_int32(3)
    assert lib.lbif_selftest_wait(0, ctypes.byref(t)) == -1 and t.value == 3
    assert lib.lbif_selftest_wait(10, None) == -1
    v = ctypes.c_int32(7)
    assert lib.lbif_get_fused(None, ctypes.byref(v)) == -1 and v.value == 7
    shapes = (ctypes.c_int32 * 5)(0, 0, 0, 0, 0)
    assert lib.lbif_get_shapes(None, shapes) == -1
    assert lib.lbif_set_shapes(None, shapes) == -1
    assert lib.lbif_autotune(None, 1, None, None, None) == -1
    assert lib.lbif_last_error(None)


def test_no_device_fails_loudly(lib):
    """Without a usable GPU, creation reports the CUDA runtime's error: there is
    no CPU path to fall back on (skipped where a GPU is present)."""
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    rc, h = _create(lib)
    assert rc == -3 and not h.value
    assert lib.lbif_last_error(None).startswith(b"create: ")


def test_missing_library_raises():
    """The binding raises when the CUDA library is absent (fresh interpreter)."""
    import subprocess
    import sys

    code = ("from paper_0712_2247_gb300 import lbif\n"
            "try:\n"
            "    lbif.load_library('/nonexistent/liblbif.so')\n"
            "except RuntimeError as e:\n"
            "    print('raised', 'missing' in str(e))\n")
    out = subprocess.run([sys.executable, "-c", code], cwd=ROOT, capture_output=True, text=True, timeout=300)
    assert out.stdout.strip() == "raised True", out.stdout + out.stderr


def test_oracle_builds_and_is_independent():
    """The oracle compiles on its own and shares no source with the CUDA path."""
    import oracle

    oracle.build()
    assert oracle.threads() >= 1  # what the benchmark reports as the oracle's cores
    csrc = glob.glob(os.path.join(ROOT, "paper_0712_2247_gb300", "csrc", "*"))
    for f in csrc:
        assert "oracle" not in open(f).read().lower(), f
    for f in glob.glob(os.path.join(ROOT, "oracle", "*")):
        if f.endswith((".c", ".py")):
            assert "paper_0712_2247_gb300" not in open(f).read().replace(
                "paper_0712_2247_gb300.inputs", ""), f


@pytest.mark.parametrize("args", [
    (0, 256, 3, 160, 16), (4, 8, 3, 160, 16), (4, 264, 3, 160, 16), (4, 250, 3, 160, 16),
    (4, 256, 0, 160, 16), (4, 256, 3, 0, 16), (4, 256, 3, 257, 16), (4, 256, 3, 160, 0),
])
def test_mlp_create_rejects_bad_widths(lib, args):
    from paper_0712_2247_gb300 import mlp

    mlp.load_library()
    h = ctypes.c_void_p()
    assert lib.lbif_mlp_create(ctypes.byref(h), *args, None) == -1
    assert not h.value
    assert b"lbif_mlp_create" in lib.lbif_mlp_last_error(None)


def test_mlp_null_handle(lib):
    from paper_0712_2247_gb300 import mlp

    mlp.load_library()
    assert lib.lbif_mlp_num_params(None) == -1
    assert lib.lbif_mlp_destroy(None) == -1
    assert lib.lbif_mlp_forward(None, None, 1, None, 0) == -1
