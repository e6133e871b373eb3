"""The pull pass's three gather forms give bit-identical steps.

The pull pass (collision, streaming with half-way bounce-back and the next
moments, Sec. Methods) reads each node's 19 arriving populations either with
plain loads, with the loads of the next plane issued one plane ahead, or from
per-direction source boxes copied into shared memory by the tensor-memory
accelerator (interior planes of interior tiles; walls, periodic edges and
ragged tiles keep direct loads). Only the route of the loads differs, so the
states must agree bit for bit, on every grid form and z-segment length, in
FP32 and FP16 storage. The accelerator form is also held to the oracle over
a long run on the benchmark's parameters.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def nerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    s = np.abs(b).max()
    return float(np.abs(a - b).max() / s) if s > 0 else float(np.abs(a).max())


@pytest.fixture(scope="module")
def L():
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    return lbif


CASES = [
    # (nx, ny, nz, sigma, periodic z, storage, extra)
    (128, 16, 40, 4, False, 0, {}),                      # walls, interior tiles in x and y
    (128, 16, 40, 4, False, 1, {}),                      # FP16 storage (16-node x alignment)
    (96, 12, 33, 4, True, 0, {}),                        # periodic z, ragged z segments
    (96, 12, 33, 4, True, 1, {}),
    (160, 20, 26, 8, False, 0, dict(shifted=True)),      # velocity-shifted forcing
    (128, 16, 30, 4, False, 0, dict(tail=True, eps=0.3, rcut=2.5, c2=True)),
]


@pytest.mark.parametrize("nx,ny,nz,sigma,zper,storage,extra", CASES)
def test_gather_forms_bit_identical(L, nx, ny, nz, sigma, zper, storage, extra):
    kw = dict(periodic_z=zper, storage=storage, body=(1e-5, -2e-6, 0.0), seed=5, **extra)
    ref = L.Slit(nx, ny, nz, sigma, 0.22, 0.85, **kw)
    ref.set_shapes(pull_gathers="loads")
    ref.step(23)
    r0, u0 = ref.moments()
    for gathers in ("prefetch", "tma"):
        for lz in (8, 16, 32):
            g = L.Slit(nx, ny, nz, sigma, 0.22, 0.85, **kw)
            g.set_shapes(pull_lz=lz, pull_gathers=gathers)
            assert g.shapes()["pull_gathers"] == gathers
            g.step(23)
            r, u = g.moments()
            assert g.status() == 0
            assert np.array_equal(r, r0) and np.array_equal(u, u0), (gathers, lz, nerr(r, r0), nerr(u, u0))
            g.close()
    ref.close()


def test_gather_forms_in_a_stacked_ensemble(L):
    """Slits stacked with gap planes between them (each plane's sources must
    stay in its own slit), frozen slits skipped."""
    H = np.array([9, 16, 12, 21], np.int32)
    eta = np.array([0.15, 0.25, 0.2, 0.18])
    F = np.array([2e-6, 1e-6, 5e-6, 3e-6])
    tau = np.array([0.8, 1.0, 0.7, 1.1])
    res = []
    for gathers in ("loads", "tma"):
        e = L.Ensemble(H, eta, F, tau, sigma=4, nx=96, ny=12, storage=0, seed=2, inplace=False)
        e.set_shapes(pull_gathers=gathers)
        e.step(40)
        res.append(e.moments())
        e.close()
    (ra, ua), (rb, ub) = res
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)


def test_tma_gathers_need_aligned_rows(L):
    # x rows of 130 FP32 nodes (520 bytes) are not a multiple of 16 bytes;
    # in-place handles have no second buffer to map
    for kw in (dict(nx=130), dict(nx=128, inplace=True)):
        nx = kw.pop("nx")
        g = L.Slit(nx, 12, 20, 4, 0.2, 0.9, **kw)
        with pytest.raises(L.LbifError) as ex:
            g.set_shapes(pull_gathers="tma")
        assert ex.value.code == -6
        assert g.shapes()["pull_gathers"] == "loads"
        g.close()
    g = L.Slit(128, 12, 20, 4, 0.2, 0.9)
    with pytest.raises(L.LbifError) as ex:
        g.set_shapes(pull_gathers="tma", pull_lz=-1)
    assert ex.value.code == -1
    g.close()


def test_tma_gathers_match_oracle_1000_steps(L):
    """128 x 12 x 72 slit on the benchmark's parameters (sigma 12, eta 0.25,
    tau 0.7, F_e = 5e-7), accelerator gathers, 1000 steps."""
    import oracle

    oracle.build()
    from paper_0712_2247_gb300.inputs import C2 as W

    nx, ny, nz = 128, 12, 72
    g = L.Slit(nx, ny, nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    g.set_shapes(pull_gathers="tma")
    o = oracle.Oracle(nx, ny, nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    g.step(1000)
    o.step(1000)
    rg, ug = g.moments()
    ro, uo = o.moments()
    ng, uxg, _ = g.profiles()
    no, uxo = o.profiles()
    e = dict(rho=nerr(rg, ro), rho_fluct=nerr(rg - o.n0, ro - o.n0), u=nerr(ug, uo), n_z=nerr(ng, no),
             ux_z=nerr(uxg, uxo))
    print("tma gathers, sigma 12, 1000 steps", e)
    assert g.status() == 0
    assert all(v < 1e-5 for v in e.values()), e
    g.close()
