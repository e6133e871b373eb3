"""The ensemble of stacked slits (one launch per kernel over all slits)."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def nerr(a, b):
    a = np.asarray(a, dtype=np.float64)
    b = np.asarray(b, dtype=np.float64)
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.fixture(scope="module")
def L():
    from paper_0712_2247_gb300 import build, lbif

    build.build()
    return lbif


@pytest.fixture(scope="module")
def O():
    import oracle

    oracle.build()
    return oracle


H = np.array([9, 16, 23, 12], np.int32)
ETA = np.array([0.12, 0.25, 0.2, 0.16])
F = np.array([2e-6, 1e-7, 5e-6, 1e-5])
TAU = np.array([0.7, 1.0, 1.2, 0.6])


@pytest.mark.parametrize("storage", [0, 1])
def test_each_slit_matches_its_own_oracle(L, O, storage):
    e = L.Ensemble(H, ETA, F, TAU, sigma=4, nx=8, ny=6, storage=storage, noise=0.0)
    # seed every slit with the same non-uniform profile shape
    hmax = int(H.max())
    nz = np.zeros((len(H), hmax), np.float32)
    for s, h in enumerate(H):
        z = np.arange(h)
        nz[s, :h] = e.n0_s[s] * (1 + 0.05 * np.cos(2 * np.pi * z / h))
    e.seed(nz)
    steps = 60
    e.step(steps)
    rho, u = e.moments()
    for s, h in enumerate(H):
        o = O.Oracle(8, 6, int(h), 4, ETA[s], TAU[s], body=(F[s], 0, 0))
        o.init_fields(np.repeat(nz[s, :h].astype(np.float64), 48).reshape(h, 6, 8))
        o.step(steps)
        n_o, u_o = o.moments()
        z0 = int(e.zlo[s])
        tol = 1e-5 if storage == 0 else 1e-3
        assert nerr(rho[z0:z0 + h], n_o) < tol, s
        assert nerr(u[:, z0:z0 + h], u_o) < (1e-5 if storage == 0 else 2e-2), s
    # gap planes between slits read as empty
    z1 = int(e.zlo[1])
    assert np.all(rho[int(H[0]):z1] == 0.0)
    e.close()


def test_stacked_equals_separate_handles(L):
    """A slit in the stack evolves bit-identically to the same slit alone."""
    e = L.Ensemble(H, ETA, F, TAU, sigma=4, nx=8, ny=8, noise=0.0, storage=0)
    hmax = int(H.max())
    nz = np.zeros((len(H), hmax), np.float32)
    for s, h in enumerate(H):
        nz[s, :h] = e.n0_s[s] * (1 + 0.02 * np.sin(np.arange(h)))
    e.seed(nz)
    e.step(25)
    n_g, ux_g = e.slit_profiles(hmax)
    for s in (0, 2):
        h = int(H[s])
        g = L.Slit(8, 8, h, 4, ETA[s], TAU[s], body=(F[s], 0, 0), noise=0.0)
        g.set_fields(np.repeat(nz[s, :h], 64).reshape(h, 8, 8).astype(np.float32))
        g.step(25)
        n1, u1, _ = g.profiles()
        assert np.array_equal(n1, n_g[s, :h]) and np.array_equal(u1, ux_g[s, :h]), s
    e.close()


def test_run_to_steady_state_and_freeze(L):
    """Cold uniform start (no noise: the state stays x,y-uniform), FP64 residual < 1e-8."""
    e = L.Ensemble(H[:3], ETA[:3], F[:3], TAU[:3], sigma=4, nx=4, ny=4, storage=0, noise=0.0)
    taken = e.run(tol=1e-8, max_steps=200000, check_every=100)
    print("steps to 1e-8", taken)
    assert np.all(taken > 0), taken
    n1, u1 = e.slit_profiles()
    # converged: a further run stops after the first residual check pair
    taken2 = e.run(tol=1e-8, max_steps=2000, check_every=100)
    assert np.all(taken2 <= 200), taken2
    n2, u2 = e.slit_profiles()
    for s, h in enumerate(H[:3]):
        assert nerr(n2[s, :h], n1[s, :h]) < 1e-6
    e.close()


def test_fp16_ensemble_reports_its_rounding_floor(L):
    e = L.Ensemble(H[:3], ETA[:3], F[:3], TAU[:3], sigma=4, nx=4, ny=4, storage=1, noise=0.0)
    taken, res = e.run(tol=1e-8, max_steps=100000, check_every=100, patience=20,
                       return_residual=True)
    print("fp16 ensemble", taken, res)
    # FP16 storage cannot reach 1e-8: every slit stalls at a finite floor
    # (measured 3e-5 .. 1.3e-3), which the run reports instead of spinning on
    assert np.all((taken > 0) | (taken == -3)), taken
    assert np.all(np.isfinite(res)) and np.all(res < 1e-2), res


def test_warm_seed_converges_faster(L):
    """Seeded with the converged profiles, slits reach the residual in fewer steps
    than from the cold uniform start (or stall at the FP32 floor, reported as -3)."""
    e = L.Ensemble(H[:3], ETA[:3], F[:3], TAU[:3], sigma=4, nx=4, ny=4, storage=0, noise=0.0)
    cold = e.run(tol=1e-8, max_steps=200000, check_every=100)
    n, u = e.slit_profiles()
    e.seed(n.astype(np.float32), u.astype(np.float32))
    warm, res = e.run(tol=1e-8, max_steps=200000, check_every=100, patience=20,
                      return_residual=True)
    print("cold", cold, "warm", warm, res)
    ok = warm > 0
    assert ok.sum() >= 2 and np.all(warm[ok] <= cold[ok]), (warm, cold)
    e.close()


def test_autotune_keeps_state(L):
    e = L.Ensemble(H, ETA, F, TAU, sigma=4, nx=16, ny=16, storage=1, seed=5)
    e.step(10)
    n0, u0 = e.slit_profiles()
    b, g, st = e.autotune(trials=2)
    assert b > 0 and g > 0 and st in (0, 1)
    n1, u1 = e.slit_profiles()
    assert np.array_equal(n0, n1) and np.array_equal(u0, u1)
    e.step(10)
    assert e.status() == 0
    # the chosen shapes and staging change no arithmetic: same result as the defaults
    d = L.Ensemble(H, ETA, F, TAU, sigma=4, nx=16, ny=16, storage=1, seed=5)
    d.step(20)
    n2, u2 = e.slit_profiles()
    n3, u3 = d.slit_profiles()
    assert np.array_equal(n2, n3) and np.array_equal(u2, u3)
    d.close()
    e.close()
