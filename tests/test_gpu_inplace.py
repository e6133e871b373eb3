"""Populations in place (one buffer) against the two-buffer layout.

In place, direction i of every node moves by c_i slots each step, so that the
pull pass reads and writes the same slots (streaming with half-way
bounce-back, Sec. Methods); the arithmetic is the two-buffer pass's, so both
layouts give bit-identical states. Checked on tiled and per-node grids, walls
and periodic z, FP32 and FP16 storage, the tail, an ensemble run to steady
state with frozen slits, checkpoints across layouts; plus the oracle, and
the memory the layout saves.
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
    (40, 12, 30, 4, False, 0, {}),               # tiled pull, ragged tiles, walls
    (64, 8, 24, 4, True, 0, {}),                 # periodic z: no ghost plane
    (16, 16, 32, 4, False, 0, {}),               # per-node pull (nx < 32)
    (40, 12, 30, 4, False, 1, {}),               # FP16 storage
    (128, 8, 36, 8, False, 0, {}),               # tiled force, sigma 8
    (32, 16, 28, 4, False, 0, dict(tail=True, eps=0.3, rcut=2.5)),
]


@pytest.mark.parametrize("nx,ny,nz,sigma,zper,storage,extra", CASES)
def test_inplace_bit_identical_to_two_buffers(L, nx, ny, nz, sigma, zper, storage, extra):
    kw = dict(periodic_z=zper, storage=storage, body=(1e-5, -2e-6, 0.0), seed=4, **extra)
    a = L.Slit(nx, ny, nz, sigma, 0.22, 0.85, inplace=False, **kw)
    b = L.Slit(nx, ny, nz, sigma, 0.22, 0.85, inplace=True, **kw)
    for k in (1, 37, 62):  # odd and even counts: the clocks wrap in x, y and z
        a.step(k)
        b.step(k)
        ra, ua = a.moments()
        rb, ub = b.moments()
        assert np.array_equal(ra, rb) and np.array_equal(ua, ub), (k, nerr(rb, ra), nerr(ub, ua))
    a.close()
    b.close()


def test_inplace_matches_oracle_1000_steps(L):
    import oracle

    oracle.build()
    from paper_0712_2247_gb300.inputs import C0S as W

    g = L.Slit(W.nx, W.ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed, inplace=True)
    o = oracle.Oracle(W.nx, W.ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    g.step(W.steps)
    o.step(W.steps)
    rg, ug = g.moments()
    ro, uo = o.moments()
    ng, uxg, _ = g.profiles()
    no, uxo = o.profiles()
    e = dict(rho=nerr(rg, ro), u=nerr(ug, uo), n_z=nerr(ng, no), ux_z=nerr(uxg, uxo))
    print("in place, 1000 steps", e)
    assert all(v < 1e-5 for v in e.values()), e
    g.close()


def test_inplace_checkpoint_crosses_layouts(L, tmp_path):
    """A checkpoint holds the populations in node order: saved in place at
    step 23, loaded into a two-buffer handle (and back), both continue
    bit-identically."""
    kw = dict(body=(1e-5, 0, 0), seed=6)
    a = L.Slit(40, 12, 30, 4, 0.25, 0.9, inplace=True, **kw)
    a.step(23)
    path = str(tmp_path / "ip.bin")
    a.save(path)
    b = L.Slit(40, 12, 30, 4, 0.25, 0.9, inplace=False, **kw)
    b.load(path)
    a.step(17)
    b.step(17)
    ra, ua = a.moments()
    rb, ub = b.moments()
    assert np.array_equal(ra, rb) and np.array_equal(ua, ub)
    path2 = str(tmp_path / "tb.bin")
    b.save(path2)
    c = L.Slit(40, 12, 30, 4, 0.25, 0.9, inplace=True, **kw)
    c.load(path2)
    assert c.t == 40
    a.step(9)
    c.step(9)
    ra, ua = a.moments()
    rc_, uc = c.moments()
    assert np.array_equal(ra, rc_) and np.array_equal(ua, uc)
    for h in (a, b, c):
        h.close()


def test_inplace_ensemble_freezing(L):
    """Stacked slits (each with its own ring of planes and its own clock) run
    to steady state: the same steps per slit and bit-identical profiles as
    the two-buffer ensemble; a frozen slit's clock stops with it."""
    H = np.array([9, 16, 12, 21], np.int32)
    eta = np.array([0.15, 0.25, 0.2, 0.18])
    F = np.array([2e-6, 1e-6, 5e-6, 3e-6])
    tau = np.array([0.8, 1.0, 0.7, 1.1])
    res = []
    for ip in (False, True):
        e = L.Ensemble(H, eta, F, tau, sigma=4, nx=32, ny=8, storage=0, noise=0.0, inplace=ip)
        hmax = int(H.max())
        nz = np.zeros((len(H), hmax), np.float32)
        for s, h in enumerate(H):
            nz[s, :h] = e.n0_s[s] * (1 + 0.05 * np.cos(2 * np.pi * np.arange(h) / h))
        e.seed(nz)
        taken = e.run(tol=1e-7, max_steps=6000, check_every=50, patience=20)
        e.step(31)  # every slit again, after the freeze
        res.append((taken, e.slit_profiles()))
        e.close()
    (ta, (na, ua)), (tb, (nb, ub)) = res
    print("steps", ta, tb)
    assert np.array_equal(ta, tb)
    assert np.array_equal(na, nb) and np.array_equal(ua, ub)


def test_inplace_halves_population_memory(L):
    torch = pytest.importorskip("torch")
    torch.cuda.synchronize()
    nx, ny, nz = 256, 256, 96

    def used(ip):
        free0 = torch.cuda.mem_get_info()[0]
        g = L.Slit(nx, ny, nz, 4, 0.2, 0.9, inplace=ip)
        torch.cuda.synchronize()
        d = free0 - torch.cuda.mem_get_info()[0]
        g.close()
        torch.cuda.synchronize()
        return d

    two, one = used(False), used(True)
    pop = 19 * 4 * nx * ny * nz
    print("device bytes: two buffers", two, "in place", one, "one population buffer", pop)
    assert two - one > 0.9 * pop
