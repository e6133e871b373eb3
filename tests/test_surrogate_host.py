"""Host-side logic of the warm start: features, scaling, target encoding."""
import numpy as np

from paper_0712_2247_gb300 import inputs
from paper_0712_2247_gb300 import surrogate as S


def _profiles(p, seed=0):
    """Mirror-symmetric synthetic profiles of the right widths."""
    rng = np.random.default_rng(seed)
    hmax = int(p.H.max())
    n = np.zeros((len(p.H), hmax))
    u = np.zeros((len(p.H), hmax))
    n0 = S.n0_of(p.eta, p.sigma)
    for s, h in enumerate(p.H):
        j = S.fold(int(h))
        a = rng.standard_normal(h // 2 + 1)
        shape = 1.0 + 0.3 * np.exp(-j / 3.0) * np.cos(j) + 0.01 * a[j]
        n[s, :h] = n0[s] * shape * (h / shape.sum())  # the slit's mass n0 H
        u[s, :h] = S.u_ref(h, p.F[s], p.tau[s]) * (j + 0.5) * (h - j - 0.5) / (h / 2.0) ** 2
    return n, u


def test_fold_is_distance_to_nearest_wall():
    assert S.fold(5).tolist() == [0, 1, 2, 1, 0]
    assert S.fold(6).tolist() == [0, 1, 2, 2, 1, 0]
    assert S.fold(1).tolist() == [0]


def test_encode_decode_round_trip():
    p = inputs.ensemble(40, seed=11, nx=4, ny=4)
    n, u = _profiles(p)
    T, M = S.encode(n, u, p)
    assert T.shape == (40, 2 * S.HMAX) and M.shape == T.shape
    for s, h in enumerate(p.H):
        m = (int(h) + 1) // 2
        assert M[s, :m].all() and not M[s, m:S.HMAX].any()
        assert M[s, S.HMAX:S.HMAX + m].all() and not M[s, S.HMAX + m:].any()
    nd, ud = S.decode(T, p)
    for s, h in enumerate(p.H):
        h = int(h)
        assert np.allclose(nd[s, :h], n[s, :h], rtol=1e-6)
        assert np.allclose(ud[s, :h], u[s, :h], rtol=1e-6, atol=1e-12)
        assert not nd[s, h:].any() and not ud[s, h:].any()


def test_encode_averages_mirror_halves():
    p = inputs.ensemble(3, seed=2, nx=4, ny=4)
    n, u = _profiles(p)
    h = int(p.H[0])
    n[0, 0] *= 1.001  # break the symmetry at one wall
    T, _ = S.encode(n, u, p)
    n0 = S.n0_of(p.eta, p.sigma)[0]
    assert np.isclose(T[0, 0], 0.5 * (n[0, 0] + n[0, h - 1]) / n0, rtol=1e-6)


def test_decode_conserves_the_slit_mass():
    p = inputs.ensemble(30, seed=6, nx=4, ny=4)
    rng = np.random.default_rng(1)
    Y = (1.0 + 0.2 * rng.standard_normal((30, 2 * S.HMAX))).astype(np.float32)
    n, _ = S.decode(Y, p)
    n0 = S.n0_of(p.eta, p.sigma)
    for s, h in enumerate(p.H):
        assert np.isclose(n[s, :h].astype(np.float64).sum(), n0[s] * h, rtol=1e-5)


def test_decode_keeps_density_positive():
    p = inputs.ensemble(2, seed=3, nx=4, ny=4)
    Y = np.full((2, 2 * S.HMAX), -1.0, np.float32)
    n, _ = S.decode(Y, p)
    assert (n[0, :p.H[0]] > 0).all()


def test_scaling_and_features():
    p = inputs.ensemble(500, seed=4)
    raw = S.raw_features(p.H, p.eta, p.F, p.tau, p.sigma)
    assert raw.shape == (500, 4)
    assert np.allclose(raw[:, 0], p.H / 4.0) and np.allclose(raw[:, 2], np.log10(p.F))
    sc = S.Scaling.fit(raw)
    z = sc(raw)
    assert z.dtype == np.float32
    assert np.allclose(z.mean(axis=0), 0, atol=1e-6) and np.allclose(z.std(axis=0), 1, atol=1e-5)


def test_velocity_scale_is_the_poiseuille_maximum():
    # centre velocity of the ideal-fluid parabola F/(2 nu) (H/2)^2 = F H^2/(8 nu)
    assert np.isclose(S.u_ref(20, 1e-6, 0.8), 1e-6 * 400 / (8 * 0.1))
