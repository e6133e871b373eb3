"""The oracle's hard-sphere force (Eq. LBHS at constant T) against an evaluator
built from different parts: the 18 quadrature directions generated here from
their definition (the six axis directions and the twelve face diagonals,
weights 1/30 and 1/15), the coarse-grained density as a convolution with the
lattice ball (|d|^2 <= (sigma/2)^2, normalised by its node count), and every
off-lattice value by scipy's linear interpolation of the padded fields (wrap
in x, y; zeros beyond the walls) instead of the oracle's corner tables.

A dropped term, a wrong sign, a transposed corner weight or a misplaced
midpoint in the oracle's shell sum would show up here as an O(1) relative
error; the two agree to rounding.
"""
import itertools
import math

import numpy as np
import pytest
from scipy import ndimage

import oracle

KT = 1.0 / 3.0


def directions():
    """(unit vector, weight) of the 18-point sphere rule."""
    out = []
    for a in range(3):
        for s in (1.0, -1.0):
            e = np.zeros(3)
            e[a] = s
            out.append((e, 1.0 / 30.0))
    h = 1.0 / math.sqrt(2.0)
    for a, b in ((0, 1), (0, 2), (1, 2)):
        for sa, sb in itertools.product((1.0, -1.0), repeat=2):
            e = np.zeros(3)
            e[a], e[b] = sa * h, sb * h
            out.append((e, 1.0 / 15.0))
    return out


def g2(eta, form):
    if form == 1:
        return (1 - eta / 2) / (1 - eta) ** 3
    return (1 - eta / 2 + eta ** 2 / 4) / (1 - eta) ** 3


def pad(f, halo, zper):
    """(nz, ny, nx) field padded by `halo` nodes: periodic in x, y (and z if
    zper), zeros beyond the walls otherwise."""
    f = np.pad(f, ((0, 0), (halo, halo), (halo, halo)), mode="wrap")
    return np.pad(f, ((halo, halo), (0, 0), (0, 0)), mode="wrap" if zper else "constant")


def coarse_g2(n, sigma, zper, form):
    R2 = (sigma / 2) ** 2
    r = sigma // 2
    d = np.arange(-r, r + 1)
    ball = ((d[:, None, None] ** 2 + d[None, :, None] ** 2 + d[None, None, :] ** 2) <= R2).astype(float)
    big = pad(n, r, zper)
    nbar = ndimage.correlate(big, ball, mode="constant", cval=0.0)[r:-r, r:-r, r:-r] / ball.sum()
    return g2(math.pi * sigma ** 3 / 6 * nbar, form)


def shell_force(n, u, sigma, zper, coupling=True, regularize=True, form=0):
    nz, ny, nx = n.shape
    G = coarse_g2(n, sigma, zper, form)
    halo = sigma + 2
    P = {k: pad(v, halo, zper) for k, v in (("n", n), ("G", G), ("ux", u[0]), ("uy", u[1]), ("uz", u[2]))}
    z, y, x = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    kappa = 2.0 / (math.sqrt(KT) * math.sqrt(math.pi))
    if regularize and not zper:
        lam = 1.0 - np.exp(-np.minimum(z + 0.5, nz - 0.5 - z) / sigma)
    else:
        lam = np.ones(n.shape)

    def at(name, off):
        coords = np.stack([z + off[2] + halo, y + off[1] + halo, x + off[0] + halo]).reshape(3, -1)
        return ndimage.map_coordinates(P[name], coords, order=1, mode="constant", cval=0.0).reshape(n.shape)

    F = np.zeros((3,) + n.shape)
    for e, w in directions():
        p, m = sigma * e, 0.5 * sigma * e
        nq, Gq = at("n", p), at("G", m)
        du = sum(e[k] * (at(c, p) - u[k]) for k, c in enumerate(("ux", "uy", "uz")))
        bracket = 1.0 - lam * kappa * du if coupling else 1.0
        t = w * Gq * n * nq * bracket
        for k in range(3):
            F[k] -= e[k] * t
    return KT * sigma ** 2 * 4 * math.pi * F


def fields(shape, seed, n0):
    rng = np.random.default_rng(seed)
    n = n0 * (1.0 + 0.2 * rng.uniform(-1, 1, shape))
    u = 0.05 * rng.uniform(-1, 1, (3,) + shape)
    return n, u


@pytest.mark.parametrize("shape,sigma,zper,opts", [
    ((6, 5, 7), 2, True, {}),
    ((7, 6, 5), 4, True, {}),
    ((14, 6, 8), 4, False, {}),
    ((14, 6, 8), 4, False, dict(regularize=False)),
    ((12, 5, 6), 4, False, dict(coupling=False, form=1)),
    ((26, 4, 5), 8, False, {}),
])
def test_oracle_shell_force_equals_independent_evaluation(shape, sigma, zper, opts):
    n0 = 6 * 0.25 / (math.pi * sigma ** 3)
    n, u = fields(shape, 17, n0)
    Fo, Go, _ = oracle.hs_force(n, sigma, zper, u=u, coupling=opts.get("coupling", True),
                                regularize=opts.get("regularize", True), g2form=opts.get("form", 0))
    Fi = shell_force(n, u, sigma, zper, **opts)
    scale = np.abs(Fi).max()
    assert scale > 0
    assert np.abs(Fo - Fi).max() <= 1e-12 * scale
    assert np.allclose(Go, coarse_g2(n, sigma, zper, opts.get("form", 0)), rtol=1e-13, atol=0)
