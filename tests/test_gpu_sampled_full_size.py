"""Force parity at the benchmark's full size on sampled outputs.

The total force at a node (body force n F_e plus the hard-sphere shell force of
Eq. LBHS) depends only on the fields within a fixed reach: the shell points lie
sigma away, their bilinear corners one node further, and the contact value g2 at
a midpoint (sigma/2 away, corners one further) averages n over a ball of radius
sigma/2. A periodic window of the fields around a column, at least that reach
wide on each side in x and y (all of z), therefore gives the oracle everything
the column's force needs; the oracle's periodic wrap inside the window only
touches nodes outside that reach. `column_force` computes the column's force
that way; the CPU test pins it against the oracle on whole small grids, the GPU
test then samples columns of the 512 x 512 x 192, sigma = 12 slit (the
benchmark's launch shape, seeded noise) after a few steps.
"""
import numpy as np
import pytest

import oracle


def reach(sigma: int) -> int:
    """Nodes in x or y that a column's force depends on (shell point + corner,
    or midpoint + corner + ball radius)."""
    return max(sigma + 1, sigma // 2 + 1 + sigma // 2)


def column_force(n, u, x0, y0, sigma, body, n0, zper=False):
    """Total force / n0 on column (x0, y0) of the fields n (nz, ny, nx) and u
    (3, nz, ny, nx), from the oracle on a periodic window of half-width
    reach(sigma) + 1 around it: shape (3, nz)."""
    h = reach(sigma) + 1
    nz, ny, nx = n.shape
    xs = np.arange(x0 - h, x0 + h + 1) % nx
    ys = np.arange(y0 - h, y0 + h + 1) % ny
    nw = np.ascontiguousarray(n[:, ys][:, :, xs], dtype=np.float64)
    uw = np.ascontiguousarray(u[:, :, ys][:, :, :, xs], dtype=np.float64)
    F, _, _ = oracle.hs_force(nw, sigma, zper, u=uw)
    c = nw[:, h, h]
    return np.stack([(c * body[a] + F[a, :, h, h]) / n0 for a in range(3)])


@pytest.mark.parametrize("shape,sigma,zper", [((40, 36, 20), 4, False), ((44, 40, 30), 8, True),
                                              ((64, 60, 30), 12, False)])
def test_window_force_equals_whole_grid_force(shape, sigma, zper):
    from paper_0712_2247_gb300 import inputs

    nx, ny, nz = shape
    n0 = 6 * 0.25 / (np.pi * sigma ** 3)
    rho, u = inputs.random_fields((nz, ny, nx), n0, 21, uamp=1e-2)
    n = rho.astype(np.float64)
    u = u.astype(np.float64)
    body = (5e-7, -1e-7, 2e-7)
    F, _, _ = oracle.hs_force(n, sigma, zper, u=u)
    for x0, y0 in ((0, 0), (nx - 1, ny // 2), (nx // 3, ny - 1), (nx // 2, ny // 2)):
        full = np.stack([(n[:, y0, x0] * body[a] + F[a, :, y0, x0]) / n0 for a in range(3)])
        win = column_force(n, u, x0, y0, sigma, body, n0, zper)
        assert np.abs(win - full).max() <= 1e-13 * np.abs(full).max(), (x0, y0)


@pytest.mark.gpu
def test_full_size_sigma12_sampled_columns():
    """512 x 512 x 192, sigma 12, eta 0.25, seeded noise, 3 steps (fused pass,
    the benchmark's launch shape): the force the GPU applies on sampled columns
    (grid corners, edges, interior) against the oracle's on the same FP32
    fields, normwise per column."""
    from paper_0712_2247_gb300 import build, lbif
    from paper_0712_2247_gb300.inputs import c2

    build.build()
    W = c2(0.25, 0)
    g = lbif.Slit(W.nx, W.ny, W.nz, W.sigma, W.eta, W.tau, body=W.body, seed=W.seed)
    assert g.fused
    g.step(3)
    rho, u = g.moments()
    F = g.forces()
    n0 = g.n0
    g.close()
    worst = 0.0
    for x0, y0 in ((0, 0), (W.nx - 1, 300), (137, W.ny - 1), (256, 255), (400, 17)):
        want = column_force(rho, u, x0, y0, W.sigma, W.body, n0)
        got = F[:, :, y0, x0].astype(np.float64)
        e = np.abs(got - want).max() / np.abs(want).max()
        worst = max(worst, e)
        assert e < 1e-5, (x0, y0, e)
    print("sampled full-size force columns, max normwise error", worst)
