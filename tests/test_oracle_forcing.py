"""The paper's first-order force source against velocity-shifted second-order
forcing (u = (j + F/2)/n in the equilibrium, source (1 - 1/2tau) w_i [(c - u).F
/ c_s^2 + (c.u)(c.F) / c_s^4]), measured on the ideal fluid in a bounce-back slit,
where the force does not depend on u and the shifted scheme is explicit.

Both schemes reach an exact discrete Navier-Stokes parabola (interior second
differences -F/nu). Their steady populations coincide: the shifted velocity
is the first-order scheme's j/n plus F/2, so the wall slip of the shifted
scheme is F (16 tau^2 - 16 tau + 1) / (24 nu) where the paper's has
F (16 tau^2 - 20 tau + 3) / (24 nu) (the half-way bounce-back slip of the
unshifted velocity, He, Zou, Luo & Dembo 1997).

With the hard-sphere force, whose density-current term depends on u, the
shifted scheme is explicit when the force is evaluated from the unshifted
moments n, u = j/n (the reading taken here; only the equilibrium velocity
(j + F/2)/n and the source are shifted). Its pins below: without any force it
is the plain step bit for bit; per step it keeps the mass exactly and adds
exactly the total force to the momentum of a periodic box (the collision
contributes F/(2 tau), the source (1 - 1/(2 tau)) F); slit profiles from a
noise-free start stay mirror-symmetric.
"""
import numpy as np
import pytest

import oracle


def steady_ux(tau, nz, F, shifted):
    o = oracle.Oracle(1, 1, nz, 4, 0.3, tau, body=(F, 0, 0), hs=False)
    o.init_fields(np.full(nz, 0.02))
    nu = (tau - 0.5) / 3
    o.step(int(60 * nz * nz / nu) // 10 + 2000, shifted=shifted)
    n, u = o.moments()
    return u[0].ravel() + (F / 2 if shifted else 0.0), n.ravel()


@pytest.mark.parametrize("tau", [0.6, 0.8, 1.0, 1.2])
@pytest.mark.parametrize("nz", [12, 20])
def test_shifted_forcing_against_the_first_order_source(tau, nz):
    F = 1e-6
    nu = (tau - 0.5) / 3
    zc = np.arange(nz) - (nz - 1) / 2
    parabola = F / (2 * nu) * ((nz / 2) ** 2 - zc ** 2)
    plain, n1 = steady_ux(tau, nz, F, False)
    shifted, n2 = steady_ux(tau, nz, F, True)
    umax = parabola.max()
    for u in (plain, shifted):
        d2 = u[2:] - 2 * u[1:-1] + u[:-2]
        assert np.abs(d2 + F / nu).max() < 1e-8 * F / nu
    assert np.abs(plain - parabola - F * (16 * tau ** 2 - 20 * tau + 3) / (24 * nu)).max() < 1e-8 * umax
    assert np.abs(shifted - plain - F / 2).max() < 1e-8 * umax
    assert np.abs(shifted - parabola - F * (16 * tau ** 2 - 16 * tau + 1) / (24 * nu)).max() < 1e-8 * umax
    assert np.abs(n1 - 0.02).max() < 1e-10 and np.abs(n2 - 0.02).max() < 1e-10


def test_shifted_forcing_without_force_is_the_plain_step():
    kw = dict(hs=False, seed=3, noise=2e-2)
    a = oracle.Oracle(6, 5, 9, 4, 0.2, 0.8, **kw)
    b = oracle.Oracle(6, 5, 9, 4, 0.2, 0.8, **kw)
    a.step(7)
    b.step(7, shifted=True)
    assert np.array_equal(a.populations(), b.populations())


@pytest.mark.parametrize("coupling", [True, False])
def test_shifted_forcing_with_the_hard_sphere_force_books_mass_and_momentum(coupling):
    """Periodic box, hard-sphere force (with and without its density-current
    term) and a body force: per step the mass is unchanged and the momentum
    grows by the total force of the state the step started from."""
    o = oracle.Oracle(8, 8, 8, 4, 0.2, 0.8, zper=True, body=(2e-5, -1e-5, 5e-6), coupling=coupling,
                      seed=5, noise=2e-2)
    for _ in range(4):
        F, _ = o.forces()
        t0 = o.totals()
        o.step(1, shifted=True)
        t1 = o.totals()
        assert abs(t1[0] - t0[0]) <= 1e-14 * t0[0]
        dp = t1[1:] - t0[1:]
        assert np.abs(dp - F.reshape(3, -1).sum(axis=1)).max() <= 1e-12 * np.abs(F).sum()


def test_shifted_forcing_keeps_slit_profiles_mirror_symmetric():
    o = oracle.Oracle(4, 4, 24, 4, 0.22, 0.8, body=(1e-6, 0, 0))
    o.init_fields(np.full((24, 4, 4), o.n0))
    for _ in range(3):
        o.step(40, shifted=True)
        n, ux = o.profiles()
        assert np.abs(n - n[::-1]).max() < 1e-13 * n.max()
        assert np.abs(ux - ux[::-1]).max() < 1e-11 * np.abs(ux).max()


def test_shifted_forcing_refuses_the_energy_source():
    o = oracle.Oracle(4, 4, 8, 4, 0.2, 0.9, body=(1e-6, 0, 0), c2=True)
    o.init_fields(np.full((8, 4, 4), o.n0))
    with pytest.raises(ValueError):
        o.step(1, shifted=True)
