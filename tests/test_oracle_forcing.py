"""The paper's first-order force source against velocity-shifted second-order
forcing (u = (j + F/2)/n in the equilibrium, source (1 - 1/2tau) w_i [(c - u).F
/ c_s^2 + (c.u)(c.F) / c_s^4]), measured on the ideal fluid in a bounce-back slit,
where the force does not depend on u and the shifted scheme is explicit.

Both schemes reach an exact discrete Navier-Stokes parabola (interior second
differences -F/nu). Their steady populations coincide: the shifted velocity
is the first-order scheme's j/n plus F/2, so the wall slip of the shifted
scheme is F (16 tau^2 - 16 tau + 1) / (24 nu) where the paper's has
F (16 tau^2 - 20 tau + 3) / (24 nu) (the half-way bounce-back slip of the
unshifted velocity, He, Zou, Luo & Dembo 1997). With the hard-sphere force,
whose coupling term depends on u, the shifted scheme would be implicit; the
oracle refuses it.
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


def test_shifted_forcing_refuses_a_velocity_dependent_force():
    o = oracle.Oracle(4, 4, 8, 4, 0.2, 0.9, body=(1e-6, 0, 0))
    o.init_fields(np.full((8, 4, 4), o.n0))
    with pytest.raises(ValueError):
        o.step(1, shifted=True)
