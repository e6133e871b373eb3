"""The paper's numerical experiments: shear viscosity from a decaying
transverse wave, static slit profiles (Sec. Numerical validation)."""
import math

import numpy as np
import pytest

from test_stability import linear_map


def shear_rate(oracle_mod, L, sigma, eta, tau):
    """Decay rate per step of the transverse (shear) mode of wave vector
    2 pi / L along x: the eigenvalue of the linearised map whose eigenvector
    carries y momentum."""
    c, _ = oracle_mod.lattice()
    M = linear_map(oracle_mod, np.array([2 * math.pi / L, 0.0, 0.0]), sigma, eta, tau)
    lam, V = np.linalg.eig(M)
    jy = np.abs(c[:, 1].astype(float) @ V) / np.linalg.norm(V, axis=0)
    return -math.log(abs(lam[int(np.argmax(jy))]))


@pytest.mark.parametrize("eta", [0.05, 0.25])
def test_shear_mode_long_wave_limit(oracle_mod, eta):
    """k -> 0: the discrete shear mode decays with nu = c_s^2 (tau - 1/2) plus
    the Longuet-Higgins-Pople collisional viscosity of the coupling term.
    Residual difference at sigma = 8: the bilinear interpolation of the
    diagonal shell points adds an O(t(1-t)/(k sigma)^2)-relative k^2 term
    (measured 0.5-0.7 %)."""
    from paper_0712_2247_gb300.experiments import nu_closed_form

    L = 4096
    k = 2 * math.pi / L
    nu = shear_rate(oracle_mod, L, 8, eta, 0.8) / k ** 2
    assert abs(nu / nu_closed_form(8, eta, 0.8) - 1) < 1e-2
    # the BGK part alone (hard-sphere force off is eta -> 0): c_s^2 (tau - 1/2)
    nu0 = shear_rate(oracle_mod, L, 8, 1e-9, 0.8) / k ** 2
    assert abs(nu0 / (0.8 - 0.5) * 3 - 1) < 1e-4


@pytest.mark.gpu
@pytest.mark.parametrize("eta", [0.10, 0.25, 0.30])
def test_shear_wave_decay_matches_the_discrete_symbol(oracle_mod, eta):
    """Transverse wave on the GPU (periodic 128 x 1 x 1 box, sigma = 8,
    amplitude 1e-4): its decay rate equals the exact shear eigenvalue of the
    linearised scheme (FP32 amplitude noise ~1e-8 against 1e-4 bounds the
    rate to ~1e-4 relative)."""
    from paper_0712_2247_gb300.experiments import shear_decay

    r = shear_decay(8, eta, 0.8, L=128)
    exact = shear_rate(oracle_mod, 128, 8, eta, 0.8)
    print(r, exact)
    assert abs(r["rate"] / exact - 1) < 1e-3


def test_static_steady_state_balances_exactly_on_the_oracle(oracle_mod):
    """FP64 oracle, static slit at n* = 0.512 (sigma = 8, L = 5 sigma) run to
    its steady state: every plane's z momentum balances exactly (interface
    fluxes of the populations against the force) and the unshifted velocity
    is exactly -F_z/(2n)."""
    from paper_0712_2247_gb300.experiments import plane_balance

    o = oracle_mod.Oracle(1, 1, 40, 8, math.pi * 0.512 / 6, 0.8, noise=0.0, seed=0)
    o.step(3000)
    n, u = o.moments()
    F, _ = o.forces()
    n, uz, fz = n[:, 0, 0], u[2, :, 0, 0], F[2, :, 0, 0]
    assert np.abs(plane_balance(n, uz, fz)).max() < 1e-12 * np.abs(fz).max()
    assert np.abs(uz + fz / (2 * n)).max() < 1e-12 * np.abs(uz).max()
    # and the wall layer: contact density well above the bulk, mirror symmetric
    assert n[0] > 1.5 * o.n0 and np.abs(n - n[::-1]).max() < 1e-12 * n.max()


@pytest.mark.gpu
def test_static_profile_matches_oracle_and_balances_forces(oracle_mod):
    """Static slit at n* = 0.512 (eta = 0.268), sigma = 8, L = 5 sigma, no
    field: the GPU profile equals the oracle's, is mirror-symmetric, and the
    equilibrium momentum balance c_s^2 dn/dz = F_z holds in the interior."""
    from paper_0712_2247_gb300 import lbif
    from paper_0712_2247_gb300.experiments import static_profile

    eta, H, steps = math.pi * 0.512 / 6, 40, 3000
    r = static_profile(8, eta, 0.8, H, steps=steps)
    o = oracle_mod.Oracle(1, 1, H, 8, eta, 0.8, noise=0.0, seed=0)
    o.step(steps)
    n, _ = o.moments()
    n_or = n[:, 0, 0] / o.n0
    n_gpu = np.array(r["n_over_n0"])
    print({k: v for k, v in r.items() if k != "n_over_n0"})
    assert np.abs(n_gpu - n_or).max() / np.abs(n_or).max() < 1e-5
    assert r["mirror"] < 1e-6
    assert r["contact_over_n0"] > 1.2  # layering: contact density above the bulk
    assert r["residual"] < 1e-6
    # exact discrete balances of the steady state, to FP32 rounding
    assert r["force_balance"] < 1e-4
    assert r["uz_relation"] < 1e-4
