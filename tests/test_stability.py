"""Stability of the explicit scheme, decided on the FP64 oracle.

The linearised update around the uniform rest state is, for one lattice wave
vector k, a 19 x 19 map: collide (BGK towards the linearised equilibrium plus
the source w_i c_i.F/c_s^2 with the linear response of the force of Eq. LBHS,
its Fourier symbol built from the interpolation and ball symbols), then stream
(multiply by exp(-i k.c_i)). Its spectral radius is the growth factor per step.
The density-current (coupling) term is an explicit nonlocal viscosity: at
sigma = 4 it is stable up to eta = 0.25 and unstable at eta = 0.30, so the
16x16x32 slit at eta = 0.30 diverges and the one at 0.25 does not.
"""
import itertools
import math

import numpy as np
import pytest

KT = 1.0 / 3.0


def _interp_symbol(k, s):
    out = 1.0 + 0j
    for a in range(3):
        b = math.floor(s[a])
        t = s[a] - b
        out *= (1 - t) * np.exp(1j * k[a] * b) + t * np.exp(1j * k[a] * (b + 1))
    return out


def _ball_symbol(k, sigma):
    r = sigma // 2
    acc, cnt = 0.0, 0
    for dz, dy, dx in itertools.product(range(-r, r + 1), repeat=3):
        if dx * dx + dy * dy + dz * dz <= r * r:
            acc += math.cos(k[0] * dx + k[1] * dy + k[2] * dz)
            cnt += 1
    return acc / cnt


def _dg2(eta):
    N = 1 - eta / 2 + eta ** 2 / 4
    return (-0.5 + eta / 2) / (1 - eta) ** 3 + 3 * N / (1 - eta) ** 4


def growth_factor(oracle_mod, k, sigma, eta, tau, coupling=True):
    M = linear_map(oracle_mod, k, sigma, eta, tau, coupling)
    return float(np.abs(np.linalg.eigvals(M)).max())


def linear_map(oracle_mod, k, sigma, eta, tau, coupling=True):
    """One step of the scheme linearised about the uniform rest state, for
    perturbations a_i = delta f_i / n0 of wave vector k (a 19 x 19 matrix)."""
    A, B = linear_map_parts(oracle_mod, k, sigma, eta, tau, coupling)
    return A + B


def linear_map_parts(oracle_mod, k, sigma, eta, tau, coupling=True):
    """The linearised step split into streaming x (BGK collision) and
    streaming x (force source driven by the force's linear response)."""
    c, w = oracle_mod.lattice()
    cf = c.astype(float)
    d, sw = oracle_mod.sphere_rule()
    n0 = 6 * eta / (math.pi * sigma ** 3)
    G0, G1 = oracle_mod.g2(eta), _dg2(eta)
    C = KT * sigma ** 2 * 4 * math.pi
    kap = 2 / (math.sqrt(KT) * math.sqrt(math.pi))
    B = _ball_symbol(k, sigma)
    An = np.zeros(3, complex)
    Au = np.zeros((3, 3), complex)
    for q in range(18):
        Iq = _interp_symbol(k, sigma * d[q])
        Jq = _interp_symbol(k, 0.5 * sigma * d[q])
        An += sw[q] * d[q] * (G0 * Iq + G1 * eta * B * Jq)
        if coupling:
            Au += sw[q] * np.outer(d[q], d[q]) * (Iq - 1)
    Mn = np.ones(19)          # dn = sum_i a_i
    Mj = cf.T                 # dj = sum_i c_i a_i ;  u = dj / n0
    Fa = -C * n0 * np.outer(An, Mn) + C * n0 * G0 * kap * (Au @ Mj)
    aeq = w[:, None] * (Mn[None, :] + 3 * cf @ Mj)
    D = np.diag(np.exp(-1j * cf @ k))
    return D @ (np.eye(19) - (np.eye(19) - aeq) / tau), D @ (3 * (w[:, None] * cf) @ Fa)


def _scan(oracle_mod, sigma, eta, tau, L=8):
    ks = 2 * np.pi * np.arange(L // 2 + 1) / L
    worst = 0.0
    for kx, ky, kz in itertools.product(ks, ks, ks):
        if ky > kx:
            continue
        worst = max(worst, growth_factor(oracle_mod, np.array([kx, ky, kz]), sigma, eta, tau))
    return worst


def test_linear_growth_sigma4(oracle_mod):
    # includes k = (pi/4)(1,1,1), the most unstable mode at eta = 0.30
    assert _scan(oracle_mod, 4, 0.25, 1.0) < 1 + 1e-9
    assert _scan(oracle_mod, 4, 0.30, 1.0) > 1.01


def test_long_wave_modes_are_neutral(oracle_mod):
    """k -> 0: mass and momentum are conserved, so the growth factor tends to 1."""
    g = growth_factor(oracle_mod, np.array([1e-4, 0, 0]), 4, 0.25, 0.8)
    assert abs(g - 1) < 1e-6


def test_c0_slit_diverges_and_eta025_does_not(oracle_mod):
    from paper_0712_2247_gb300.inputs import C0, C0S

    o = oracle_mod.Oracle(C0.nx, C0.ny, C0.nz, C0.sigma, C0.eta, C0.tau, body=C0.body, seed=C0.seed)
    o.step(30)
    n, _ = o.moments()
    assert not np.all(np.isfinite(n)) or n.min() < 0 or n.max() > 100 * o.n0
    s = oracle_mod.Oracle(C0S.nx, C0S.ny, C0S.nz, C0S.sigma, C0S.eta, C0S.tau, body=C0S.body,
                          seed=C0S.seed)
    s.step(300)
    n, u = s.moments()
    assert np.all(np.isfinite(n)) and n.min() > 0.5 * s.n0 and n.max() < 3 * s.n0
    # the initial noise has decayed: the state is x,y-uniform again
    assert np.abs(n - n.mean(axis=(1, 2), keepdims=True)).max() < 1e-10 * s.n0


def test_without_coupling_bulk_is_stable_but_slits_diverge(oracle_mod):
    """Dropping the density-current term removes the bulk instability (the
    linearised map is neutral up to eta = 0.45), yet a slit started uniform
    then diverges nonlinearly at eta = 0.25, where the coupled slit settles:
    the coupling term is the viscosity that damps the wall layering."""
    ks = 2 * np.pi * np.arange(5) / 8
    worst = 0.0
    for kx, ky, kz in itertools.product(ks, ks, ks):
        if ky > kx:
            continue
        worst = max(worst, growth_factor(oracle_mod, np.array([kx, ky, kz]), 4, 0.45, 0.9,
                                         coupling=False))
    assert worst < 1 + 1e-9
    runs = {}
    for c in (0, 1):
        o = oracle_mod.Oracle(1, 1, 30, 4, 0.25, 0.9, body=(1e-6, 0, 0), coupling=c, noise=0.0, seed=0)
        o.step(300)
        n, _ = o.moments()
        runs[c] = (n[:, 0, 0], o.n0)
    n, n0 = runs[0]
    assert not np.all(np.isfinite(n)) or n.max() > 100 * n0
    n, n0 = runs[1]
    assert np.all(np.isfinite(n)) and 0.1 * n0 < n.min() and n.max() < 5 * n0


def _lagged_radius(oracle_mod, sigma, eta, tau, coupling):
    ks = 2 * np.pi * np.arange(5) / 8
    worst = 0.0
    for kx, ky, kz in itertools.product(ks, ks, ks):
        if ky > kx or kz > ky:
            continue
        A, B = linear_map_parts(oracle_mod, np.array([kx, ky, kz]), sigma, eta, tau, coupling)
        # state (a_t, a_{t-1}): the force of the previous step drives the collision
        L = np.block([[A, B], [np.eye(19), np.zeros((19, 19))]])
        worst = max(worst, float(np.abs(np.linalg.eigvals(L)).max()))
    return worst


def test_lagged_force_single_pass_variant_is_unstable(oracle_mod):
    """Driving the collision of step t with the force of step t - 1 (what a
    push-form single pass, collision then moments of the same node, needs)
    makes the scheme
    unstable: the linearised two-step map grows even at eta = 0.02 with the
    density-current term (at 0.25 without it), and the FP64 oracle's lagged
    steps diverge where plain steps stay at rest."""
    assert _lagged_radius(oracle_mod, 4, 0.02, 0.9, True) > 1.02
    assert _lagged_radius(oracle_mod, 4, 0.02, 0.9, False) < 1 + 1e-9
    assert _lagged_radius(oracle_mod, 4, 0.25, 0.9, False) > 1.05
    for lagged in (False, True):
        o = oracle_mod.Oracle(8, 8, 8, 4, 0.02, 0.9, zper=True, noise=1e-3, seed=1)
        o.step(1500, lagged=lagged)
        n, _ = o.moments()
        dev = np.abs(n / o.n0 - 1).max() if np.all(np.isfinite(n)) else np.inf
        assert (dev > 1.0) if lagged else (dev < 1e-3)
