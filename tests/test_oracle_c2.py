"""The energy source of Eq. C2eq at constant T in the FP64 oracle, pinned to
what it must satisfy: no mass or momentum, zero for a uniform bulk and for a
transverse wave (mirror points cancel), and the long-wave limit
C2 -> -kT sigma^3 (4 pi / 6) g2 n^2 div u, the first moment of the shell
integral for a slowly varying velocity."""
import math

import numpy as np


def test_c2_source_adds_no_mass_or_momentum(oracle_mod):
    """One step from the same state with and without the source: the totals
    agree to rounding (the source is sum-free and has no first moment)."""
    from paper_0712_2247_gb300 import inputs

    out = {}
    for c2 in (False, True):
        o = oracle_mod.Oracle(12, 10, 8, 4, 0.2, 0.9, zper=True, seed=None, c2=c2)
        rho, u = inputs.random_fields((8, 10, 12), o.n0, 7, amp=0.05, uamp=1e-2)
        o.init_fields(rho.astype(np.float64), u.astype(np.float64))
        o.step(1)
        n, u = o.moments()
        out[c2] = (n.sum(), (u * n).sum(axis=(1, 2, 3)), n)
    assert abs(out[True][0] / out[False][0] - 1) < 1e-14
    assert np.abs(out[True][1] - out[False][1]).max() < 1e-15 * out[False][0]
    assert np.abs(out[True][2] - out[False][2]).max() > 1e-12 * out[False][2].max()  # the source acted


def test_c2_vanishes_for_uniform_bulk_and_transverse_wave(oracle_mod):
    o = oracle_mod.Oracle(16, 16, 16, 4, 0.25, 0.8, zper=True, seed=None, c2=True)
    n0 = o.n0
    o.init_fields(np.full((16, 16, 16), n0), np.stack([np.full((16, 16, 16), 1e-3)] + [np.zeros((16, 16, 16))] * 2))
    assert np.abs(o.c2_field()).max() < 1e-18
    x = np.arange(64)
    t = oracle_mod.Oracle(64, 1, 1, 4, 0.25, 0.8, zper=True, seed=None, c2=True)
    u = np.zeros((3, 1, 1, 64))
    u[1, 0, 0] = 1e-3 * np.sin(2 * math.pi * x / 64)
    t.init_fields(np.full((1, 1, 64), t.n0), u)
    assert np.abs(t.c2_field()).max() < 1e-18


def test_c2_long_wave_limit(oracle_mod):
    L, s, eta = 256, 4, 0.1
    o = oracle_mod.Oracle(L, 1, 1, s, eta, 0.9, zper=True, seed=None, c2=True)
    x = np.arange(L)
    k, eps = 2 * math.pi / L, 1e-4
    u = np.zeros((3, 1, 1, L))
    u[0, 0, 0] = eps * np.sin(k * x)
    o.init_fields(np.full((1, 1, L), o.n0), u)
    C = o.c2_field()[0, 0]
    ref = -(1 / 3) * s ** 3 * 4 * math.pi * oracle_mod.g2(eta) * o.n0 ** 2 * eps * k * np.cos(k * x) / 6
    # O((k sigma)^2) corrections (k sigma = 0.1) and the interpolation
    assert np.abs(C - ref).max() < 3e-3 * np.abs(ref).max()
