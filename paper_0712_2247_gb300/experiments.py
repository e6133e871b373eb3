"""The paper's two numerical experiments, run on the GPU path.

Shear viscosity (Sec. Numerical validation, the transverse-wave test of
Fig. 1): a small transverse velocity wave u_y = A sin(k x) in a periodic box
decays as exp(-nu k^2 t) in the hydrodynamic limit; the measured decay rate
gives the kinematic viscosity, the sum of the BGK part c_s^2 (tau - 1/2) and
the collisional part of the density-current term of Eq. LBHS.

Static slit profiles (Sec. Numerical validation, Fig. 2): a hard-sphere
fluid between two walls, no external field, run to equilibrium; its density
profile layers next to the walls. At equilibrium every plane's z momentum
balances: the flux through the interface z + 1/2,
  Pi(z+1/2) = c_s^2 (n(z) + n(z+1))/2 + (n u_z^2 (z) + n u_z^2 (z+1))/2
              + (F_z(z) - F_z(z+1))/4,
changes by F_z(z) from one interface to the next, and the unshifted velocity
is u_z = -F_z/(2n) (pre-collision momentum; the force adds F_z in the
collision). Both hold exactly in the discrete steady state.

Both only drive the C ABI (set fields, step, read moments and forces).
"""
from __future__ import annotations

import argparse
import json
import math
from typing import Optional

import numpy as np

from . import lbif

KT = 1.0 / 3.0


def g2_printed(eta):
    """Contact value as printed in Sec. Methods (the library's default form)."""
    return (1.0 - eta / 2.0 + eta * eta / 4.0) / (1.0 - eta) ** 3


def nu_closed_form(sigma, eta, tau):
    """Kinematic viscosity of the long-wave limit: BGK part plus the
    Longuet-Higgins-Pople collisional part (4 sqrt(pi)/15) sqrt(kT m) g2 n^2
    sigma^4 divided by the mass density m n (m = 1)."""
    n0 = 6.0 * eta / (math.pi * sigma ** 3)
    return KT * (tau - 0.5) + (4.0 * math.sqrt(math.pi) / 15.0) * math.sqrt(KT) * g2_printed(eta) * n0 * sigma ** 4


def _amplitude(g, L):
    _, u = g.moments()
    x = np.arange(L)
    return 2.0 / L * float(np.sum(u[1, 0, 0, :].astype(np.float64) * np.sin(2 * math.pi * x / L)))


def shear_decay(sigma: int, eta: float, tau: float, L: int = 128, amp: float = 1e-4,
                t0: int = 50, t1: Optional[int] = None, storage: int = lbif.STORE_F32):
    """Decay rate per step of a transverse wave of wavelength L (periodic
    L x 1 x 1 box; the state varies along x only). t1 defaults to the time at
    which the long-wave closed form predicts a decay by e^2."""
    k = 2 * math.pi / L
    if t1 is None:
        t1 = t0 + max(50, int(2.0 / (nu_closed_form(sigma, eta, tau) * k * k)))
    g = lbif.Slit(L, 1, 1, sigma, eta, tau, periodic_z=True, noise=0.0, storage=storage)
    try:
        x = np.arange(L)
        rho = np.full((1, 1, L), g.n0, np.float32)
        u = np.zeros((3, 1, 1, L), np.float32)
        u[1, 0, 0, :] = amp * np.sin(k * x)
        g.set_fields(rho, u)
        g.step(t0)
        a0 = _amplitude(g, L)
        g.step(t1 - t0)
        a1 = _amplitude(g, L)
    finally:
        g.close()
    rate = math.log(a0 / a1) / (t1 - t0)
    return {"sigma": sigma, "eta": eta, "n_star": 6 * eta / math.pi, "tau": tau, "L": L,
            "t0": t0, "t1": t1, "rate": rate, "nu": rate / (k * k),
            "nu_closed_form": nu_closed_form(sigma, eta, tau)}


def plane_balance(n, uz, fz):
    """Pi(z+1/2) - Pi(z-1/2) - F_z(z) over the interior planes (zero at a
    steady state; see the module docstring)."""
    pi = (KT * (n[:-1] + n[1:]) / 2 + (n[:-1] * uz[:-1] ** 2 + n[1:] * uz[1:] ** 2) / 2
          + (fz[:-1] - fz[1:]) / 4)
    return (pi[1:] - pi[:-1]) - fz[1:-1]


def static_profile(sigma: int, eta: float, tau: float, H: int, steps: int = 4000,
                   storage: int = lbif.STORE_F32):
    """Equilibrium profile of a 1 x 1 x H slit without external field from a
    uniform start; returns n(z)/n0, the plane momentum balance residual
    max|Pi(z+1/2) - Pi(z-1/2) - F_z| / max|F_z|, the deviation from
    u_z = -F_z/(2n), the mirror asymmetry and the final residual (relative
    change per step)."""
    g = lbif.Slit(1, 1, H, sigma, eta, tau, noise=0.0, storage=storage)
    try:
        g.step(steps - 100)
        n_prev, _, _ = g.profiles()
        g.step(100)
        n, _, _ = g.profiles()
        _, u = g.moments()
        F = g.forces()  # F / n0, shape (3, nz, ny, nx)
    finally:
        g.close()
    n0 = 6.0 * eta / (math.pi * sigma ** 3)
    fz = F[2, :, 0, 0].astype(np.float64) * n0
    uz = u[2, :, 0, 0].astype(np.float64)
    bal = np.abs(plane_balance(n, uz, fz)).max() / np.abs(fz).max()
    uzr = np.abs(uz + fz / (2 * n)).max() / np.abs(uz).max()
    return {"sigma": sigma, "eta": eta, "n_star": 6 * eta / math.pi, "H": H, "steps": steps,
            "n_over_n0": (n / n0).tolist(), "contact_over_n0": float(n[0] / n0),
            "force_balance": float(bal), "uz_relation": float(uzr),
            "mirror": float(np.abs(n - n[::-1]).max() / n.max()),
            "residual": float(np.linalg.norm(n - n_prev) / (100 * np.linalg.norm(n)))}


def poiseuille_profiles(n_stars, L_over_sigma, sigma: int = 8, tau: float = 0.8, F: float = 2.4e-6,
                        nx: int = 4, tol: float = 1e-8, max_steps: int = 400000, patience: int = 20,
                        storage: int = lbif.STORE_F32):
    """Steady streaming profiles of slits of width L = L_over_sigma sigma
    (one value or one per density) driven by a uniform field F along x
    (Sec. Numerical validation, Figs. 3 and 4), run together as one batched
    ensemble from a uniform start to the FP64 residual tol. Returns per slit
    n(z)/n0, u_x(z), the steps taken and the final residual."""
    n_stars = list(n_stars)
    Ls = L_over_sigma if hasattr(L_over_sigma, "__len__") else [L_over_sigma] * len(n_stars)
    H = np.array([int(round(l * sigma)) for l in Ls], np.int32)
    eta = np.array([math.pi * ns / 6.0 for ns in n_stars])
    e = lbif.Ensemble(H, eta, np.full(len(H), F), np.full(len(H), tau), sigma, nx, nx, storage=storage,
                      noise=0.0)
    try:
        steps, res = e.run(tol=tol, max_steps=max_steps, patience=patience, return_residual=True)
        n_z, ux_z = e.slit_profiles()
    finally:
        e.close()
    n0 = 6.0 * eta / (math.pi * sigma ** 3)
    out = []
    for s in range(len(H)):
        h = int(H[s])
        out.append({"n_star": n_stars[s], "L_over_sigma": Ls[s], "H": h, "steps": int(steps[s]),
                    "residual": float(res[s]), "n_over_n0": (n_z[s, :h] / n0[s]).tolist(),
                    "ux": ux_z[s, :h].tolist()})
    return out


def main(argv=None):
    ap = argparse.ArgumentParser(description="shear-viscosity and static-profile experiments")
    ap.add_argument("which", choices=["shear", "static"])
    ap.add_argument("--sigma", type=int, default=8)
    ap.add_argument("--tau", type=float, default=0.8)
    a = ap.parse_args(argv)
    import torch

    torch.cuda.init()
    if a.which == "shear":
        for eta in (0.05, 0.10, 0.15, 0.20, 0.25, 0.30):
            print(json.dumps(shear_decay(a.sigma, eta, a.tau)), flush=True)
    else:
        for n_star in (0.256, 0.512, 0.609):
            try:
                r = static_profile(a.sigma, math.pi * n_star / 6, a.tau, 5 * a.sigma)
                r.pop("n_over_n0")
            except lbif.LbifError as e:  # the explicit scheme's limit (a result, not a fault)
                r = {"sigma": a.sigma, "n_star": n_star, "diverged": str(e)}
            print(json.dumps(r), flush=True)


if __name__ == "__main__":
    main()
