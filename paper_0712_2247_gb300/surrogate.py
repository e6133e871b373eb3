"""Learned warm start for the slit ensemble.

A perceptron maps a slit's parameters (H/sigma, eta, log10 F, tau) to its
steady profiles n(z) and u_x(z), z < H <= HMAX (masked beyond H). Its only
use is to seed the populations (equilibrium of the predicted profiles); the
lattice Boltzmann iteration then runs to the same residual criterion as a
cold start, so the network changes the starting point, never the result.

Training data are steady profiles that the method itself produces. The
steady state of a slit with periodic lateral boundaries is x,y-uniform, so
the profiles are generated on thin 4x4xH slits (the thin-grid and tiled
kernels are bit-identical on x,y-uniform states).

Targets are scaled to O(1): n(z)/n0 and u_x(z)/(F H^2/(8 nu)), with the
kinematic viscosity nu = c_s^2 (tau - 1/2), c_s^2 = 1/3 (Section 2, the BGK
relaxation and its viscosity). The steady profiles of a slit between two
identical walls are mirror-symmetric about its centre, so the network
predicts each profile from a wall to the centre: output j of the n block and
of the u_x block is the value at distance j from the nearest wall, for
j < ceil(H/2) (the rest is masked). The layering next to a wall then sits on
the same outputs for every width H.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import time
from dataclasses import dataclass
from typing import Optional

import numpy as np

from . import inputs, lbif
from .mlp import MLP

HMAX = 80
NFEAT = 4


def raw_features(H, eta, F, tau, sigma):
    return np.stack([np.asarray(H, float) / sigma, np.asarray(eta, float), np.log10(np.asarray(F, float)),
                     np.asarray(tau, float)], axis=1)


@dataclass
class Scaling:
    """Zero-mean, unit-variance scaling of the raw features (fitted on the training set)."""
    mean: np.ndarray
    std: np.ndarray

    @classmethod
    def fit(cls, raw):
        return cls(raw.mean(axis=0), raw.std(axis=0) + 1e-12)

    def __call__(self, raw):
        return ((raw - self.mean) / self.std).astype(np.float32)


def nu(tau):
    return (np.asarray(tau, float) - 0.5) / 3.0


def u_ref(H, F, tau):
    return np.asarray(F, float) * np.asarray(H, float) ** 2 / (8.0 * nu(tau))


def n0_of(eta, sigma):
    return 6.0 * np.asarray(eta, float) / (math.pi * sigma ** 3)


def fold(h: int):
    """Distance from the nearest wall of the planes z = 0..h-1."""
    z = np.arange(h)
    return np.minimum(z, h - 1 - z)


def encode(n_z, ux_z, p: inputs.Ensemble, hmax: int = HMAX):
    """Profiles (slits x >= H) -> targets (slits x 2 hmax) and mask. The two
    mirror halves are averaged (they agree up to rounding)."""
    ns = len(p.H)
    T = np.zeros((ns, 2 * hmax), np.float32)
    M = np.zeros((ns, 2 * hmax), np.float32)
    n0 = n0_of(p.eta, p.sigma)
    ur = u_ref(p.H, p.F, p.tau)
    for s in range(ns):
        h = int(p.H[s])
        m = (h + 1) // 2
        n = np.asarray(n_z[s, :h], np.float64)
        u = np.asarray(ux_z[s, :h], np.float64)
        T[s, :m] = 0.5 * (n[:m] + n[::-1][:m]) / n0[s]
        T[s, hmax:hmax + m] = 0.5 * (u[:m] + u[::-1][:m]) / ur[s]
        M[s, :m] = 1.0
        M[s, hmax:hmax + m] = 1.0
    return T, M


def decode(Y, p: inputs.Ensemble, hmax: int = HMAX):
    """Network outputs -> profiles n_z, ux_z (slits x hmax, zero beyond H)."""
    Y = np.asarray(Y, np.float64)
    ns = len(p.H)
    n0 = n0_of(p.eta, p.sigma)
    ur = u_ref(p.H, p.F, p.tau)
    n_z = np.zeros((ns, hmax), np.float32)
    ux_z = np.zeros((ns, hmax), np.float32)
    for s in range(ns):
        h = int(p.H[s])
        j = fold(h)
        n = np.maximum(Y[s, j], 0.05)  # a density stays positive
        # The dynamics conserve mass, so the seed must carry the slit's mass
        # n0 H (its mean packing fraction eta); otherwise the run converges to
        # the steady state of a different slit.
        n_z[s, :h] = n * (h / n.sum()) * n0[s]
        ux_z[s, :h] = Y[s, hmax + j] * ur[s]
    return n_z, ux_z


def subset(p: inputs.Ensemble, idx) -> inputs.Ensemble:
    return inputs.Ensemble(p.H[idx], p.eta[idx], p.F[idx], p.tau[idx], p.sigma, p.nx, p.ny)


def steady_profiles(p: inputs.Ensemble, nx: int = 4, ny: int = 4, tol: float = 1e-8,
                    max_steps: int = 400000, check_every: int = 100, patience: int = 30,
                    chunk: int = 4096, storage: int = lbif.STORE_F32, seeds=None, log=None):
    """Run every slit from a cold uniform start (or from seed profiles) to the
    residual criterion; returns profiles, steps per slit, best residuals, wall time."""
    ns = len(p.H)
    hmax = int(p.H.max())
    n_z = np.zeros((ns, hmax))
    ux_z = np.zeros((ns, hmax))
    steps = np.zeros(ns, np.int64)
    res = np.zeros(ns)
    wall = 0.0
    for a in range(0, ns, chunk):
        b = min(ns, a + chunk)
        e = lbif.Ensemble(p.H[a:b], p.eta[a:b], p.F[a:b], p.tau[a:b], p.sigma, nx, ny,
                          storage=storage, noise=0.0)
        try:
            import torch

            torch.cuda.synchronize()
            t0 = time.perf_counter()
            if seeds is not None:
                e.seed(seeds[0][a:b], seeds[1][a:b])
            st, r = e.run(tol=tol, max_steps=max_steps, check_every=check_every, patience=patience,
                          return_residual=True)
            torch.cuda.synchronize()
            wall += time.perf_counter() - t0
            nn, uu = e.slit_profiles(hmax)
        finally:
            e.close()
        n_z[a:b], ux_z[a:b], steps[a:b], res[a:b] = nn, uu, st, r
        if log:
            log(f"slits {a}..{b}: steps max {st.max()} mean {st[st > 0].mean() if (st > 0).any() else 0:.0f} "
                f"not converged {(st < 0).sum()}")
    return n_z, ux_z, steps, res, wall


def _cosine(step, total, lr_max, lr_min):
    return lr_min + 0.5 * (lr_max - lr_min) * (1.0 + math.cos(math.pi * min(step, total) / total))


def train(net: MLP, X, T, M, steps: int = 6000, batch: int = 512, lr_max: float = 2e-3,
          lr_min: float = 2e-5, seed: int = 4, log=None, log_every: int = 500):
    """Adam on minibatches (a fresh permutation every epoch, uploaded as one
    contiguous block); every product runs on the tensor cores."""
    import torch

    rng = np.random.default_rng(seed)
    ns = X.shape[0]
    batch = min(batch, ns, net.max_batch)
    losses = []
    k = 0
    while k < steps:
        perm = rng.permutation(ns)
        Xd = torch.from_numpy(np.ascontiguousarray(X[perm])).cuda()
        Td = torch.from_numpy(np.ascontiguousarray(T[perm])).cuda()
        Md = torch.from_numpy(np.ascontiguousarray(M[perm])).cuda()
        for a in range(0, ns - batch + 1, batch):
            if k >= steps:
                break
            lr = _cosine(k, steps, lr_max, lr_min)
            loss = net.train_step(Xd[a:a + batch], Td[a:a + batch], Md[a:a + batch], lr=lr)
            losses.append(loss)
            if log and (k % log_every == 0 or k == steps - 1):
                log(f"step {k} lr {lr:.2e} loss {loss:.3e}")
            k += 1
    return np.asarray(losses)


def predict(net: MLP, scaling: Scaling, p: inputs.Ensemble, hmax: int = HMAX):
    X = scaling(raw_features(p.H, p.eta, p.F, p.tau, p.sigma))
    Y = np.concatenate([net.forward(np.ascontiguousarray(X[a:a + net.max_batch]))
                        for a in range(0, len(X), net.max_batch)])
    return decode(Y, p, hmax)


def profile_error(a_n, a_u, b_n, b_u, H):
    """Per slit max|a - b| / max|b| over z < H for n and u_x."""
    en = np.zeros(len(H))
    eu = np.zeros(len(H))
    for s, h in enumerate(H):
        h = int(h)
        en[s] = np.abs(a_n[s, :h] - b_n[s, :h]).max() / np.abs(b_n[s, :h]).max()
        eu[s] = np.abs(a_u[s, :h] - b_u[s, :h]).max() / np.abs(b_u[s, :h]).max()
    return en, eu


def warm_vs_cold(net: MLP, scaling: Scaling, p: inputs.Ensemble, nx: int = 32, ny: int = 32,
                 tol: float = 1e-8, max_steps: int = 400000, patience: int = 10, log=None):
    """Same held-out slits from a cold uniform start and from the network's
    prediction, both run to the residual criterion on the GPU."""
    import torch

    torch.cuda.synchronize()
    t0 = time.perf_counter()
    seeds = predict(net, scaling, p)
    t_pred = time.perf_counter() - t0
    cn, cu, cs, cr, cw = steady_profiles(p, nx, ny, tol, max_steps, patience=patience, chunk=len(p.H), log=log)
    wn, wu, ws, wr, ww = steady_profiles(p, nx, ny, tol, max_steps, patience=patience, chunk=len(p.H),
                                         seeds=seeds, log=log)
    h = int(p.H.max())
    en, eu = profile_error(wn, wu, cn, cu, p.H)
    sn, su = profile_error(seeds[0][:, :h], seeds[1][:, :h], cn, cu, p.H)
    ok = (cs > 0) & (ws > 0)
    both = (cr < tol) & (wr < tol)
    return {
        "slits": int(len(p.H)), "grid": f"{nx}x{ny}xH", "tol": tol,
        "cold": {"wall_s": cw, "steps_mean": float(cs[cs > 0].mean()), "steps_max": int(cs.max()),
                 "not_converged": int((cs <= 0).sum())},
        "warm": {"wall_s": ww + t_pred, "predict_s": t_pred, "steps_mean": float(ws[ws > 0].mean()),
                 "steps_max": int(ws.max()), "not_converged": int((ws <= 0).sum())},
        "wall_speedup": cw / (ww + t_pred),
        "both_converged": int(both.sum()),
        "steps_ratio_mean": float((cs[ok] / ws[ok]).mean()) if ok.any() else None,
        "final_profile_diff": {"n_max": float(en.max()), "ux_max": float(eu.max()),
                               "n_max_both_below_tol": float(en[both].max()) if both.any() else None,
                               "ux_max_both_below_tol": float(eu[both].max()) if both.any() else None},
        "per_slit": {"H": p.H.tolist(), "cold_steps": cs.tolist(), "warm_steps": ws.tolist(),
                     "cold_res": cr.tolist(), "warm_res": wr.tolist(), "diff_n": en.tolist(),
                     "diff_ux": eu.tolist()},
        "prediction_error": {"n_median": float(np.median(sn)), "ux_median": float(np.median(su)),
                             "n_max": float(sn.max()), "ux_max": float(su.max())},
    }


def main(argv=None):
    ap = argparse.ArgumentParser(description="train the warm-start network and compare warm and cold starts")
    ap.add_argument("--train", type=int, default=20000, help="training slits (thin 4x4xH)")
    ap.add_argument("--heldout", type=int, default=512)
    ap.add_argument("--steps", type=int, default=20000, help="Adam steps")
    ap.add_argument("--batch", type=int, default=1024)
    ap.add_argument("--cache", default=None, help="directory for the generated profiles and weights")
    ap.add_argument("--eval-nx", type=int, default=32)
    ap.add_argument("--max-steps", type=int, default=400000)
    ap.add_argument("--out", default=None)
    a = ap.parse_args(argv)
    log = lambda s: print(s, flush=True)

    ptr = inputs.ensemble(a.train, seed=4)
    data = os.path.join(a.cache, f"steady_{a.train}.npz") if a.cache else None
    if data and os.path.exists(data):
        z = np.load(data)
        n_z, ux_z, steps, res, gen_wall = z["n_z"], z["ux_z"], z["steps"], z["res"], float(z["wall"])
    else:
        n_z, ux_z, steps, res, gen_wall = steady_profiles(ptr, log=log)
        if data:
            os.makedirs(a.cache, exist_ok=True)
            np.savez(data, n_z=n_z, ux_z=ux_z, steps=steps, res=res, wall=gen_wall)
    use = np.nonzero(steps != -2)[0]  # diverged slits carry no profile
    raw = raw_features(ptr.H, ptr.eta, ptr.F, ptr.tau, ptr.sigma)
    scaling = Scaling.fit(raw[use])
    T, M = encode(n_z, ux_z, ptr)
    net = MLP(NFEAT, 256, 3, 2 * HMAX, max_batch=max(a.batch, 1024), seed=4)
    t0 = time.perf_counter()
    losses = train(net, scaling(raw[use]), T[use], M[use], steps=a.steps, batch=a.batch, log=log)
    train_wall = time.perf_counter() - t0
    phe = inputs.ensemble(a.heldout, seed=5, nx=a.eval_nx, ny=a.eval_nx)
    out = {
        "train": {"slits": a.train, "generation_wall_s": gen_wall, "not_converged": int((steps < 0).sum()),
                  "steps_mean": float(steps[steps > 0].mean()), "adam_steps": a.steps, "batch": a.batch,
                  "train_wall_s": train_wall, "loss_first": float(losses[0]), "loss_last": float(losses[-50:].mean())},
        "eval": warm_vs_cold(net, scaling, phe, a.eval_nx, a.eval_nx, max_steps=a.max_steps, log=log),
    }
    if a.cache:
        np.savez(os.path.join(a.cache, "weights.npz"), params=net.get_params(), mean=scaling.mean, std=scaling.std)
    s = json.dumps(out)
    print(s)
    if a.out:
        with open(a.out, "w") as f:
            f.write(s + "\n")


if __name__ == "__main__":
    main()
