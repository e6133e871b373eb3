"""The trained warm start on the GPU: a network trained by the device kernels
on steady profiles that the method generates seeds held-out slits, which then
reach the same steady state in fewer steps than from a cold uniform start."""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _narrow(p, hmax, count, S, fmin=0.0):
    idx = np.nonzero((p.H <= hmax) & (p.F >= fmin))[0][:count]
    return S.subset(p, idx)


def test_trained_network_beats_cold_start():
    from paper_0712_2247_gb300 import inputs
    from paper_0712_2247_gb300 import surrogate as S
    from paper_0712_2247_gb300.mlp import MLP

    ptr = _narrow(inputs.ensemble(3000, seed=4, nx=4, ny=4), 32, 768, S)
    n_z, ux_z, steps, res, _ = S.steady_profiles(ptr, max_steps=60000)
    use = np.nonzero(steps != -2)[0]
    assert len(use) > 700
    raw = S.raw_features(ptr.H, ptr.eta, ptr.F, ptr.tau, ptr.sigma)
    sc = S.Scaling.fit(raw[use])
    T, M = S.encode(n_z, ux_z, ptr)
    net = MLP(4, 256, 3, 2 * S.HMAX, max_batch=512, seed=4)
    losses = S.train(net, sc(raw[use]), T[use], M[use], steps=2500, batch=256)
    assert losses[-20:].mean() < losses[0] / 100

    # held-out slits with F >= 1e-6: their u_x (>= 4e-5) is resolved well
    # enough in FP32 for the residual to reach 1e-8 from either start
    phe = _narrow(inputs.ensemble(800, seed=5, nx=8, ny=8), 32, 48, S, fmin=1e-6)
    r = S.warm_vs_cold(net, sc, phe, nx=8, ny=8, max_steps=60000)
    print({k: v for k, v in r.items() if k != "per_slit"})
    cs = np.array(r["per_slit"]["cold_steps"])
    ws = np.array(r["per_slit"]["warm_steps"])
    ok = (cs > 0) & (ws > 0)
    assert ok.sum() >= 24
    assert ws[ok].sum() < 0.75 * cs[ok].sum()
    assert r["prediction_error"]["n_median"] < 0.02
    # Both runs end at the same steady state, to the distance the residual
    # allows; u_x carries the FP32 rounding floor of the slit (~1e-8 absolute
    # against u_x of 4e-5 and up, over a few hundred steps of relaxation time).
    assert r["final_profile_diff"]["n_max_both_below_tol"] < 1e-5
    assert r["final_profile_diff"]["ux_max_both_below_tol"] < 5e-3
    net.close()
