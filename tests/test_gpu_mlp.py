"""Parity of the tensor-core warm-start network with the FP64 oracle.

The device rounds every product operand (layer inputs, weights, propagated
errors) to bfloat16 and accumulates in FP32; ``oracle.mlp`` with bf16=True
rounds the same operands and accumulates in FP64. The remaining differences:
FP32 accumulation over K <= 256 terms (relative error ~1e-5 of the sum of
|terms|), and activations whose FP32 and FP64 pre-activations round to
neighbouring bfloat16 values (one bfloat16 ulp, 2^-8 relative, on a few
elements). Tolerances below are set from those two effects.
"""
import numpy as np
import pytest

from oracle import mlp as omlp

pytestmark = pytest.mark.gpu

CASES = [  # nin, hidden, nhidden, nout, batch
    (4, 256, 3, 160, 300),   # production shape, ragged batch (3 row tiles)
    (4, 64, 1, 37, 16),      # ragged output width, single tile
    (7, 144, 2, 200, 129),   # ragged input width and batch just over one tile
    (4, 256, 3, 160, 1),     # one row
]


def _data(nin, nout, batch, seed):
    rng = np.random.default_rng(seed)
    X = rng.standard_normal((batch, nin)).astype(np.float32)
    T = (0.5 * rng.standard_normal((batch, nout))).astype(np.float32)
    M = (rng.random((batch, nout)) < 0.8).astype(np.float32)
    return X, T, M


@pytest.fixture(scope="module")
def mlp_mod():
    from paper_0712_2247_gb300 import mlp

    return mlp


@pytest.mark.parametrize("nin,hidden,nhidden,nout,batch", CASES)
def test_forward_matches_oracle(mlp_mod, nin, hidden, nhidden, nout, batch):
    net = mlp_mod.MLP(nin, hidden, nhidden, nout, max_batch=512, seed=1)
    p = net.get_params()
    p[-nout:] = np.linspace(-0.3, 0.3, nout, dtype=np.float32)  # nonzero output bias
    net.set_params(p)
    X, _, _ = _data(nin, nout, batch, 2)
    Y = net.forward(X)
    shapes = omlp.layer_shapes(nin, hidden, nhidden, nout)
    Yb, _ = omlp.forward(p.astype(np.float64), X, shapes, bf16=True)
    scale = np.abs(Yb).max()
    err = np.abs(Y - Yb)
    assert err.max() <= 2e-3 * scale, (err.max(), scale)
    assert np.median(err) <= 1e-4 * scale
    # the exact FP64 network differs only by the bfloat16 operand rounding
    Y64, _ = omlp.forward(p.astype(np.float64), X, shapes, bf16=False)
    assert np.abs(Y - Y64).max() <= 3e-2 * np.abs(Y64).max()
    net.close()


@pytest.mark.parametrize("nin,hidden,nhidden,nout,batch", CASES)
def test_device_forward_equals_host_forward(mlp_mod, nin, hidden, nhidden, nout, batch):
    """Device arrays: the last product writes the caller's (batch x nout)
    array itself, rows past the batch untouched; the same products as the
    host path, so the same bits. A forward after a training step (which keeps
    the back-propagation copies) gives the same bits as one before."""
    torch = pytest.importorskip("torch")
    net = mlp_mod.MLP(nin, hidden, nhidden, nout, max_batch=512, seed=6)
    X, T, M = _data(nin, nout, batch, 7)
    Yh = net.forward(X)
    Xd = torch.from_numpy(X).cuda()
    guard = torch.full((batch + 3, nout), 7.0, dtype=torch.float32, device="cuda")
    Yd = net.forward(Xd)
    assert np.array_equal(Yd.cpu().numpy(), Yh)
    # the device entry writes exactly batch rows into a caller's view
    lib = net._lib
    rc = lib.lbif_mlp_forward(net._h, Xd.data_ptr(), batch, guard.data_ptr(), 1)
    assert rc == 0
    g = guard.cpu().numpy()
    assert np.array_equal(g[:batch], Yh) and np.all(g[batch:] == 7.0)
    net.gradients(X, T, M)
    assert np.array_equal(net.forward(X), Yh)
    net.close()


@pytest.mark.parametrize("nin,hidden,nhidden,nout,batch", CASES)
def test_gradients_match_oracle(mlp_mod, nin, hidden, nhidden, nout, batch):
    net = mlp_mod.MLP(nin, hidden, nhidden, nout, max_batch=512, seed=3)
    p = net.get_params()
    X, T, M = _data(nin, nout, batch, 4)
    loss, g = net.gradients(X, T, M)
    shapes = omlp.layer_shapes(nin, hidden, nhidden, nout)
    lo, go = omlp.loss_and_grads(p.astype(np.float64), X, T, M, shapes, bf16=True)
    assert abs(loss - lo) <= 1e-4 * lo
    k = 0
    for o, i in shapes:  # per weight block and per bias block
        for n in (o * i, o):
            a, b = g[k:k + n].astype(np.float64), go[k:k + n]
            assert np.linalg.norm(a - b) <= 5e-3 * np.linalg.norm(b) + 1e-12, (k, n)
            k += n
    assert k == g.size
    net.close()


def test_adam_step_matches_oracle(mlp_mod):
    net = mlp_mod.MLP(4, 256, 3, 160, max_batch=256, seed=5)
    p0 = net.get_params()
    X, T, M = _data(4, 160, 200, 6)
    _, g = net.gradients(X, T, M)
    net.train_step(X, T, M, lr=1e-3)
    p1 = net.get_params()
    pe, _, _ = omlp.adam_step(p0.astype(np.float64), g.astype(np.float64), 0.0, 0.0, 1, 1e-3)
    # one Adam step moves every parameter by lr g/(|g| + eps); FP32 update arithmetic
    assert np.abs(p1 - pe).max() <= 1e-3 * 1e-3 + 1e-7
    net.close()


def test_training_fits_a_smooth_map(mlp_mod):
    """Adam on the device drives the loss of a smooth 4 -> 160 map down."""
    import torch

    rng = np.random.default_rng(7)
    X = rng.uniform(-1, 1, (1024, 4)).astype(np.float32)
    z = np.linspace(0, 1, 160)
    T = (np.sin(np.pi * z[None, :] * (1 + X[:, :1])) * X[:, 1:2] + 0.3 * X[:, 2:3] * z).astype(np.float32)
    M = np.ones_like(T)
    net = mlp_mod.MLP(4, 256, 3, 160, max_batch=1024, seed=8)
    Xd, Td, Md = (torch.from_numpy(a).cuda() for a in (X, T, M))
    first = net.train_step(Xd, Td, Md, lr=2e-3)
    for _ in range(400):
        last = net.train_step(Xd, Td, Md, lr=2e-3)
    assert np.isfinite(last) and last < first / 30, (first, last)
    # host and device entry points agree
    Yh = net.forward(X)
    Yd = net.forward(Xd).cpu().numpy()
    assert np.array_equal(Yh, Yd)
    net.close()
