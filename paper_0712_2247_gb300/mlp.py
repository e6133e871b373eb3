"""Binding of the warm-start network (``lbif_mlp_*`` in ``include/lbif.h``).

Argument marshalling and parameter initialisation only; the forward pass,
back-propagation and Adam run in the CUDA kernels of ``liblbif.so`` (products
on the tensor cores, BF16 operands, FP32 accumulation). Arrays are numpy
float32 (host) or contiguous torch float32 CUDA tensors (device).
"""
from __future__ import annotations

import ctypes
import math
from typing import Optional

import numpy as np

from . import lbif

_vp, _i32, _i64, _f32, _f64 = ctypes.c_void_p, ctypes.c_int32, ctypes.c_int64, ctypes.c_float, ctypes.c_double
_pd = ctypes.POINTER(ctypes.c_double)

SIGNATURES = {
    "lbif_mlp_create": (_i32, [ctypes.POINTER(_vp), _i32, _i32, _i32, _i32, _i32, _vp]),
    "lbif_mlp_num_params": (_i64, [_vp]),
    "lbif_mlp_set_params": (_i32, [_vp, _vp]),
    "lbif_mlp_get_params": (_i32, [_vp, _vp]),
    "lbif_mlp_forward": (_i32, [_vp, _vp, _i32, _vp, _i32]),
    "lbif_mlp_gradients": (_i32, [_vp, _vp, _vp, _vp, _i32, _vp, _pd, _i32]),
    "lbif_mlp_train_step": (_i32, [_vp, _vp, _vp, _vp, _i32, _f32, _f32, _f32, _f32, _pd, _i32]),
    "lbif_mlp_destroy": (_i32, [_vp]),
    "lbif_mlp_last_error": (ctypes.c_char_p, [_vp]),
}


def load_library():
    lib = lbif.load_library()
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


def layer_shapes(nin, hidden, nhidden, nout):
    dims = [nin] + [hidden] * nhidden + [nout]
    return [(dims[i + 1], dims[i]) for i in range(len(dims) - 1)]


def init_params(nin=4, hidden=256, nhidden=3, nout=160, seed=0):
    """Flat float32 parameters: W uniform in +-sqrt(3/fan_in) (unit-variance
    pre-activations for unit-variance inputs), b = 0."""
    rng = np.random.default_rng(seed)
    out = []
    for o, i in layer_shapes(nin, hidden, nhidden, nout):
        a = math.sqrt(3.0 / i)
        out.append(rng.uniform(-a, a, size=(o, i)).ravel())
        out.append(np.zeros(o))
    return np.concatenate(out).astype(np.float32)


class MLP:
    """nin -> nhidden x hidden (GELU) -> nout perceptron trained on the GPU."""

    def __init__(self, nin: int = 4, hidden: int = 256, nhidden: int = 3, nout: int = 160,
                 max_batch: int = 4096, seed: int = 0, stream: Optional[int] = None):
        self._lib = load_library()
        h = ctypes.c_void_p()
        rc = self._lib.lbif_mlp_create(ctypes.byref(h), nin, hidden, nhidden, nout, max_batch, stream)
        if rc != 0:
            raise lbif.LbifError(rc, self._lib.lbif_mlp_last_error(None).decode())
        self._h = h
        self.nin, self.hidden, self.nhidden, self.nout, self.max_batch = nin, hidden, nhidden, nout, max_batch
        self.shapes = layer_shapes(nin, hidden, nhidden, nout)
        self.num_params = int(self._lib.lbif_mlp_num_params(h))
        self.set_params(init_params(nin, hidden, nhidden, nout, seed))

    def _check(self, rc):
        if rc != 0:
            raise lbif.LbifError(rc, self._lib.lbif_mlp_last_error(self._h).decode())

    def set_params(self, p):
        p = np.ascontiguousarray(p, dtype=np.float32)
        if p.size != self.num_params:
            raise ValueError(f"MLP: {p.size} parameters where {self.num_params} are needed")
        self._check(self._lib.lbif_mlp_set_params(self._h, p.ctypes.data))

    def get_params(self):
        p = np.empty(self.num_params, np.float32)
        self._check(self._lib.lbif_mlp_get_params(self._h, p.ctypes.data))
        return p

    def _args(self, X, *rest):
        """Host/device side and batch of X (batch x nin) and of the targets and
        masks (batch x nout); wrong shapes or mixed sides raise."""
        dev = lbif._on_device(X, *rest)
        b = X.shape[0]
        if tuple(X.shape) != (b, self.nin):
            raise ValueError(f"MLP: inputs of shape {tuple(X.shape)}, need (batch, {self.nin})")
        for a in rest:
            if tuple(a.shape) != (b, self.nout):
                raise ValueError(f"MLP: array of shape {tuple(a.shape)}, need ({b}, {self.nout})")
        return dev, b

    def forward(self, X):
        dev, b = self._args(X)
        if dev:
            import torch

            Y = torch.empty((b, self.nout), dtype=torch.float32, device=X.device)
        else:
            Y = np.empty((b, self.nout), np.float32)
        self._check(self._lib.lbif_mlp_forward(self._h, lbif._ptr(X), b, lbif._ptr(Y), dev))
        return Y

    def gradients(self, X, T, mask):
        """Loss and its gradient (flat float32, host array or device tensor like X)."""
        dev, b = self._args(X, T, mask)
        if dev:
            import torch

            g = torch.empty(self.num_params, dtype=torch.float32, device=X.device)
        else:
            g = np.empty(self.num_params, np.float32)
        loss = ctypes.c_double()
        self._check(self._lib.lbif_mlp_gradients(self._h, lbif._ptr(X), lbif._ptr(T), lbif._ptr(mask), b,
                                                 lbif._ptr(g), ctypes.byref(loss), dev))
        return loss.value, g

    def train_step(self, X, T, mask, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
        dev, b = self._args(X, T, mask)
        loss = ctypes.c_double()
        self._check(self._lib.lbif_mlp_train_step(self._h, lbif._ptr(X), lbif._ptr(T), lbif._ptr(mask), b,
                                                  lr, beta1, beta2, eps, ctypes.byref(loss), dev))
        return loss.value

    def close(self):
        if getattr(self, "_h", None) and self._h.value:
            self._lib.lbif_mlp_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
