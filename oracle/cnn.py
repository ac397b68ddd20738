"""Oracle of the learned initial guess (test infrastructure: only tests/,
__graft_entry__.smoke() and bench.py's CPU baseline may use it).

The network maps the last three steps' extracellular and transmembrane
potentials, sampled on the node grid of a structured slice, to the increments
of both potentials at the next step (the next step's solution X = (U, V));
added to the last state they give the initial guess of PCG (the paper's
method is unchanged: the guess only changes the iteration count).
Architecture: three 3 x 3 convolutions with zero padding ("same" size),
6 -> 32 -> 32 -> 2 channels, ReLU after the first two; loss: mean squared
error over all grid points and both output channels.

Everything here is plain FP64 numpy written from the definitions:
  conv:  out[i, j, o] = b[o] + sum_{c, ky, kx} W[o, c, ky, kx] x[i + ky - 1, j + kx - 1, c]
         (x = 0 outside the grid);
  loss:  L = (1/P) sum_p (y_p - t_p)^2 over the P grid points (and batch);
  back-propagation by the chain rule: dL/dy = 2 (y - t) / P, then for each
  layer dW = sum_p x_patch(p) dout(p), db = sum_p dout(p), and the input
  gradient is the correlation of dout with the flipped kernel.
An optional `rnd` function (e.g. rounding to BF16) is applied where a
reduced-precision implementation rounds: to the weights and to the inputs of
each layer; every sum is then exact-order-free FP64.
"""
from __future__ import annotations

import numpy as np

LAYERS = ((6, 32), (32, 32), (32, 2))


def init_params(seed: int, layers=LAYERS):
    """He-style random weights (normal, std sqrt(2 / (9 cin))) and zero biases."""
    rng = np.random.default_rng(seed)
    params = []
    for cin, cout in layers:
        W = rng.normal(0.0, np.sqrt(2.0 / (9 * cin)), size=(cout, cin, 3, 3))
        params.append((W, np.zeros(cout)))
    return params


def _pad(x):
    return np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))


def conv3x3(x, W, b):
    """x: (B, H, W, cin); W: (cout, cin, 3, 3); b: (cout,) -> (B, H, W, cout)."""
    B, H, Wd, _ = x.shape
    xp = _pad(x)
    out = np.broadcast_to(b, (B, H, Wd, W.shape[0])).astype(np.float64).copy()
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + H, kx:kx + Wd, :]
            out += patch @ W[:, :, ky, kx].T
    return out


def conv3x3_backward(x, W, dout):
    """Gradients of conv3x3 w.r.t. x, W and b for the output gradient dout."""
    B, H, Wd, _ = x.shape
    xp = _pad(x)
    dW = np.zeros_like(W, dtype=np.float64)
    dxp = np.zeros_like(xp, dtype=np.float64)
    for ky in range(3):
        for kx in range(3):
            patch = xp[:, ky:ky + H, kx:kx + Wd, :]
            dW[:, :, ky, kx] = np.einsum("bhwo,bhwc->oc", dout, patch)
            dxp[:, ky:ky + H, kx:kx + Wd, :] += dout @ W[:, :, ky, kx]
    db = dout.sum(axis=(0, 1, 2))
    return dxp[:, 1:H + 1, 1:Wd + 1, :], dW, db


def forward(params, x, rnd=None):
    """Network output (B, H, W, cout) and the per-layer inputs / pre-activations."""
    r = rnd if rnd is not None else (lambda a: a)
    a = x
    cache = []
    n = len(params)
    for k, (W, b) in enumerate(params):
        a_in = r(a)
        Wr = r(W)
        z = conv3x3(a_in, Wr, b)
        cache.append((a_in, Wr, z))
        a = np.maximum(z, 0.0) if k < n - 1 else z
    return a, cache


def loss_and_grads(params, x, target, rnd=None):
    """MSE loss over all outputs (target (B, H, W, cout)) and its gradients
    [(dW, db), ...] (same structure as params)."""
    y, cache = forward(params, x, rnd)
    P = y.size
    diff = y - target
    loss = float((diff * diff).sum() / P)
    g = (2.0 / P) * diff
    grads = [None] * len(params)
    for k in range(len(params) - 1, -1, -1):
        a_in, Wr, z = cache[k]
        if k < len(params) - 1:
            g = g * (z > 0.0)
        dx, dW, db = conv3x3_backward(a_in, Wr, g)
        grads[k] = (dW, db)
        g = dx
    return loss, grads


def round_bf16(a):
    """Round FP64 values to the nearest BF16 (ties to even) via FP32."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    u = (u + 0x7FFF + ((u >> 16) & 1)) & 0xFFFF0000
    return u.astype(np.uint32).view(np.float32).astype(np.float64)
