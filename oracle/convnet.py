"""FP64 CPU oracle of the learned initial-guess network (test infrastructure only).

The network maps (u^0, log10 nu) on an H x W grid to the corrections u^n - u^0 of
all M levels (NHWC layout, channels last):

    z0 = conv(in, W0) ;  x = relu(z0)                       in: 2 channels
    per block b:  h = relu(conv(x, Wb1)) ;  x = x + conv(h, Wb2)
    out = conv(x, Wh)                                       M channels

Every conv is a 3 x 3 cross-correlation with zero padding and a bias. The loss is
the mean squared error over all outputs. Plain numpy in FP64: ``conv3x3`` is the
definition written out tap by tap, and the backward pass is the chain rule in the
same order. Pinned by ``tests/test_oracle_convnet.py`` against scipy's correlate
and against central finite differences of the loss.

Parameters travel as one flat vector, layer by layer: W [Cout][3][3][Cin] then
bias [Cout], in the order lift, (block conv 1, block conv 2) x blocks, head.
"""
from __future__ import annotations

import numpy as np


def layer_shapes(channels: int, blocks: int, levels: int, cin: int = 2):
    """(Cout, Cin) of every conv layer in order."""
    shapes = [(channels, cin)]
    for _ in range(blocks):
        shapes += [(channels, channels), (channels, channels)]
    shapes.append((levels, channels))
    return shapes


def unflatten(theta, shapes):
    out, o = [], 0
    for co, ci in shapes:
        n = co * 9 * ci
        W = theta[o:o + n].reshape(co, 3, 3, ci)
        o += n
        b = theta[o:o + co]
        o += co
        out.append((W, b))
    assert o == theta.size
    return out


def flatten(params):
    return np.concatenate([np.concatenate([W.ravel(), b.ravel()]) for W, b in params])


def conv3x3(x, W, b):
    """y[n,h,w,o] = b[o] + sum_{r,s,c} W[o,r,s,c] x[n,h+r-1,w+s-1,c] (zero outside)."""
    n, H, Wd, c = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((n, H, Wd, W.shape[0]))
    for r in range(3):
        for s in range(3):
            y += np.einsum("nhwc,oc->nhwo", xp[:, r:r + H, s:s + Wd, :], W[:, r, s, :])
    return y + b


def conv3x3_backward(x, W, dy):
    """Gradients of sum(dy * conv3x3(x, W, b)) with respect to x, W and b."""
    n, H, Wd, c = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for r in range(3):
        for s in range(3):
            dW[:, r, s, :] = np.einsum("nhwo,nhwc->oc", dy, xp[:, r:r + H, s:s + Wd, :])
            dxp[:, r:r + H, s:s + Wd, :] += np.einsum("nhwo,oc->nhwc", dy, W[:, r, s, :])
    db = dy.sum(axis=(0, 1, 2))
    return dxp[:, 1:-1, 1:-1, :], dW, db


def net_input(u0, lognu):
    """u0 [N, H, W], lognu [N] -> [N, H, W, 2]."""
    u0 = np.asarray(u0, dtype=np.float64)
    return np.stack([u0, np.broadcast_to(np.asarray(lognu, dtype=np.float64)[:, None, None], u0.shape)], axis=-1)


def forward(params, inp, keep=False):
    (W0, b0), blocks, (Wh, bh) = params[0], params[1:-1], params[-1]
    cache = {"inp": inp}
    z0 = conv3x3(inp, W0, b0)
    x = np.maximum(z0, 0.0)
    cache["x0"] = x
    xs, hs = [], []
    for k in range(0, len(blocks), 2):
        (W1, b1), (W2, b2) = blocks[k], blocks[k + 1]
        xs.append(x)
        h = np.maximum(conv3x3(x, W1, b1), 0.0)
        hs.append(h)
        x = x + conv3x3(h, W2, b2)
    cache["xs"], cache["hs"], cache["xl"] = xs, hs, x
    out = conv3x3(x, Wh, bh)
    return (out, cache) if keep else out


def loss_and_grad(params, inp, target):
    """MSE loss and its gradient with respect to every parameter (same structure as params)."""
    out, cache = forward(params, inp, keep=True)
    diff = out - target
    loss = float(np.mean(diff * diff))
    dout = 2.0 * diff / diff.size
    grads = [None] * len(params)
    (Wh, bh) = params[-1]
    dx, dWh, dbh = conv3x3_backward(cache["xl"], Wh, dout)
    grads[-1] = (dWh, dbh)
    nb = (len(params) - 2) // 2
    for blk in reversed(range(nb)):
        (W1, b1), (W2, b2) = params[1 + 2 * blk], params[2 + 2 * blk]
        x_in, h = cache["xs"][blk], cache["hs"][blk]
        dh, dW2, db2 = conv3x3_backward(h, W2, dx)          # x_out = x_in + conv(h)
        dh = dh * (h > 0)
        dxi, dW1, db1 = conv3x3_backward(x_in, W1, dh)
        grads[1 + 2 * blk] = (dW1, db1)
        grads[2 + 2 * blk] = (dW2, db2)
        dx = dx + dxi
    dx = dx * (cache["x0"] > 0)
    _, dW0, db0 = conv3x3_backward(cache["inp"], params[0][0], dx)
    grads[0] = (dW0, db0)
    return loss, grads
