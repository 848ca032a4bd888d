"""FP64 numpy reference of the warm-start U-Net (test infrastructure).

The paper has no network; this is the plain definition the GPU training and
inference kernels are checked against (forward values and every gradient).
Tensors are NHWC float64.  Layer semantics:

  conv3x3(x, W, b): zero padding 1, stride 1,
      y[n, h, w, co] = b[co] + sum_{dh, dw in -1..1} sum_ci x[n, h+dh, w+dw, ci] W[dh+1, dw+1, ci, co]
  relu(x) = max(x, 0)
  pool(x):  2 x 2 average
  up(x):    2 x 2 nearest-neighbour copy
  cat(a, b): channels of a, then channels of b
  conv1x1(x, W, b) = b + x W
  loss = mean((pred - target)^2 * channel_weight) over all elements

Network with level channels c0..c3:
  e0 = relu(conv(relu(conv(x))))                      c0, H x W
  e1 = relu(conv(relu(conv(pool(e0)))))               c1, H/2
  e2 = relu(conv(relu(conv(pool(e1)))))               c2, H/4
  b  = relu(conv(relu(conv(pool(e2)))))               c3, H/8
  d2 = relu(conv(relu(conv(cat(up(b), e2)))))         c2
  d1 = relu(conv(relu(conv(cat(up(d2), e1)))))        c1
  d0 = relu(conv(relu(conv(cat(up(d1), e0)))))        c0
  out = conv1x1(d0)                                   cout
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, W, b):
    n, H, Wd, ci = x.shape
    co = W.shape[3]
    xp = np.zeros((n, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    y = np.broadcast_to(b, (n, H, Wd, co)).copy()
    for dh in range(3):
        for dw in range(3):
            y += xp[:, dh:dh + H, dw:dw + Wd, :] @ W[dh, dw]
    return y


def conv3x3_backward(x, W, dy):
    """(dx, dW, db) of conv3x3 for upstream gradient dy."""
    n, H, Wd, ci = x.shape
    xp = np.zeros((n, H + 2, Wd + 2, ci))
    xp[:, 1:-1, 1:-1] = x
    dxp = np.zeros_like(xp)
    dW = np.zeros_like(W)
    for dh in range(3):
        for dw in range(3):
            win = xp[:, dh:dh + H, dw:dw + Wd, :]
            dW[dh, dw] = np.einsum("nhwc,nhwk->ck", win, dy)
            dxp[:, dh:dh + H, dw:dw + Wd, :] += dy @ W[dh, dw].T
    return dxp[:, 1:-1, 1:-1], dW, dy.sum(axis=(0, 1, 2))


def pool(x):
    n, H, W, c = x.shape
    return x.reshape(n, H // 2, 2, W // 2, 2, c).mean(axis=(2, 4))


def pool_backward(dy):
    return np.repeat(np.repeat(dy, 2, axis=1), 2, axis=2) / 4.0


def up(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up_backward(dy):
    n, H, W, c = dy.shape
    return dy.reshape(n, H // 2, 2, W // 2, 2, c).sum(axis=(2, 4))


def layer_shapes(cin, cout, ch):
    """(name, weight shape, bias length) of every layer, in order."""
    c0, c1, c2, c3 = ch
    spec = [("e0a", cin, c0), ("e0b", c0, c0), ("e1a", c0, c1), ("e1b", c1, c1),
            ("e2a", c1, c2), ("e2b", c2, c2), ("b_a", c2, c3), ("b_b", c3, c3),
            ("d2a", c3 + c2, c2), ("d2b", c2, c2), ("d1a", c2 + c1, c1), ("d1b", c1, c1),
            ("d0a", c1 + c0, c0), ("d0b", c0, c0)]
    out = [(name, (3, 3, a, b), b) for name, a, b in spec]
    out.append(("head", (1, 1, c0, cout), cout))
    return out


def init_params(cin, cout, ch, seed=0):
    rng = np.random.default_rng(seed)
    params = {}
    for name, shape, nb in layer_shapes(cin, cout, ch):
        fan_in = shape[0] * shape[1] * shape[2]
        params[name + ".W"] = rng.standard_normal(shape) * np.sqrt(2.0 / fan_in)
        params[name + ".b"] = 0.01 * rng.standard_normal(nb)
    return params


def forward(params, x, keep=False):
    cache = {}

    def block(name, inp):
        a = conv3x3(inp, params[name + "a.W"] if name != "b" else params["b_a.W"],
                    params[name + "a.b"] if name != "b" else params["b_a.b"])
        ra = np.maximum(a, 0)
        wb = params[name + "b.W"] if name != "b" else params["b_b.W"]
        bb = params[name + "b.b"] if name != "b" else params["b_b.b"]
        bo = conv3x3(ra, wb, bb)
        rb = np.maximum(bo, 0)
        cache[name] = (inp, a, ra, bo, rb)
        return rb

    e0 = block("e0", x)
    e1 = block("e1", pool(e0))
    e2 = block("e2", pool(e1))
    bt = block("b", pool(e2))
    d2 = block("d2", np.concatenate([up(bt), e2], axis=3))
    d1 = block("d1", np.concatenate([up(d2), e1], axis=3))
    d0 = block("d0", np.concatenate([up(d1), e0], axis=3))
    out = d0 @ params["head.W"][0, 0] + params["head.b"]
    cache["d0out"] = d0
    return (out, cache) if keep else out


def loss_and_grads(params, x, target, weight=None):
    """MSE loss and the gradient of every parameter (backpropagation)."""
    out, cache = forward(params, x, keep=True)
    wch = np.ones(out.shape[3]) if weight is None else np.asarray(weight, dtype=np.float64)
    diff = out - target
    loss = float(np.mean(diff ** 2 * wch))
    dout = 2.0 * diff * wch / diff.size
    g = {}
    d0 = cache["d0out"]
    g["head.W"] = np.einsum("nhwc,nhwk->ck", d0, dout)[None, None]
    g["head.b"] = dout.sum(axis=(0, 1, 2))
    dd0 = dout @ params["head.W"][0, 0].T

    def block_back(name, dout_b):
        inp, a, ra, bo, rb = cache[name]
        ka, kb = ("b_a", "b_b") if name == "b" else (name + "a", name + "b")
        dbo = dout_b * (bo > 0)
        dra, g[kb + ".W"], g[kb + ".b"] = conv3x3_backward(ra, params[kb + ".W"], dbo)
        da = dra * (a > 0)
        dinp, g[ka + ".W"], g[ka + ".b"] = conv3x3_backward(inp, params[ka + ".W"], da)
        return dinp

    c0 = cache["e0"][4].shape[3]
    c1 = cache["e1"][4].shape[3]
    c2 = cache["e2"][4].shape[3]
    dcat0 = block_back("d0", dd0)
    dup1, de0 = dcat0[..., :-c0], dcat0[..., -c0:]
    dcat1 = block_back("d1", up_backward(dup1))
    dup2, de1 = dcat1[..., :-c1], dcat1[..., -c1:]
    dcat2 = block_back("d2", up_backward(dup2))
    dupb, de2 = dcat2[..., :-c2], dcat2[..., -c2:]
    dpool2 = block_back("b", up_backward(dupb))
    de2 = de2 + pool_backward(dpool2)
    dpool1 = block_back("e2", de2)
    de1 = de1 + pool_backward(dpool1)
    dpool0 = block_back("e1", de1)
    de0 = de0 + pool_backward(dpool0)
    block_back("e0", de0)
    return loss, g
