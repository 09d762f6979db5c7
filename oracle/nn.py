"""FP64 reference of the warm-start network (test infrastructure only).

TEST INFRASTRUCTURE ONLY: the tests use it to check the CUDA network's
forward pass, gradients and optimiser step; the product path never imports
it.  Plain numpy in FP64, NHWC activations, weights [kh][kw][ci][co].

Network (the warm-start predictor of the workload description; the paper
has no network): a 4-level encoder-decoder with `base` channels at the top
level, doubling per level.
  level l encoder: conv3x3 -> ReLU -> conv3x3 -> ReLU   (l = 0..3, 2x2 average
                   pooling between levels)
  level l decoder: nearest 2x upsampling of level l+1, concatenation
                   [upsampled, skip_l] along channels, conv3x3 -> ReLU ->
                   conv3x3 -> ReLU   (l = 2, 1, 0)
  head:            conv1x1 to the outputs (no activation)
Loss: mean squared error over all output values.  Optimiser: Adam with
bias correction.
"""
from __future__ import annotations

import numpy as np


def conv3x3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} x[n,i+dy-1,j+dx-1,c] w[dy,dx,c,o] (zero padding)."""
    n, h, wd, c = x.shape
    xp = np.zeros((n, h + 2, wd + 2, c))
    xp[:, 1:-1, 1:-1, :] = x
    y = np.zeros((n, h, wd, w.shape[3]))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nijc,co->nijo", xp[:, dy:dy + h, dx:dx + wd, :], w[dy, dx])
    return y + b


def conv3x3_backward(x, w, gy):
    """Gradients of conv3x3 with respect to x, w and b."""
    n, h, wd, c = x.shape
    xp = np.zeros((n, h + 2, wd + 2, c))
    xp[:, 1:-1, 1:-1, :] = x
    gw = np.zeros_like(w)
    gxp = np.zeros_like(xp)
    for dy in range(3):
        for dx in range(3):
            gw[dy, dx] = np.einsum("nijc,nijo->co", xp[:, dy:dy + h, dx:dx + wd, :], gy)
            gxp[:, dy:dy + h, dx:dx + wd, :] += np.einsum("nijo,co->nijc", gy, w[dy, dx])
    return gxp[:, 1:-1, 1:-1, :], gw, gy.sum(axis=(0, 1, 2))


def conv1x1(x, w, b):
    return np.einsum("nijc,co->nijo", x, w) + b


def conv1x1_backward(x, w, gy):
    return np.einsum("nijo,co->nijc", gy, w), np.einsum("nijc,nijo->co", x, gy), gy.sum(axis=(0, 1, 2))


def pool2(x):
    n, h, w, c = x.shape
    return x.reshape(n, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def pool2_backward(gy):
    return np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2) * 0.25


def up2(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def up2_backward(gy):
    n, h, w, c = gy.shape
    return gy.reshape(n, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def layer_shapes(c_in=3, c_out=3, base=32, levels=4):
    """(name, kind, ci, co) of every layer, in the order of the parameters."""
    ch = [base * 2 ** l for l in range(levels)]
    out = []
    prev = c_in
    for l in range(levels):
        out.append((f"e{l}a", "c3", prev, ch[l]))
        out.append((f"e{l}b", "c3", ch[l], ch[l]))
        prev = ch[l]
    for l in range(levels - 2, -1, -1):
        out.append((f"d{l}a", "c3", ch[l + 1] + ch[l], ch[l]))
        out.append((f"d{l}b", "c3", ch[l], ch[l]))
    out.append(("head", "c1", ch[0], c_out))
    return out


def init_params(seed=0, c_in=3, c_out=3, base=32, levels=4):
    """He-normal weights, zero biases (a reference initialisation; the CUDA
    network may be given these exact values)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, kind, ci, co in layer_shapes(c_in, c_out, base, levels):
        k = 3 if kind == "c3" else 1
        std = np.sqrt(2.0 / (k * k * ci))
        w = rng.standard_normal((k, k, ci, co) if k == 3 else (ci, co)) * std
        p[name + ".w"] = w
        p[name + ".b"] = np.zeros(co)
    return p


def forward(p, x, levels=4):
    """Returns (prediction, cache for backward)."""
    cache = {}
    skips = []
    h = x
    for l in range(levels):
        if l > 0:
            cache[f"pool{l}_in"] = h
            h = pool2(h)
        for s in "ab":
            name = f"e{l}{s}"
            cache[name + ".x"] = h
            z = conv3x3(h, p[name + ".w"], p[name + ".b"])
            cache[name + ".z"] = z
            h = np.maximum(z, 0.0)
        skips.append(h)
    for l in range(levels - 2, -1, -1):
        u = up2(h)
        h = np.concatenate([u, skips[l]], axis=3)
        cache[f"cat{l}"] = (u.shape[3], skips[l].shape[3])
        for s in "ab":
            name = f"d{l}{s}"
            cache[name + ".x"] = h
            z = conv3x3(h, p[name + ".w"], p[name + ".b"])
            cache[name + ".z"] = z
            h = np.maximum(z, 0.0)
    cache["head.x"] = h
    y = conv1x1(h, p["head.w"], p["head.b"])
    return y, cache


def mse(y, t):
    return float(((y - t) ** 2).mean())


def backward(p, cache, y, t, levels=4):
    """Gradients of mse(y, t) with respect to every parameter."""
    g = {}
    gy = 2.0 * (y - t) / y.size
    gh, g["head.w"], g["head.b"] = conv1x1_backward(cache["head.x"], p["head.w"], gy)
    gskip = [None] * levels
    for l in range(0, levels - 1):
        for s in "ba":
            name = f"d{l}{s}"
            gz = gh * (cache[name + ".z"] > 0)
            gh, g[name + ".w"], g[name + ".b"] = conv3x3_backward(cache[name + ".x"], p[name + ".w"], gz)
        cu, cs = cache[f"cat{l}"]
        gskip[l] = gh[..., cu:]
        gh = up2_backward(gh[..., :cu])
        if l < levels - 2:
            pass
    # gh is now the gradient at the output of the bottom level
    for l in range(levels - 1, -1, -1):
        if l < levels - 1:
            gh = gh + gskip[l]
        for s in "ba":
            name = f"e{l}{s}"
            gz = gh * (cache[name + ".z"] > 0)
            gh, g[name + ".w"], g[name + ".b"] = conv3x3_backward(cache[name + ".x"], p[name + ".w"], gz)
        if l > 0:
            gh = pool2_backward(gh)
    return g


def adam_step(p, g, state, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update in place; state holds 't' and the moment estimates."""
    state["t"] = state.get("t", 0) + 1
    t = state["t"]
    for k in p:
        m = state.setdefault("m." + k, np.zeros_like(p[k]))
        v = state.setdefault("v." + k, np.zeros_like(p[k]))
        m[...] = beta1 * m + (1 - beta1) * g[k]
        v[...] = beta2 * v + (1 - beta2) * g[k] * g[k]
        mh = m / (1 - beta1 ** t)
        vh = v / (1 - beta2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)
    return p
