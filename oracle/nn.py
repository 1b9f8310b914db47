"""FP64 reference of the warm-start network's layers (the learned part of the
workloads; the paper itself has no network).

Layouts: activations [C][D][H][W] (channel-planar, D = z, H = y, W = x) of one
sample; 3 x 3 x 3 convolution weights [C_out][C_in][27] with tap index
t = (dz + 1) * 9 + (dy + 1) * 3 + (dx + 1), zero padding 1, stride 1, plus a
bias [C_out].  Pooling: 2 x 2 x 2 average; upsampling: nearest, factor 2.

Every function is a direct restatement of the operation's definition
(explicit shifted sums), written for small tensors; gradients are the
corresponding adjoints.  Pinned by finite differences and brute-force loops in
tests/test_oracle_nn.py.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def _shift(x, dz, dy, dx):
    """y[..., z, y, x] = x[..., z + dz, y + dy, x + dx] with zero outside."""
    out = np.zeros_like(x)
    D, H, W = x.shape[-3:]
    zs, ze = max(0, -dz), min(D, D - dz)
    ys, ye = max(0, -dy), min(H, H - dy)
    xs, xe = max(0, -dx), min(W, W - dx)
    out[..., zs:ze, ys:ye, xs:xe] = x[..., zs + dz:ze + dz, ys + dy:ye + dy, xs + dx:xe + dx]
    return out


def conv3d(x, w, b):
    """y[o] = b[o] + sum_{i,t} w[o, i, t] x[i] shifted by tap t."""
    co = w.shape[0]
    y = np.zeros((co,) + x.shape[1:])
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        y += np.einsum("oi,i...->o...", w[:, :, t], xs)
    return y + b[:, None, None, None]


def conv3d_backward(x, w, gy):
    """Gradients (gx, gw, gb) of sum(gy * conv3d(x, w, b))."""
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for t, (dz, dy, dx) in enumerate(TAPS):
        xs = _shift(x, dz, dy, dx)
        gw[:, :, t] = np.tensordot(gy, xs, axes=([1, 2, 3], [1, 2, 3]))
        gx += _shift(np.einsum("oi,o...->i...", w[:, :, t], gy), -dz, -dy, -dx)
    gb = gy.sum(axis=(1, 2, 3))
    return gx, gw, gb


def relu(x):
    return np.maximum(x, 0.0)


def relu_backward(y, gy):
    """y = relu(x) (post-activation); gradient passes where y > 0."""
    return np.where(y > 0.0, gy, 0.0)


def pool2(x):
    C, D, H, W = x.shape
    return x.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).mean(axis=(2, 4, 6))


def pool2_backward(gy):
    return np.repeat(np.repeat(np.repeat(gy, 2, axis=1), 2, axis=2), 2, axis=3) / 8.0


def up2(x):
    return np.repeat(np.repeat(np.repeat(x, 2, axis=1), 2, axis=2), 2, axis=3)


def up2_backward(gy):
    C, D, H, W = gy.shape
    return gy.reshape(C, D // 2, 2, H // 2, 2, W // 2, 2).sum(axis=(2, 4, 6))


# ---------------------------------------------------------------------------
# The network: a 4-level U-Net with additive skips.
# enc0: conv(in,16) relu, conv(16,16) relu -> s0; pool
# enc1: conv(16,32) relu, conv(32,32) relu -> s1; pool
# enc2: conv(32,64) relu, conv(64,64) relu -> s2; pool
# mid : conv(64,64) relu; up; + s2
# dec2: conv(64,32) relu; up; + s1
# dec1: conv(32,16) relu; up; + s0
# dec0: conv(16,16) relu
# head: conv(16,out)

def layer_shapes(c_in=5, c_out=3, widths=(16, 32, 64, 64)):
    c0, c1, c2, c3 = widths
    return [(c0, c_in), (c0, c0), (c1, c0), (c1, c1), (c2, c1), (c2, c2), (c3, c2),
            (c1, c3), (c0, c1), (c0, c0), (c_out, c0)]


def init_params(seed=0, c_in=5, c_out=3, widths=(16, 32, 64, 64)):
    """He-normal weights (seeded), zero biases; list of (w, b)."""
    rng = np.random.default_rng(seed)
    params = []
    for co, ci in layer_shapes(c_in, c_out, widths):
        std = np.sqrt(2.0 / (27 * ci))
        params.append((rng.normal(0.0, std, size=(co, ci, 27)), np.zeros(co)))
    return params


def forward(params, x, keep=False, quant=None):
    """x: [C_in][D][H][W] with D, H, W divisible by 8.  Returns y (and the cache).

    `quant` (optional) is applied to every stored activation -- each ReLU
    output, pooling output and upsample-plus-skip sum, not the head's output --
    to model a network that stores its activations at reduced precision
    (e.g. quant=to_bf16)."""
    cache = []
    q = (lambda a: a) if quant is None else quant

    def conv(i, a, act=True):
        w, b = params[i]
        z = conv3d(a, w, b)
        y = q(relu(z)) if act else z
        cache.append(("conv", i, a, y, act))
        return y

    a = conv(0, x)
    s0 = conv(1, a)
    a = q(pool2(s0))
    a = conv(2, a)
    s1 = conv(3, a)
    a = q(pool2(s1))
    a = conv(4, a)
    s2 = conv(5, a)
    a = q(pool2(s2))
    a = conv(6, a)
    a = q(up2(a) + s2)
    a = conv(7, a)
    a = q(up2(a) + s1)
    a = conv(8, a)
    a = q(up2(a) + s0)
    a = conv(9, a)
    y = conv(10, a, act=False)
    return (y, cache) if keep else y


def backward(params, cache, gy):
    """Gradients [(gw, gb)] of sum(gy * forward(x)) from the forward cache."""
    grads = [None] * len(params)
    conv_in = {i: (a, y, act) for (_, i, a, y, act) in cache}

    def bconv(i, g):
        a, y, act = conv_in[i]
        if act:
            g = relu_backward(y, g)
        gx, gw, gb = conv3d_backward(a, params[i][0], g)
        grads[i] = (gw, gb)
        return gx

    g = bconv(10, gy)
    g = bconv(9, g)
    gs0 = g.copy()
    g = up2_backward(g)
    g = bconv(8, g)
    gs1 = g.copy()
    g = up2_backward(g)
    g = bconv(7, g)
    gs2 = g.copy()
    g = up2_backward(g)
    g = bconv(6, g)
    g = pool2_backward(g) + gs2
    g = bconv(5, g)
    g = bconv(4, g)
    g = pool2_backward(g) + gs1
    g = bconv(3, g)
    g = bconv(2, g)
    g = pool2_backward(g) + gs0
    g = bconv(1, g)
    bconv(0, g)
    return grads


def to_bf16(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64."""
    f = np.asarray(a, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
