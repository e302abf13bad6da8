"""NumPy reference of the learned preconditioner's 3D U-Net, forward and backward.

Test infrastructure only (see the package docstring).  The paper has no learned
component; this network is the one the library trains and applies on the GPU
(3 levels of 16/32/64 channels, 3x3x3 convolutions with zero padding, ReLU, 2x2x2
average pooling, nearest 2x upsampling, skip connections by channel concatenation).
It is written out plainly in float64 so that the GPU kernels' values and gradients can
be checked against it; its own gradients are pinned by finite differences in
tests/test_oracle_unet.py.

Tensor layout: activations are (nz, ny, nx, C) arrays (channels last, x fastest among
the spatial axes), weights of a 3x3x3 convolution are (27, Cout, Cin) with tap
t = (dz+1)*9 + (dy+1)*3 + (dx+1), so that

    y[z, y, x, o] = b[o] + sum_t sum_i w[t, o, i] * x[z+dz, y+dy, x+dx, i]

with zero outside the volume.
"""

from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]

# (name, cin, cout, relu) in execution order; "cat1"/"cat2" mark the skip inputs
LAYERS = [
    ("e1a", 4, 16, True), ("e1b", 16, 16, True),
    ("e2a", 16, 32, True), ("e2b", 32, 32, True),
    ("e3a", 32, 64, True), ("e3b", 64, 64, True),
    ("d2a", 64 + 32, 32, True), ("d2b", 32, 32, True),
    ("d1a", 32 + 16, 16, True), ("d1b", 16, 16, True),
    ("out", 16, 2, False),
]


def shift(x, dz, dy, dx):
    """x[z+dz, y+dy, x+dx] with zero outside."""
    out = np.zeros_like(x)
    nz, ny, nx = x.shape[:3]
    sz = slice(max(0, -dz), min(nz, nz - dz))
    sy = slice(max(0, -dy), min(ny, ny - dy))
    sx = slice(max(0, -dx), min(nx, nx - dx))
    tz = slice(max(0, dz), min(nz, nz + dz))
    ty = slice(max(0, dy), min(ny, ny + dy))
    tx = slice(max(0, dx), min(nx, nx + dx))
    out[sz, sy, sx] = x[tz, ty, tx]
    return out


def conv3d(x, w, b):
    y = np.zeros(x.shape[:3] + (w.shape[1],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shift(x, dz, dy, dx) @ w[t].T
    return y + b


def conv3d_backward(x, w, dy):
    """(dx, dw, db) of conv3d for the upstream gradient dy."""
    dx = np.zeros_like(x)
    dw = np.zeros_like(w)
    for t, (oz, oy, ox) in enumerate(TAPS):
        xs = shift(x, oz, oy, ox)
        dw[t] = np.einsum("zyxo,zyxi->oi", dy, xs)
        dx += shift(dy @ w[t], -oz, -oy, -ox)
    return dx, dw, dy.sum(axis=(0, 1, 2))


def pool(x):
    nz, ny, nx, c = x.shape
    return x.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).mean(axis=(1, 3, 5))


def pool_backward(dy):
    return np.repeat(np.repeat(np.repeat(dy, 2, 0), 2, 1), 2, 2) / 8.0


def upsample(x):
    return np.repeat(np.repeat(np.repeat(x, 2, 0), 2, 1), 2, 2)


def upsample_backward(dy):
    nz, ny, nx, c = dy.shape
    return dy.reshape(nz // 2, 2, ny // 2, 2, nx // 2, 2, c).sum(axis=(1, 3, 5))


def bf16_round(a):
    """Round to the nearest bfloat16 (8 significant bits, ties to even), returned as
    float64: the storage format of the GPU network's activations, weights and
    back-propagated gradients.  The value is first rounded to float32 (the GPU's
    accumulators are float32), then its low 16 bits are rounded off."""
    a32 = np.ascontiguousarray(a, dtype=np.float32)
    u = a32.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)


def init_params(seed: int):
    """He-style initialisation: w ~ N(0, 2 / (27 cin)), b = 0."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, cin, cout, _ in LAYERS:
        p[name + ".w"] = rng.normal(0.0, np.sqrt(2.0 / (27 * cin)), (27, cout, cin))
        p[name + ".b"] = np.zeros(cout)
    return p


def forward(p, x, bf16=False):
    """Network output (nz, ny, nx, 2) and the cache for backward.

    bf16=True rounds, with ``bf16_round``, exactly the tensors the GPU network stores
    in bfloat16: the input, the weights, every convolution's output after bias and
    ReLU (not the final layer's, which is float32) and every pooled tensor; all sums
    stay float64.  Upsampling and concatenation only copy."""
    cache = {}
    rnd = bf16_round if bf16 else (lambda a: a)

    def layer(name, inp, relu, store=True):
        pre = conv3d(inp, rnd(p[name + ".w"]), p[name + ".b"])
        out = np.maximum(pre, 0.0) if relu else pre
        out = rnd(out) if store else out
        cache[name] = (inp, out, relu)
        cache[name + ".pre"] = pre
        return out

    x = rnd(x)
    a1 = layer("e1b", layer("e1a", x, True), True)
    a2 = layer("e2b", layer("e2a", rnd(pool(a1)), True), True)
    a3 = layer("e3b", layer("e3a", rnd(pool(a2)), True), True)
    d2 = layer("d2b", layer("d2a", np.concatenate([upsample(a3), a2], axis=3), True), True)
    d1 = layer("d1b", layer("d1a", np.concatenate([upsample(d2), a1], axis=3), True), True)
    y = layer("out", d1, False, store=False)
    return y, cache


def backward(p, cache, dy, bf16=False, record=None):
    """Gradients of every parameter for the upstream gradient dy of the output.

    bf16=True rounds what the GPU stores in bfloat16 on the way back: the output
    gradient, every layer's data gradient, the upsampling gradient (sum of the 8 fine
    children) and the pooling gradient plus its skip gradient; the weights are the
    rounded ones of the forward pass; parameter gradients are float64 sums.  A dict
    passed as ``record`` receives each layer's output gradient before and after the
    ReLU mask (keys name + ".in" and name)."""
    g = {}
    rnd = bf16_round if bf16 else (lambda a: a)

    def back(name, dout):
        inp, out, relu = cache[name]
        if record is not None:
            record[name + ".in"] = dout
        if relu:
            dout = dout * (out > 0)
        if record is not None:
            record[name] = dout
        dx, dw, db = conv3d_backward(inp, rnd(p[name + ".w"]), dout)
        g[name + ".w"], g[name + ".b"] = dw, db
        return rnd(dx)

    dy = rnd(dy)
    dd1 = back("d1a", back("d1b", back("out", dy)))
    c1 = cache["e1b"][1].shape[3]
    d_up2, d_a1_skip = dd1[..., :-c1], dd1[..., -c1:]
    dd2 = back("d2a", back("d2b", rnd(upsample_backward(d_up2))))
    c2 = cache["e2b"][1].shape[3]
    d_up3, d_a2_skip = dd2[..., :-c2], dd2[..., -c2:]
    da3 = back("e3a", back("e3b", rnd(upsample_backward(d_up3))))
    da2 = back("e2a", back("e2b", rnd(pool_backward(da3) + d_a2_skip)))
    back("e1a", back("e1b", rnd(pool_backward(da2) + d_a1_skip)))
    return g


def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba, ICLR 2015, Algorithm 1) of the arrays p with
    gradients g and moments m, v at step t >= 1; returns (p, m, v).  The moments are
    exponential averages of g and g^2, divided by 1 - b^t to remove their bias, and the
    step is lr * m_hat / (sqrt(v_hat) + eps)."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    m_hat = m / (1.0 - b1**t)
    v_hat = v / (1.0 - b2**t)
    return p - lr * m_hat / (np.sqrt(v_hat) + eps), m, v


def relative_loss(y, t):
    """L = sum |y - t|^2 / sum |t|^2 and dL/dy."""
    den = float((t * t).sum())
    d = y - t
    return float((d * d).sum()) / den, 2.0 * d / den
