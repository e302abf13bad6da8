"""Pins for the NumPy U-Net reference (oracle.unet).

The convolution is pinned by a direct six-fold loop written from its definition, the
pooling/upsampling pair by the adjoint identity <P x, y> = <x, P^T y>, and every
parameter gradient of the full network by central finite differences (the backward
pass is hand-written, so a dropped skip, a wrong tap flip or a wrong pooling factor
fails here).
"""

import numpy as np
import pytest

from oracle import unet


def test_conv3d_matches_direct_loop():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(3, 4, 5, 2))
    w = rng.normal(size=(27, 3, 2))
    b = rng.normal(size=3)
    y = unet.conv3d(x, w, b)
    ref = np.zeros((3, 4, 5, 3))
    for z in range(3):
        for yy in range(4):
            for xx in range(5):
                for o in range(3):
                    s = b[o]
                    for t, (dz, dy, dx) in enumerate(unet.TAPS):
                        zz, y2, x2 = z + dz, yy + dy, xx + dx
                        if 0 <= zz < 3 and 0 <= y2 < 4 and 0 <= x2 < 5:
                            s += w[t, o] @ x[zz, y2, x2]
                    ref[z, yy, xx, o] = s
    assert np.allclose(y, ref, atol=1e-12)


def test_pool_upsample_adjoints():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(4, 6, 8, 3))
    yp = rng.normal(size=(2, 3, 4, 3))
    assert np.isclose((unet.pool(x) * yp).sum(), (x * unet.pool_backward(yp)).sum())
    assert np.isclose((unet.upsample(yp) * x).sum(), (yp * unet.upsample_backward(x)).sum())


@pytest.mark.parametrize("name", ["e1a.w", "e2b.w", "e3a.b", "d2a.w", "d1a.w", "out.w", "out.b"])
def test_gradients_match_finite_differences(name):
    rng = np.random.default_rng(2)
    p = unet.init_params(3)
    x = rng.normal(size=(4, 4, 8, 4))
    t = rng.normal(size=(4, 4, 8, 2))
    y, cache = unet.forward(p, x)
    _, dy = unet.relative_loss(y, t)
    g = unet.backward(p, cache, dy)
    flat = p[name].reshape(-1)
    idx = rng.choice(flat.size, min(4, flat.size), replace=False)
    for i in idx:
        old = flat[i]
        h = 1e-6 * max(1.0, abs(old))
        flat[i] = old + h
        lp, _ = unet.relative_loss(unet.forward(p, x)[0], t)
        flat[i] = old - h
        lm, _ = unet.relative_loss(unet.forward(p, x)[0], t)
        flat[i] = old
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[name].reshape(-1)[i]) <= 1e-6 * max(1e-3, abs(fd)), (name, i, fd)
