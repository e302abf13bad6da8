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


def test_bf16_round_is_nearest_even_with_8_significant_bits():
    # exact cases: ties go to the even 7-bit fraction
    cases = {1.0: 1.0, 1.0 + 2**-8: 1.0, 1.0 + 3 * 2**-8: 1.0 + 2**-6, 1.0 + 2**-7: 1.0 + 2**-7,
             -(1.0 + 2**-8 + 2**-12): -(1.0 + 2**-7), 3.0: 3.0, 0.0: 0.0, 2.0**-100: 2.0**-100}
    for x, want in cases.items():
        assert unet.bf16_round(np.array([x]))[0] == want, x
    rng = np.random.default_rng(3)
    a = rng.normal(size=10000) * 10.0 ** rng.uniform(-20, 20, 10000)
    r = unet.bf16_round(a)
    assert np.all(np.abs(r - a) <= 2.0**-8 * np.abs(a))  # half an ulp of an 8-bit significand
    assert np.array_equal(unet.bf16_round(r), r)  # idempotent
    # the rounded values have at most 8 significant bits
    m, _ = np.frexp(r[r != 0])
    assert np.all(m * 2**8 == np.round(m * 2**8))


def test_adam_step_closed_forms():
    # a constant gradient g: the bias-corrected moments are g and g^2 at every step, so
    # each step moves by lr g / (|g| + eps)
    g = np.array([0.3, -2.0, 1e-3, 0.0])
    p = np.array([1.0, 1.0, 1.0, 1.0])
    m = np.zeros(4)
    v = np.zeros(4)
    lr, eps = 1e-2, 1e-8
    for t in range(1, 5):
        p_new, m, v = unet.adam_step(p, g, m, v, t, lr, eps=eps)
        assert np.allclose(p_new - p, -lr * g / (np.abs(g) + eps), rtol=1e-12, atol=1e-15)
        p = p_new
    # first step from zero moments with different b1, b2: the same closed form
    p1, m1, v1 = unet.adam_step(np.zeros(2), np.array([2.0, -0.5]), np.zeros(2), np.zeros(2), 1, 0.1,
                                b1=0.5, b2=0.25)
    assert np.allclose(p1, -0.1 * np.array([2.0, -0.5]) / (np.array([2.0, 0.5]) + 1e-8))
    assert np.allclose(m1, [1.0, -0.25]) and np.allclose(v1, [3.0, 0.1875])
