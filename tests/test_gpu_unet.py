"""The learned preconditioner's network on the GPU against the NumPy reference,
element by element.

The GPU stores activations, weights and back-propagated gradients in bfloat16 and
accumulates in float32.  The reference is run with the same bfloat16 rounding at the
same storage points (oracle.unet.forward / backward with bf16=True, sums in float64),
so the two differ by float32 accumulation order and by the stored values that the two
accumulations round to neighbouring bfloat16 numbers.  Such a flip at the coarse
levels reaches a whole region through the upsampling, so the differences grow with
the volume (measured: relative L2 error of the output 0.04-0.5%, of the parameter
gradients 0.2-0.6% on the volumes below, 2-4% on 16 x 8 x 16 and larger).

Bars, element by element:
* output y_i: 2^-8 S_i with S_i = |b| + sum over taps and input channels of |w| |x| of
  the last convolution at that voxel (measured worst ratio below 0.6);
* weight gradient dW[t, o, i] = sum_v dy_v[o] x_{v+t}[i] and bias gradient: 2^-5 (S_e +
  mean S) with S_e = sum_v |dy_v[o]| |x_{v+t}[i]| (sum_v |dy_v[o]|) taken with the
  gradient before the ReLU mask, so that a voxel whose mask flips is covered (measured
  worst ratio 0.31).
A wrong tap, channel or brick edge in a kernel moves the affected elements by a
sizeable fraction of S, far above these bars; the relative L2 norms are checked too.
The volumes 8 x 12 x 16 and 8 x 8 x 20 make the coarser levels (6 x 4, 3 x 2 in y;
10 and 5 in x) ragged against the convolution's 4 x 4 x 8 bricks.  Adam is checked
against oracle.unet.adam_step fed with the GPU's own gradients, three steps, element
by element.  The reference itself is pinned by finite differences and closed forms in
tests/test_oracle_unet.py.

Both convolution paths are checked: the tcgen05 kernels (MMAs from shared-memory
descriptors, accumulator in tensor memory; used where a lateral plane fits) and the
mma.sync kernels (transec_unet_set_path 1).  Each kernel alone is checked bit for bit
on small-integer data (test_single_convolution_exact), where every sum is exact in
FP32; in the network the two kernels' FP32 sums can differ in their last bits (the
tcgen05 kernel takes wide inputs in channel passes, so its accumulation order differs),
and the bfloat16 values that the two round to different neighbours reach the gradients
through the backward pass (measured relative L2 error of the parameter gradients against the reference up
to 1.6 % on the 8 x 8 x 20 volume with the tcgen05 kernels, 0.6 % with mma.sync), so
the norm bar of the gradients is 2e-2; the element bars are the same for both.
"""

import numpy as np
import pytest

from tests.gpu_util import library, need_gpu
from oracle import unet as ref

pytestmark = pytest.mark.gpu

SHAPES = [(8, 8, 16), (8, 12, 16), (8, 8, 20)]  # nz, ny, nx
PATHS = [0, 1]  # tcgen05 where the plane fits, mma.sync only


def _unflatten(flat):
    p, q = {}, 0
    for name, cin, cout, _ in ref.LAYERS:
        n = 27 * cout * cin
        p[name + ".w"] = flat[q:q + n].reshape(27, cout, cin).astype(np.float64)
        q += n
        p[name + ".b"] = flat[q:q + cout].astype(np.float64)
        q += cout
    return p


def _flatten(g):
    return np.concatenate([np.concatenate([g[n + ".w"].ravel(), g[n + ".b"]]) for n, *_ in ref.LAYERS])


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


def _setup(pkg, shape, seed=5, path=0):
    nz, ny, nx = shape
    u = pkg.binding.transec_unet_create(0, nx, ny, nz, seed)
    pkg.binding.transec_unet_set_path(u, path)
    rng = np.random.default_rng(seed)
    x = rng.normal(size=shape + (4,)).astype(np.float32)
    t = rng.normal(size=shape + (2,)).astype(np.float32)
    # biases are zero at initialisation; give them values so that they are tested too
    flat = pkg.binding.transec_unet_get_params(u)
    params = _unflatten(flat)
    for name, *_ in ref.LAYERS:
        params[name + ".b"] = rng.normal(0, 0.05, params[name + ".b"].shape)
    pkg.binding.transec_unet_set_params(u, _flatten(params).astype(np.float32))
    params = _unflatten(pkg.binding.transec_unet_get_params(u))
    return u, x, t, params


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("shape", SHAPES)
def test_forward_matches_reference_elementwise(shape, path):
    need_gpu()
    pkg = library()
    u, x, t, params = _setup(pkg, shape, path=path)
    try:
        y = np.zeros(shape + (2,), np.float32)
        pkg.binding.transec_unet_forward(u, x, y)
        yr, cache = ref.forward(params, x.astype(np.float64), bf16=True)
        d1 = cache["out"][0]
        bar = 2.0**-8 * ref.conv3d(np.abs(d1), np.abs(ref.bf16_round(params["out.w"])), np.abs(params["out.b"]))
        ratio = np.abs(y - yr) / bar
        assert ratio.max() <= 1.0, (ratio.max(), np.unravel_index(ratio.argmax(), ratio.shape))
        assert _rel(y, yr) <= 5e-3
    finally:
        pkg.binding.transec_unet_destroy(u)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("shape", SHAPES)
def test_gradients_match_reference_elementwise(shape, path):
    need_gpu()
    pkg = library()
    u, x, t, params = _setup(pkg, shape, seed=6, path=path)
    try:
        # the backward starts from the loss gradient of the GPU's own output, so that the
        # comparison covers the backward pass alone (the forward is checked above)
        y = np.zeros(shape + (2,), np.float32)
        pkg.binding.transec_unet_forward(u, x, y)
        loss, g = pkg.binding.transec_unet_train_step(u, x, t, 0.0, want_grads=True)
        _, cache = ref.forward(params, x.astype(np.float64), bf16=True)
        lr, dy = ref.relative_loss(y.astype(np.float64), t.astype(np.float64))
        douts = {}
        gr = ref.backward(params, cache, dy, bf16=True, record=douts)
        assert abs(loss - lr) <= 1e-5 * lr
        gg = _unflatten(g)
        worst, rel = {}, {}
        for name, *_ in ref.LAYERS:
            inp = cache[name][0]
            _, sw, sb = ref.conv3d_backward(np.abs(inp), np.zeros_like(params[name + ".w"]),
                                            np.abs(douts[name + ".in"]))
            for suffix, s in ((".w", sw), (".b", sb)):
                err = np.abs(gg[name + suffix] - gr[name + suffix])
                worst[name + suffix] = float((err / (2.0**-5 * (s + s.mean()))).max())
                rel[name + suffix] = float(_rel(gg[name + suffix], gr[name + suffix]))
        print("max error / element bar:", worst)
        print("relative L2 error:", rel)
        assert max(worst.values()) <= 1.0, worst
        assert max(rel.values()) <= 2e-2, rel
    finally:
        pkg.binding.transec_unet_destroy(u)


def test_adam_steps_match_reference():
    """Three Adam steps on the FP32 master parameters: each step's update from the GPU's
    gradient of that step (returned before the update) against oracle.unet.adam_step in
    float64; FP32 arithmetic bounds the difference by a few ulps of the parameter plus a
    relative 1e-5 of the step."""
    need_gpu()
    pkg = library()
    shape = SHAPES[0]
    u, x, t, params = _setup(pkg, shape, seed=8)
    try:
        p = pkg.binding.transec_unet_get_params(u).astype(np.float64)
        m = np.zeros_like(p)
        v = np.zeros_like(p)
        lr = 1e-3
        for step in range(1, 4):
            _, g = pkg.binding.transec_unet_train_step(u, x, t, lr, want_grads=True)
            p_ref, m, v = ref.adam_step(p, g.astype(np.float64), m, v, step, lr)
            got = pkg.binding.transec_unet_get_params(u).astype(np.float64)
            err = np.abs(got - p_ref)
            bar = 4 * np.spacing(np.abs(p_ref).astype(np.float32)).astype(np.float64) + 1e-5 * lr
            assert np.all(err <= bar), (step, float((err / bar).max()))
            assert np.abs(got - p).max() > 0.5 * lr  # the step moved the parameters
            p = got
    finally:
        pkg.binding.transec_unet_destroy(u)


CONV_CASES = [((8, 8, 16), 16, 16), ((8, 8, 20), 48, 16), ((4, 4, 10), 96, 32), ((4, 4, 10), 32, 96),
              ((2, 2, 5), 64, 64), ((2, 3, 7), 16, 48), ((6, 20, 20), 64, 32)]  # (nz, ny, nx), cin, cout


def _bf16_bits(a):
    """bfloat16 bit patterns of float32 values that bfloat16 holds exactly."""
    u = np.ascontiguousarray(a, np.float32).view(np.uint32)
    assert np.all(u & 0xFFFF == 0)
    return (u >> 16).astype(np.uint16)


@pytest.mark.parametrize("path", PATHS)
@pytest.mark.parametrize("case", CONV_CASES)
def test_single_convolution_exact(case, path):
    """One convolution through each kernel with small-integer inputs and weights: every
    product and partial sum is an integer below 2^24, exact in FP32 in any order, so the
    output must equal the oracle's float64 convolution bit for bit.  A wrong tap,
    channel, channel pass, halo cell or tile row shows as a mismatch.  The cases cover
    one and several channel passes, N = 16 to 96, ragged and odd lateral sizes and a
    20 x 20 plane."""
    need_gpu()
    pkg = library()
    shape, cin, cout = case
    rng = np.random.default_rng(cin * 131 + cout)
    x = rng.integers(-2, 3, shape + (cin,)).astype(np.float32)
    w = rng.integers(-2, 3, (27, cout, cin)).astype(np.float32)
    b = rng.integers(-3, 4, cout).astype(np.float32)
    y = pkg.binding.transec_unet_conv3d(_bf16_bits(x), _bf16_bits(w), b, path=path)
    want = ref.conv3d(x.astype(np.float64), w.astype(np.float64), b.astype(np.float64))
    assert np.array_equal(y, want.astype(np.float32)), float(np.abs(y - want).max())


def test_training_reduces_loss():
    need_gpu()
    pkg = library()
    u, x, t, _ = _setup(pkg, SHAPES[0], seed=7)
    try:
        losses = [pkg.binding.transec_unet_train_step(u, x, t, 1e-3)[0] for _ in range(60)]
        assert losses[-1] < 0.5 * losses[0], losses[::10]
    finally:
        pkg.binding.transec_unet_destroy(u)


def test_zero_output_layer():
    """transec_unet_zero_output zeroes the output layer's weights (the learned
    preconditioner's start) and leaves every other parameter as it was."""
    need_gpu()
    pkg = library()
    u, x, t, params = _setup(pkg, SHAPES[0], seed=9)
    try:
        pkg.binding.transec_unet_zero_output(u)
        after = _unflatten(pkg.binding.transec_unet_get_params(u))
        for name, *_ in ref.LAYERS:
            if name == "out":
                assert np.all(after["out.w"] == 0) and np.array_equal(after["out.b"], params["out.b"])
            else:
                assert np.array_equal(after[name + ".w"], params[name + ".w"])
                assert np.array_equal(after[name + ".b"], params[name + ".b"])
    finally:
        pkg.binding.transec_unet_destroy(u)
