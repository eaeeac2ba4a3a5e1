"""Pins of the denoiser oracle (oracle/denoise.py) against library routines,
impulse responses and networks whose output is known in closed form."""
import numpy as np
import pytest
import torch
from scipy import ndimage

from oracle import denoise as DN


def test_bf16_round_matches_torch():
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.standard_normal(20000) * 10.0 ** rng.integers(-6, 6, 20000),
                        # exact ties between two bfloat16 values, both parities
                        (np.arange(1, 200, dtype=np.float32) * 2.0 ** -7 + 2.0 ** -9).astype(np.float64),
                        [0.0, -0.0, 1.0, -3.5]])
    ref = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    assert np.array_equal(DN.bf16_round(x), ref)


def test_conv3_single_channel_is_scipy_correlate():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((5, 6, 7))
    w = rng.standard_normal((3, 3, 3))
    got = DN.conv3(x[..., None], w[None, ..., None], np.zeros(1), relu=False)[..., 0]
    ref = ndimage.correlate(x, w, mode="constant", cval=0.0)
    np.testing.assert_allclose(got, ref, rtol=1e-12, atol=1e-12)


def test_conv3_impulse_response_fixes_taps_and_channels():
    rng = np.random.default_rng(2)
    w = rng.standard_normal((4, 3, 3, 3, 3))
    x = np.zeros((5, 5, 5, 3))
    x[2, 2, 2, 1] = 1.0
    out = DN.conv3(x, w, np.zeros(4), relu=False)
    # out[z, y, x, o] = w[o, 2 - z + 1, ...] around the impulse: the kernel appears flipped
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                np.testing.assert_array_equal(out[3 - dz, 3 - dy, 3 - dx], w[:, dz, dy, dx, 1])
    mask = np.ones(out.shape[:3], bool)
    mask[1:4, 1:4, 1:4] = False
    assert not out[mask].any()


def test_conv3_bias_relu_and_boundary():
    w = np.zeros((2, 3, 3, 3, 1))
    w[:, 1, 1, 1, 0] = 1.0
    w[:, 0, 1, 1, 0] = 1.0                   # the voxel below in z
    b = np.array([0.5, -10.0])
    x = np.ones((3, 3, 3, 1))
    out = DN.conv3(x, w, b)
    assert np.all(out[0, ..., 0] == 1.5)     # z = 0 sees the zero padding below
    assert np.all(out[1:, ..., 0] == 2.5)
    assert not out[..., 1].any()             # ReLU


def test_pool2_is_strided_maximum_filter():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((6, 4, 8, 2))
    ref = np.stack([ndimage.maximum_filter(x[..., c], size=2, origin=-1, mode="nearest")[::2, ::2, ::2]
                    for c in range(2)], axis=-1)
    np.testing.assert_array_equal(DN.pool2(x), ref)


def test_up2_is_kronecker_with_ones():
    rng = np.random.default_rng(4)
    x = rng.standard_normal((2, 3, 4, 2))
    ref = np.stack([np.kron(x[..., c], np.ones((2, 2, 2))) for c in range(2)], axis=-1)
    np.testing.assert_array_equal(DN.up2(x), ref)


def test_param_layout_and_count():
    p = DN.init_params(0)
    assert p.size == DN.n_params()
    layers, (hw, hb) = DN.unpack_params(p)
    assert len(layers) == 14 and hw.shape == (16,)
    assert layers[0][0].shape == (16, 3, 3, 3, 16) and not layers[0][0][..., 2:].any()
    assert 0.9e6 < p.size < 1.1e6


def _identity_net(pick_up: bool):
    """Weights that copy channels through every conv3 (center tap = identity on
    the first min(cin, cout) channels, or, in the decoders' first conv, on the
    upsampled half when pick_up) and a head that reads channel 0."""
    convs, (hc, _) = DN.layer_shapes()
    parts = []
    for i, (ci, co) in enumerate(convs):
        w = np.zeros((co, 3, 3, 3, ci))
        off = ci // 2 if (pick_up and i in (8, 10, 12)) else 0
        for o in range(min(co, ci - off)):
            w[o, 1, 1, 1, off + o] = 1.0
        parts += [w.ravel(), np.zeros(co)]
    hw = np.zeros(hc)
    hw[0] = 1.0
    return np.concatenate(parts + [hw, np.zeros(1)])


@pytest.mark.parametrize("pick_up", [False, True])
def test_unet_identity_paths(pick_up):
    rng = np.random.default_rng(5)
    dose = rng.random((16, 16, 8))
    rho = np.ones_like(dose)
    out = DN.unet_forward(dose, rho, _identity_net(pick_up))
    x0 = DN.bf16_round(dose / dose.max())
    if not pick_up:
        ref = dose + dose.max() * x0                       # skip path: the input itself
    else:
        # through the bottleneck: three max-poolings then three nearest upsamplings
        pooled = ndimage.maximum_filter(x0, size=8, origin=(-4, -4, -4), mode="nearest")[::8, ::8, ::8]
        ref = dose + dose.max() * np.kron(pooled, np.ones((8, 8, 8)))
    np.testing.assert_allclose(out, ref, rtol=1e-12, atol=1e-12)


def test_untrained_head_returns_input_dose():
    rng = np.random.default_rng(6)
    dose = rng.random((8, 8, 8))
    out = DN.unet_forward(dose, np.ones_like(dose), DN.init_params(1, head_scale=0.0))
    np.testing.assert_array_equal(out, dose)


def test_gradient_matches_finite_differences():
    """The oracle's backward pass against central differences of its own FP64
    loss, on a small network (widths 8) and volume, at random coordinates of
    every layer and the head."""
    rng = np.random.default_rng(7)
    widths = (8, 8, 8, 8)
    dose = rng.random((8, 8, 16)) + 0.2
    rho = rng.random((8, 8, 16)) + 0.5
    target = dose * (1.0 + 0.1 * rng.standard_normal(dose.shape))
    p = DN.init_params(5, widths, head_scale=0.3)
    p[:-1] += 0.01 * rng.standard_normal(p.size - 1)          # non-zero biases
    loss, g = DN.unet_loss_and_grad(dose, rho, target, p, widths, rounding=False)
    convs, _ = DN.layer_shapes(widths)
    picks, k = [], 0
    for ci, co in convs:
        n = 27 * ci * co
        lo = k if ci != DN.IN_CHANNELS else k           # first layer: only real input channels matter
        picks += list(rng.integers(lo, k + n, 3)) + [k + n + int(rng.integers(0, co))]
        k += n + co
    picks += [k, k + 3, k + 8]
    h = 1e-6
    for j in picks:
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        lp = DN.unet_loss_and_grad(dose, rho, target, pp, widths, rounding=False)[0]
        lm = DN.unet_loss_and_grad(dose, rho, target, pm, widths, rounding=False)[0]
        fd = (lp - lm) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * max(1.0, abs(fd)) + 1e-7, (j, fd, g[j])


def test_wgrad_and_dgrad_are_adjoint_of_conv():
    """<conv3(x, w), gz> = <w, wgrad(x, gz)> = <x, dgrad(gz, w)>."""
    rng = np.random.default_rng(8)
    x = rng.standard_normal((4, 5, 6, 3))
    w = rng.standard_normal((2, 3, 3, 3, 3))
    gz = rng.standard_normal((4, 5, 6, 2))
    y = DN.conv3(x, w, np.zeros(2), relu=False)
    a = np.sum(y * gz)
    np.testing.assert_allclose(np.sum(w * DN.conv3_wgrad(x, gz)), a, rtol=1e-12)
    np.testing.assert_allclose(np.sum(x * DN.conv3_dgrad(gz, w)), a, rtol=1e-12)
