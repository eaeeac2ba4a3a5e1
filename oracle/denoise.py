"""Plain FP64 reference of the dose denoiser (test infrastructure).

Only tests/, the smoke check and the benchmark's CPU legs import this module;
the product path never does.

The paper ends at Monte Carlo dose (Sec. 2.3) and reports uncertainty-limited
run times (Sec. 3); the denoiser is the extension that maps a low-history dose
and the phantom density to an estimate of the high-history dose, so that fewer
histories reach a target error. Its network is a 3D U-Net:

- conv3: 3x3x3 cross-correlation with zero padding ("same" size), bias, ReLU;
- pool2: 2x2x2 max pooling, stride 2;
- up2: nearest-neighbour 2x upsampling;
- channel concatenation of the skip tensor (first) and the upsampled tensor;
- head: 1x1x1 convolution to one channel, scaled by the input's maximum dose
  and added to the input dose (residual connection).

Arithmetic is FP64. Activations are rounded to bfloat16 (round to nearest
even) at the points where the GPU path stores them, so that both sides see the
same stored values; the rounding function is pinned against PyTorch's
bfloat16 conversion in the tests.

Architecture (widths C = (16, 32, 64, 128), four levels):
  x0 = [dose / Dmax, rho, 0 x 14] (16 channels)
  e0 = conv3(conv3(x0, 16->16), 16->16)                       level 0
  e1 = conv3(conv3(pool2(e0), 16->32), 32->32)                level 1
  e2 = conv3(conv3(pool2(e1), 32->64), 64->64)                level 2
  b  = conv3(conv3(pool2(e2), 64->128), 128->64)              level 3
  d2 = conv3(conv3(cat(e2, up2(b)), 128->64), 64->32)
  d1 = conv3(conv3(cat(e1, up2(d2)), 64->32), 32->16)
  d0 = conv3(conv3(cat(e0, up2(d1)), 32->16), 16->16)
  out = dose + Dmax * head(d0)
"""
from __future__ import annotations

import numpy as np

WIDTHS = (16, 32, 64, 128)
IN_CHANNELS = 16          # dose, density and zero channels up to the MMA K step


def bf16_round(x) -> np.ndarray:
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    The value is first taken to float32 and then its low 16 bits are rounded
    off with the round-half-to-even rule on the kept bits."""
    f = np.asarray(x, dtype=np.float32)
    u = f.view(np.uint32).astype(np.uint64)
    keep_lsb = (u >> np.uint64(16)) & np.uint64(1)
    u = (u + np.uint64(0x7FFF) + keep_lsb) & np.uint64(0xFFFF0000)
    return u.astype(np.uint32).view(np.float32).astype(np.float64)


def conv3(x: np.ndarray, w: np.ndarray, b: np.ndarray, relu: bool = True) -> np.ndarray:
    """3x3x3 zero-padded cross-correlation.

    x: [D, H, W, Cin]; w: [Cout, 3, 3, 3, Cin] indexed (dz, dy, dx);
    b: [Cout]. out[z, y, x, o] = b[o] + sum over taps and input channels of
    w[o, dz, dy, dx, c] * x[z + dz - 1, y + dy - 1, x + dx - 1, c], with x = 0
    outside the volume; then max(., 0) when relu."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    D, H, W, _ = x.shape
    xp = np.pad(x, ((1, 1), (1, 1), (1, 1), (0, 0)))
    out = np.broadcast_to(np.asarray(b, dtype=np.float64), (D, H, W, w.shape[0])).copy()
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                out += np.tensordot(xp[dz:dz + D, dy:dy + H, dx:dx + W], w[:, dz, dy, dx, :], axes=([3], [1]))
    return np.maximum(out, 0.0) if relu else out


def conv3_abs(x: np.ndarray, w: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Sum of the magnitudes of every term of conv3 (bias included): the scale
    of the accumulation error of a finite-precision evaluation."""
    return conv3(np.abs(x), np.abs(w), np.abs(b), relu=False)


def pool2(x: np.ndarray) -> np.ndarray:
    """2x2x2 max pooling with stride 2 (even sizes)."""
    D, H, W, C = x.shape
    return x.reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).max(axis=(1, 3, 5))


def up2(x: np.ndarray) -> np.ndarray:
    """Nearest-neighbour 2x upsampling: out[z, y, x] = in[z // 2, y // 2, x // 2]."""
    return x.repeat(2, axis=0).repeat(2, axis=1).repeat(2, axis=2)


def layer_shapes(widths=WIDTHS):
    """(c_in, c_out) of the 14 conv3 layers in network order, then the head."""
    c0, c1, c2, c3 = widths
    convs = [(IN_CHANNELS, c0), (c0, c0), (c0, c1), (c1, c1), (c1, c2), (c2, c2), (c2, c3), (c3, c2),
             (2 * c2, c2), (c2, c1), (2 * c1, c1), (c1, c0), (2 * c0, c0), (c0, c0)]
    return convs, (c0, 1)


def n_params(widths=WIDTHS) -> int:
    convs, (hc, _) = layer_shapes(widths)
    return sum(27 * ci * co + co for ci, co in convs) + hc + 1


def unpack_params(flat: np.ndarray, widths=WIDTHS):
    """Flat parameter vector -> [(w [Cout,3,3,3,Cin], b [Cout]) x 14], (head w [C0], head b).
    Order: per conv layer its weights (C order) then its bias; then the head."""
    flat = np.asarray(flat, dtype=np.float64)
    convs, (hc, _) = layer_shapes(widths)
    out, k = [], 0
    for ci, co in convs:
        n = 27 * ci * co
        out.append((flat[k:k + n].reshape(co, 3, 3, 3, ci), flat[k + n:k + n + co]))
        k += n + co
    hw = flat[k:k + hc]
    hb = flat[k + hc]
    assert k + hc + 1 == flat.size
    return out, (hw, hb)


def init_params(seed: int, widths=WIDTHS, head_scale: float = 0.0) -> np.ndarray:
    """He-normal conv weights, zero biases, head weights scaled by head_scale
    (0: the untrained network returns its input dose)."""
    rng = np.random.default_rng(seed)
    convs, (hc, _) = layer_shapes(widths)
    parts = []
    for i, (ci, co) in enumerate(convs):
        fan_in = 27 * (2 if i == 0 else ci)
        w = rng.standard_normal((co, 3, 3, 3, ci)) * np.sqrt(2.0 / fan_in)
        if i == 0:
            w[..., 2:] = 0.0                 # padding channels carry nothing
        parts += [w.ravel(), np.zeros(co)]
    parts += [rng.standard_normal(hc) * head_scale, np.zeros(1)]
    return np.concatenate(parts)


def pack_input(dose: np.ndarray, rho: np.ndarray):
    """[D, H, W] dose and density -> [D, H, W, 16] stored input and Dmax."""
    dmax = float(np.max(dose))
    scale = 1.0 / dmax if dmax > 0 else 0.0
    x = np.zeros(dose.shape + (IN_CHANNELS,))
    x[..., 0] = bf16_round(np.asarray(dose, dtype=np.float64) * scale)
    x[..., 1] = bf16_round(rho)
    return x, dmax


def unet_forward(dose: np.ndarray, rho: np.ndarray, flat_params: np.ndarray, widths=WIDTHS,
                 return_layers: bool = False, rounding: bool = True):
    """Denoised dose [D, H, W] (D, H, W divisible by 8). Every conv3 output is
    rounded to bfloat16 before use, as stored by the GPU path (rounding=False:
    plain FP64 throughout, for derivative checks); the head is evaluated
    without rounding."""
    layers, (hw, hb) = unpack_params(flat_params, widths)
    x, dmax = pack_input(dose, rho)
    if not rounding:
        x[..., 0] = np.asarray(dose, dtype=np.float64) / dmax
        x[..., 1] = rho
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    acts = []

    def c(i, t):
        w, b = layers[i]
        y = rnd(conv3(t, rnd(w), rnd(b), relu=True))
        acts.append(y)
        return y

    e0 = c(1, c(0, x))
    e1 = c(3, c(2, pool2(e0)))
    e2 = c(5, c(4, pool2(e1)))
    bt = c(7, c(6, pool2(e2)))
    d2 = c(9, c(8, np.concatenate([e2, up2(bt)], axis=3)))
    d1 = c(11, c(10, np.concatenate([e1, up2(d2)], axis=3)))
    d0 = c(13, c(12, np.concatenate([e0, up2(d1)], axis=3)))
    r = d0 @ np.asarray(hw, dtype=np.float64) + float(hb)
    out = np.asarray(dose, dtype=np.float64) + dmax * r
    return (out, acts) if return_layers else out


# ------------------------------------------------------------- gradients ---
# Training minimises the mean squared error between the denoised dose and a
# high-history dose, both divided by the input's maximum dose:
#   loss = mean_v (dose_v / Dmax + head(d0)_v - target_v / Dmax)^2.
# The derivatives below are those of the FP64 network evaluated at the
# activations passed in (the rounding of stored activations is not
# differentiated: it is a storage step, not part of the model).

def conv3_wgrad(x: np.ndarray, gz: np.ndarray) -> np.ndarray:
    """dloss/dw for out = conv3(x, w): dw[o, dz, dy, dx, c] = sum over voxels
    of gz[z, y, x, o] * x[z + dz - 1, y + dy - 1, x + dx - 1, c] (zero padding)."""
    D, H, W, C = x.shape
    xp = np.pad(np.asarray(x, dtype=np.float64), ((1, 1), (1, 1), (1, 1), (0, 0)))
    g = np.asarray(gz, dtype=np.float64)
    dw = np.zeros((g.shape[-1], 3, 3, 3, C))
    for dz in range(3):
        for dy in range(3):
            for dx in range(3):
                dw[:, dz, dy, dx, :] = np.tensordot(g, xp[dz:dz + D, dy:dy + H, dx:dx + W],
                                                    axes=([0, 1, 2], [0, 1, 2]))
    return dw


def conv3_dgrad(gz: np.ndarray, w: np.ndarray) -> np.ndarray:
    """dloss/dx for out = conv3(x, w): the correlation of gz with the weights
    mirrored in all three axes and transposed in channels."""
    wf = np.asarray(w, dtype=np.float64)[:, ::-1, ::-1, ::-1, :].transpose(4, 1, 2, 3, 0)
    return conv3(gz, wf, np.zeros(wf.shape[0]), relu=False)


def pool2_backward(x: np.ndarray, gy: np.ndarray) -> np.ndarray:
    """Gradient of 2x2x2 max pooling: each window's gradient goes to the first
    voxel (in (dz, dy, dx) order) that holds the window maximum."""
    D, H, W, C = x.shape
    y = pool2(x)
    gx = np.zeros_like(np.asarray(x, dtype=np.float64))
    taken = np.zeros(y.shape, bool)
    for dz in range(2):
        for dy in range(2):
            for dx in range(2):
                xs = x[dz::2, dy::2, dx::2]
                hit = (xs == y) & ~taken
                gx[dz::2, dy::2, dx::2] = np.where(hit, gy, 0.0)
                taken |= hit
    return gx


def up2_backward(gy: np.ndarray) -> np.ndarray:
    """Gradient of nearest 2x upsampling: the sum over each 2x2x2 block."""
    D, H, W, C = gy.shape
    return np.asarray(gy, dtype=np.float64).reshape(D // 2, 2, H // 2, 2, W // 2, 2, C).sum(axis=(1, 3, 5))


def unet_loss_and_grad(dose, rho, target, flat_params, widths=WIDTHS, rounding: bool = True,
                       acts=None):
    """(loss, flat gradient) of the normalised MSE. acts: the 14 stored conv
    outputs to differentiate at (default: this module's forward pass)."""
    layers, (hw, hb) = unpack_params(flat_params, widths)
    rnd = bf16_round if rounding else (lambda a: np.asarray(a, dtype=np.float64))
    x0, dmax = pack_input(dose, rho)
    if not rounding:
        x0[..., 0] = np.asarray(dose, dtype=np.float64) / dmax
        x0[..., 1] = rho
    if acts is None:
        _, acts = unet_forward(dose, rho, flat_params, widths, return_layers=True, rounding=rounding)
    a = acts
    e0, e1, e2 = a[1], a[3], a[5]
    ins = [x0, a[0], pool2(e0), a[2], pool2(e1), a[4], pool2(e2), a[6],
           np.concatenate([e2, up2(a[7])], 3), a[8],
           np.concatenate([e1, up2(a[9])], 3), a[10],
           np.concatenate([e0, up2(a[11])], 3), a[12]]
    dn = np.asarray(dose, dtype=np.float64) / dmax
    tn = np.asarray(target, dtype=np.float64) / dmax
    r = a[13] @ hw + hb
    res = dn + r - tn
    nvox = res.size
    loss = float(np.mean(res ** 2))
    g_r = 2.0 * res / nvox
    g_hw = np.tensordot(g_r, a[13], axes=([0, 1, 2], [0, 1, 2]))
    g_hb = g_r.sum()
    grads = [None] * 14
    g_out = {13: g_r[..., None] * hw}

    def layer_back(i, gy):
        w, _ = layers[i]
        gz = gy * (a[i] > 0)
        grads[i] = (conv3_wgrad(ins[i], gz), gz.sum(axis=(0, 1, 2)))
        return conv3_dgrad(gz, rnd(w)) if i > 0 else None

    c0, c1, c2, _ = widths
    g = layer_back(13, g_out[13])
    g = layer_back(12, g)                                  # gradient of cat(e0, up2(d1))
    g_e0_skip, g_d1 = g[..., :c0], up2_backward(g[..., c0:])
    g = layer_back(11, g_d1)
    g = layer_back(10, g)                                  # cat(e1, up2(d2))
    g_e1_skip, g_d2 = g[..., :c1], up2_backward(g[..., c1:])
    g = layer_back(9, g_d2)
    g = layer_back(8, g)                                   # cat(e2, up2(b))
    g_e2_skip, g_b = g[..., :c2], up2_backward(g[..., c2:])
    g = layer_back(7, g_b)
    g = layer_back(6, g)                                   # gradient of pool2(e2)
    g = layer_back(5, g_e2_skip + pool2_backward(e2, g))
    g = layer_back(4, g)
    g = layer_back(3, g_e1_skip + pool2_backward(e1, g))
    g = layer_back(2, g)
    g = layer_back(1, g_e0_skip + pool2_backward(e0, g))
    layer_back(0, g)
    flat = []
    for i in range(14):
        flat += [grads[i][0].ravel(), grads[i][1]]
    flat += [g_hw, np.array([g_hb])]
    return loss, np.concatenate(flat)
