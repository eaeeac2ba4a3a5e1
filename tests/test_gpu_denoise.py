"""GPU parity of the denoiser kernels (tcgen05 3x3x3 convolution, pooling,
upsampling, the U-Net forward) against the FP64 oracle in oracle/denoise.py.

Both sides use the same BF16 inputs and weights. A convolution output is the
FP32 tensor-core sum of K = 27 c_in products rounded once to BF16, so
|gpu - ref| <= 2^-8 |ref| + 2 K 2^-23 S, S the sum of the magnitudes of all
terms (oracle.denoise.conv3_abs); pooling and upsampling move stored values and
are bit-exact."""
import numpy as np
import pytest

from oracle import denoise as DN

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def L():
    from paper_1503_01725_b300 import lsm
    lsm.load_library()
    return lsm


def to_vol(L, x, c_total=None, c_offset=0, fill=0.0):
    import torch
    n, d, h, w, c = x.shape
    t = L.alloc_vol(n, d, h, w, c_total or c)
    if fill:
        t[:, 1:-1, 1:-1, 1:-1] = fill
    t[:, 1:-1, 1:-1, 1:-1, c_offset:c_offset + c] = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16)
    return t


def interior(t, c_offset=0, c=None):
    c = t.shape[-1] - c_offset if c is None else c
    return t[:, 1:-1, 1:-1, 1:-1, c_offset:c_offset + c].double().cpu().numpy()


def conv_tolerance(x, w, b, ref):
    k = 27 * w.shape[-1]
    return 2.0 ** -8 * np.abs(ref) + 2 * k * 2.0 ** -23 * DN.conv3_abs(x, w, b) + 1e-30


def rand_bf16(rng, shape, scale=1.0):
    return DN.bf16_round(rng.standard_normal(shape) * scale)


CONFIGS = [(16, 16), (32, 16), (16, 32), (32, 32), (64, 32), (32, 64), (64, 64), (128, 64), (64, 128), (16, 128),
           (128, 16)]


@pytest.mark.parametrize("cin,cout", CONFIGS)
@pytest.mark.parametrize("relu", [True, False])
def test_conv3d_matches_oracle(L, cin, cout, relu):
    import torch
    rng = np.random.default_rng(cin * 7 + cout + relu)
    n, d, h, w = 2, 5, 6, 7                    # ragged: tiles straddle rows, planes and volumes
    x = rand_bf16(rng, (n, d, h, w, cin))
    wt = rand_bf16(rng, (cout, 3, 3, 3, cin), 1.0 / np.sqrt(27 * cin))
    b = rand_bf16(rng, cout, 0.1)
    conv = L.lsm_conv3d_create(cin, cout, wt, b, relu=relu)
    tin = to_vol(L, x, c_total=cin + 16, c_offset=16, fill=7.0)   # read a channel slice
    tout = to_vol(L, np.zeros((n, d, h, w, cout)), c_total=cout + 16, c_offset=8, fill=3.0)
    # interior rows are written whole, their two x-halo voxels as zero: plant
    # garbage there first (the other halo voxels must already be zero)
    tout[:, 1:-1, 1:-1, 0, 8:8 + cout] = 5.0
    tout[:, 1:-1, 1:-1, -1, 8:8 + cout] = 5.0
    L.lsm_conv3d_forward(conv, L.vol(tin, 16, cin), L.vol(tout, 8, cout))
    torch.cuda.synchronize()
    got = interior(tout, 8, cout)
    for i in range(n):
        ref = DN.conv3(x[i], wt, b, relu)
        err = np.abs(got[i] - ref)
        tol = conv_tolerance(x[i], wt, b, ref)
        assert np.all(err <= tol), (err / tol).max()
    o = tout.double().cpu().numpy()
    halo = np.ones(o.shape[:4], bool)
    halo[:, 1:-1, 1:-1, 1:-1] = False
    assert not o[halo][:, 8:8 + cout].any()
    assert np.all(o[~halo][:, :8] == 3.0) and np.all(o[~halo][:, 8 + cout:] == 3.0)


def test_conv3d_many_tiles_per_cta(L):
    """64^3 volume (2178 tiles) on one CTA per SM: every CTA runs ~15 tiles
    through both tensor-memory accumulators and the stage ring."""
    import torch
    rng = np.random.default_rng(11)
    x = rand_bf16(rng, (1, 64, 64, 64, 32))
    wt = rand_bf16(rng, (32, 3, 3, 3, 32), 0.03)
    b = rand_bf16(rng, 32, 0.1)
    conv = L.lsm_conv3d_create(32, 32, wt, b, relu=True)
    tin, tout = to_vol(L, x), L.alloc_vol(1, 64, 64, 64, 32)
    L.lsm_conv3d_forward(conv, L.vol(tin), L.vol(tout), ctas_per_sm=1)
    torch.cuda.synchronize()
    got = interior(tout)[0]
    ref = DN.conv3(x[0], wt, b, True)
    assert np.all(np.abs(got - ref) <= conv_tolerance(x[0], wt, b, ref))


def test_pool_and_upsample_bit_exact(L):
    import torch
    rng = np.random.default_rng(12)
    x = rand_bf16(rng, (2, 6, 4, 8, 24))
    tin = to_vol(L, x, c_total=32, c_offset=8)
    tp = L.alloc_vol(2, 3, 2, 4, 24)
    L.lsm_pool3d(L.vol(tin, 8, 24), L.vol(tp))
    tu = L.alloc_vol(2, 6, 4, 8, 40)
    L.lsm_upsample3d(L.vol(tp), L.vol(tu, 16, 24))
    torch.cuda.synchronize()
    p = interior(tp)
    for i in range(2):
        assert np.array_equal(p[i], DN.pool2(x[i]))
        assert np.array_equal(interior(tu, 16, 24)[i], DN.up2(DN.pool2(x[i])))
    assert not interior(tu, 0, 16).any()
    assert not tu[:, 0].double().abs().sum().item()


def _gpu_layer_inputs(acts, x0):
    """Input of each conv layer built from the GPU's stored activations."""
    e0, e1, e2 = acts[1], acts[3], acts[5]
    return [x0, acts[0], DN.pool2(e0), acts[2], DN.pool2(e1), acts[4], DN.pool2(e2), acts[6],
            np.concatenate([e2, DN.up2(acts[7])], 3), acts[8],
            np.concatenate([e1, DN.up2(acts[9])], 3), acts[10],
            np.concatenate([e0, DN.up2(acts[11])], 3), acts[12]]


def test_unet_forward_layer_by_layer(L):
    rng = np.random.default_rng(13)
    n, d, h, w = 2, 16, 24, 16
    dose = rng.random((n, d, h, w)).astype(np.float32) * 3.0
    rho = (0.5 + rng.random((n, d, h, w))).astype(np.float32)
    params = DN.init_params(3, head_scale=0.05)
    params[-1] = 0.01
    net = L.lsm_unet_create(params)
    out = L.lsm_unet_forward(net, dose, rho)
    layers, (hw, hb) = DN.unpack_params(params)
    convs, _ = DN.layer_shapes()
    for i in range(n):
        x0, dmax = DN.pack_input(dose[i].astype(np.float64), rho[i].astype(np.float64))
        acts = []
        for li, (ci, co) in enumerate(convs):
            lv = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0][li]
            a = L.lsm_unet_activation(net, li, (n, d >> lv, h >> lv, w >> lv, co))
            acts.append(a[i])
        ins = _gpu_layer_inputs(acts, x0)
        for li in range(14):
            wb, bb = DN.bf16_round(layers[li][0]), DN.bf16_round(layers[li][1])
            ref = DN.conv3(ins[li], wb, bb, True)
            err = np.abs(acts[li] - ref)
            tol = conv_tolerance(ins[li], wb, bb, ref)
            assert np.all(err <= tol), (li, (err / tol).max())
        # head on the GPU's last activation, FP32 on the device
        head = dose[i].astype(np.float64) + dmax * (acts[13] @ hw + hb)
        np.testing.assert_allclose(out[i], head, rtol=1e-5, atol=1e-5 * dmax)
        # end to end against the oracle's own forward pass (its BF16 roundings can
        # differ from the GPU's by one unit where FP32 and FP64 sums straddle a
        # rounding boundary, and such differences propagate)
        ref = DN.unet_forward(dose[i], rho[i], params)
        rel = np.linalg.norm(out[i] - ref) / np.linalg.norm(ref - dose[i])
        assert rel < 0.05


def test_unet_device_buffers_and_untrained_identity(L):
    import torch
    rng = np.random.default_rng(14)
    dose = torch.tensor(rng.random((8, 16, 32)), dtype=torch.float32, device="cuda")
    rho = torch.ones_like(dose)
    net = L.lsm_unet_create(DN.init_params(4, head_scale=0.0))
    out = L.lsm_unet_forward(net, dose, rho)
    torch.cuda.synchronize()
    assert torch.equal(out, dose)


def _acts(L, net, n, d, h, w):
    convs, _ = DN.layer_shapes()
    lv = [0, 0, 1, 1, 2, 2, 3, 3, 2, 2, 1, 1, 0, 0]
    return [L.lsm_unet_activation(net, i, (n, d >> lv[i], h >> lv[i], w >> lv[i], co))
            for i, (ci, co) in enumerate(convs)]


def test_training_gradient_matches_oracle(L):
    """Gradients of one training step (lr = 0) against the oracle's backward
    pass taken at the GPU's own stored activations. Activation gradients are
    stored in BF16 on the GPU (about 2^-8 relative per store, compounding over
    the 14 layers), so each layer's gradient is compared in relative L2 norm
    and direction; the head's gradient is an FP32 sum and is compared tightly."""
    import torch
    rng = np.random.default_rng(21)
    n, d, h, w = 1, 16, 16, 24
    dose = (rng.random((n, d, h, w)) * 2 + 0.1).astype(np.float32)
    rho = (0.5 + rng.random((n, d, h, w))).astype(np.float32)
    target = (dose * (1 + 0.2 * rng.standard_normal(dose.shape))).astype(np.float32)
    params = DN.init_params(6, head_scale=0.1)
    params[:-17] += 0.002 * rng.standard_normal(params.size - 17)
    net = L.lsm_unet_create(params)
    t = [torch.tensor(a, device="cuda") for a in (dose, rho, target)]
    loss = L.lsm_unet_train_step(net, *t, lr=0.0)
    g = L.lsm_unet_grad(net).astype(np.float64)
    acts = [a[0] for a in _acts(L, net, n, d, h, w)]
    p32 = params.astype(np.float32).astype(np.float64)
    lo, go = DN.unet_loss_and_grad(dose[0].astype(np.float64), rho[0].astype(np.float64),
                                   target[0].astype(np.float64), p32, acts=acts)
    assert loss == pytest.approx(lo, rel=1e-4)
    convs, (hc, _) = DN.layer_shapes()
    k = 0
    for i, (ci, co) in enumerate(convs):
        nw = 27 * ci * co
        for part in (slice(k, k + nw), slice(k + nw, k + nw + co)):
            a, b = g[part], go[part]
            if i == 0 and part.stop == k + nw:
                a = a.reshape(co, 27, ci)[..., :2].ravel()      # only the real input channels
                b = b.reshape(co, 27, ci)[..., :2].ravel()
            rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
            cos = a @ b / max(np.linalg.norm(a) * np.linalg.norm(b), 1e-30)
            assert rel < 0.05 and cos > 0.998, (i, rel, cos)
        k += nw + co
    np.testing.assert_allclose(g[k:], go[k:], rtol=2e-3, atol=1e-6 * np.abs(go[k:]).max())


@pytest.mark.parametrize("shape", [(1, 16, 16, 24), (2, 24, 40, 16), (1, 64, 64, 64)])
def test_tensor_core_weight_gradients_equal_cuda_core_ones(L, shape):
    """The tcgen05 weight gradient (GEMM over voxels on channel-major copies)
    against the FP32 CUDA-core one on the same training step: both multiply the
    same BF16 values (exact in FP32) and differ only in the order of the FP32
    sums, layer by layer. Shapes with ragged rows, two volumes, several row
    tiles and chunk splits."""
    import torch
    n, d, h, w = shape
    rng = np.random.default_rng(23)
    dose = (rng.random(shape) * 2 + 0.1).astype(np.float32)
    rho = (0.5 + rng.random(shape)).astype(np.float32)
    target = (dose * (1 + 0.2 * rng.standard_normal(shape))).astype(np.float32)
    params = DN.init_params(8, head_scale=0.1)
    t = [torch.tensor(a, device="cuda") for a in (dose, rho, target)]
    grads = []
    try:
        for tc in (False, True):
            L.lsm_unet_set_wgrad(tc)
            net = L.lsm_unet_create(params)
            L.lsm_unet_train_step(net, *t, lr=0.0)
            grads.append(L.lsm_unet_grad(net).astype(np.float64))
    finally:
        L.lsm_unet_set_wgrad(True)
    g0, g1 = grads
    convs, _ = DN.layer_shapes()
    k = 0
    for i, (ci, co) in enumerate(convs):
        nw = 27 * ci * co
        a, b = g1[k:k + nw], g0[k:k + nw]
        rel = np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
        assert rel < 2e-5, (i, ci, co, rel)
        # bias and head: the same kernels in both modes (FP32 atomics: order only)
        b1, b0 = g1[k + nw:k + nw + co], g0[k + nw:k + nw + co]
        np.testing.assert_allclose(b1, b0, rtol=1e-5, atol=1e-5 * np.abs(b0).max())
        k += nw + co
    np.testing.assert_allclose(g1[k:], g0[k:], rtol=1e-5, atol=1e-5 * np.abs(g0[k:]).max())


def test_training_reduces_loss(L):
    """Adam steps on a fixed pair lower the loss: the target is a smoothed,
    rescaled copy of the input, a mapping the network can represent."""
    import torch
    from scipy import ndimage
    rng = np.random.default_rng(22)
    n, d, h, w = 2, 16, 16, 16
    zz, yy, xx = np.meshgrid(*[np.linspace(-1, 1, s) for s in (d, h, w)], indexing="ij")
    clean = np.exp(-(xx ** 2 + yy ** 2) * 3) * np.exp(-0.5 * (zz + 1))
    dose = np.stack([clean, 0.7 * clean]) * (1 + 0.3 * rng.standard_normal((n, d, h, w)))
    dose = dose.clip(0).astype(np.float32)
    target = (0.6 * np.stack([ndimage.uniform_filter(x, 3) for x in dose])).astype(np.float32)
    rho = np.ones_like(dose)
    net = L.lsm_unet_create(DN.init_params(7, head_scale=0.01))
    t = [torch.tensor(a, device="cuda") for a in (dose, rho, target)]
    losses = [L.lsm_unet_train_step(net, *t, lr=3e-3) for _ in range(80)]
    assert losses[-1] < 0.3 * losses[0], losses[::10]
    p = L.lsm_unet_params(net)
    assert np.all(np.isfinite(p))
    # inference with the trained parameters agrees with the training forward pass
    out = L.lsm_unet_forward(net, dose, rho)
    err = np.mean(((out - target) / dose.reshape(n, -1).max(1)[:, None, None, None]) ** 2)
    assert err < losses[0]


def test_replayed_forward_graph_follows_weights_and_shapes(L):
    """The layers between input packing and the head run as a captured CUDA
    graph from the second forward on: repeated forwards are identical; after
    training steps change the weights, the replayed graph gives what a fresh
    network with the new parameters gives; a new shape rebuilds it."""
    import torch
    rng = np.random.default_rng(5)
    n, d, h, w = 1, 16, 16, 24
    dose = rng.random((n, d, h, w)).astype(np.float32)
    rho = (0.5 + rng.random((n, d, h, w))).astype(np.float32)
    target = (0.8 * dose).astype(np.float32)
    net = L.lsm_unet_create(DN.init_params(9, head_scale=0.05))
    outs = [L.lsm_unet_forward(net, dose, rho) for _ in range(3)]   # direct, captured + replayed, replayed
    np.testing.assert_array_equal(outs[1], outs[0])
    np.testing.assert_array_equal(outs[2], outs[0])
    t = [torch.tensor(a, device="cuda") for a in (dose, rho, target)]
    for _ in range(3):
        L.lsm_unet_train_step(net, *t, lr=1e-2)
    after = L.lsm_unet_forward(net, dose, rho)
    fresh = L.lsm_unet_create(L.lsm_unet_params(net))
    np.testing.assert_array_equal(after, L.lsm_unet_forward(fresh, dose, rho))
    assert np.abs(after - outs[0]).max() > 0
    # a caller capturing the forward into its own graph gets the same result
    s_ = torch.cuda.Stream()
    dd, rr = torch.tensor(dose, device="cuda"), torch.tensor(rho, device="cuda")
    o_ = torch.empty_like(dd)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s_):
        L.lsm_unet_forward(net, dd, rr, out=o_, stream=s_)
    g.replay()
    torch.cuda.synchronize()
    np.testing.assert_array_equal(o_.cpu().numpy(), after)
    # another shape: new buffers, a new graph
    d2 = rng.random((2, 8, 16, 16)).astype(np.float32)
    r2 = np.ones_like(d2)
    a2 = [L.lsm_unet_forward(net, d2, r2) for _ in range(3)]
    np.testing.assert_array_equal(a2[2], a2[0])
    np.testing.assert_array_equal(L.lsm_unet_forward(net, dose, rho), after)


def test_gamma_and_dose_error_match_oracle(L):
    from oracle import gamma as G
    rng = np.random.default_rng(23)
    d, h, w = 24, 20, 28
    z, y, x = np.meshgrid(*[np.arange(s, dtype=float) for s in (d, h, w)], indexing="ij")
    # a flat-topped field: a 4 % excess fails on the plateau, passes in the penumbra
    r = np.sqrt((x - 14) ** 2 + (y - 10) ** 2)
    ref = 1.0 / (1 + np.exp(r - 7)) * (1 + 0.0 * z)
    ev = ref * 1.04 * (1 + 0.01 * rng.standard_normal(ref.shape))
    ref32, ev32 = ref.astype(np.float32), ev.astype(np.float32)
    for vox, crit, dta in (((2.5, 2.5, 2.5), 0.02, 2.0), ((2.0, 3.0, 1.5), 0.03, 3.0)):
        rate, n, pm = L.lsm_gamma(ev32, ref32, vox, crit, dta, pass_map=True)
        rate_o, n_o = G.gamma_pass_rate(ev32, ref32, vox, crit, dta)
        assert n == n_o
        assert abs(rate - rate_o) <= 2e-3, (rate, rate_o)
        assert 0.05 < rate < 0.999                      # a case with both outcomes
    sig = (0.01 * ref).astype(np.float32)
    e = L.lsm_dose_error(ev32, ref32, sig)
    assert e == pytest.approx(G.rms_relative_error(ev32, ref32, sig), rel=1e-5)


def test_trained_denoiser_on_a_held_out_case(L):
    """Full size (128^3, config of the denoiser workload): the committed
    weights on held-out case 192 (5 cm field, heterogeneous phantom), judged
    against a 1e9-history run: the denoised 1e6-history dose has a lower RMS
    error than the 1e8-history dose and passes gamma 2 %/2 mm on >= 99 %."""
    from paper_1503_01725_b300 import denoiser as DZ
    net = DZ.load()
    p = DZ.generate([192], n_lo=1_000_000, n_hi=100_000_000, n_ref=1_000_000_000)[0]
    row = DZ.evaluate(net, [p])[0]
    assert row["denoised_rms"] < row["target_hi_rms"] < row["mc_lo_rms"]
    assert row["denoised_gamma"] >= 0.99
