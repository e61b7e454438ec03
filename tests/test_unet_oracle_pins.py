"""Pins of the FP64 U-Net oracle against things other than itself: a library correlation,
brute-force loops, adjoint identities, central differences of the forward pass and the
closed forms of Adam's bias correction."""
import numpy as np
import pytest
from scipy import signal

from oracle import unet_oracle as U


def test_conv3x3_matches_scipy_correlation():
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 7, 9, 3))
    w = rng.standard_normal((4, 3, 3, 3))
    b = rng.standard_normal(4)
    y = U.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate2d(x[n, :, :, i], w[o, :, :, i], mode="same",
                                                boundary="fill", fillvalue=0.0) for i in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_conv3x3_centre_tap_is_conv1x1():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 5, 6, 3))
    w1 = rng.standard_normal((2, 3))
    b = rng.standard_normal(2)
    w3 = np.zeros((2, 3, 3, 3))
    w3[:, 1, 1, :] = w1
    np.testing.assert_allclose(U.conv3x3(x, w3, b), U.conv1x1(x, w1, b), rtol=1e-13, atol=1e-13)


def test_pool_and_upsample_brute_force():
    rng = np.random.default_rng(3)
    x = rng.standard_normal((2, 6, 8, 3))
    p = U.maxpool2(x)
    for n in range(2):
        for h in range(3):
            for w in range(4):
                for c in range(3):
                    assert p[n, h, w, c] == max(x[n, 2 * h + a, 2 * w + d, c]
                                                for a in range(2) for d in range(2))
    u = U.upsample2(p)
    for h in range(6):
        for w in range(8):
            np.testing.assert_array_equal(u[:, h, w, :], p[:, h // 2, w // 2, :])
    # the backward of upsampling is its adjoint
    y = rng.standard_normal(u.shape)
    assert np.sum(u * y) == pytest.approx(np.sum(p * U.upsample2_backward(y)), rel=1e-13)


def test_maxpool_backward_first_maximum_and_differences():
    x = np.array([[1.0, 3.0], [3.0, 2.0]]).reshape(1, 2, 2, 1)
    dx = U.maxpool2_backward(x, np.full((1, 1, 1, 1), 5.0))
    np.testing.assert_array_equal(dx.reshape(2, 2), [[0.0, 5.0], [0.0, 0.0]])
    rng = np.random.default_rng(4)
    x = rng.standard_normal((1, 4, 6, 2))
    dy = rng.standard_normal((1, 2, 3, 2))
    g = U.maxpool2_backward(x, dy)
    h = 1e-6
    for idx in [(0, 0, 0, 0), (0, 3, 5, 1), (0, 1, 2, 0), (0, 2, 3, 1)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += h
        xm[idx] -= h
        fd = (np.sum(U.maxpool2(xp) * dy) - np.sum(U.maxpool2(xm) * dy)) / (2 * h)
        assert fd == pytest.approx(g[idx], abs=1e-8)


def test_network_shapes_and_counts():
    assert U.param_count(4, 32, 4, 2) == 1947202
    # about 10.6 GFLOP per 256x128 sample
    assert U.flops_per_sample(4, 32, 4, 2, 128, 256) == pytest.approx(10.65e9, rel=1e-3)
    rng = np.random.default_rng(5)
    p = U.init_params(rng, 3, 4, 4, 2)
    y = U.forward(p, rng.standard_normal((2, 8, 12, 4)), 3, 4, 4, 2)
    assert y.shape == (2, 8, 12, 2)


@pytest.mark.parametrize("levels,base,H,W", [(2, 3, 4, 6), (3, 2, 8, 12), (4, 2, 8, 16)])
def test_gradient_matches_central_differences(levels, base, H, W):
    """Every layer's weight and bias gradient and the masked loss, against central
    differences of the FP64 forward pass."""
    rng = np.random.default_rng(10 + levels)
    cin, cout, n = 4, 2, 2
    p = U.init_params(rng, levels, base, cin, cout)
    x = rng.standard_normal((n, H, W, cin))
    t = rng.standard_normal((n, H, W, cout))
    mask = (rng.random((n, H, W)) > 0.3).astype(np.float64)
    L, g, y = U.loss_and_gradient(p, x, t, mask, levels, base, cin, cout)
    L2, _ = U.loss(U.forward(p, x, levels, base, cin, cout), t, mask)
    assert L == pytest.approx(L2, rel=1e-14)
    # sample entries of every parameter block
    idx, off = [], 0
    for _, k, ci, co in U.layer_shapes(levels, base, cin, cout):
        nw = k * k * ci * co
        idx += list(off + rng.choice(nw, size=min(nw, 4), replace=False))
        idx += [off + nw + int(rng.integers(co))]
        off += nw + co
    h = 1e-6
    for i in idx:
        pp, pm = p.copy(), p.copy()
        pp[i] += h
        pm[i] -= h
        Lp, _ = U.loss(U.forward(pp, x, levels, base, cin, cout), t, mask)
        Lm, _ = U.loss(U.forward(pm, x, levels, base, cin, cout), t, mask)
        fd = (Lp - Lm) / (2 * h)
        assert fd == pytest.approx(g[i], rel=1e-5, abs=1e-9), i


def test_loss_closed_form_and_mask():
    y = np.full((1, 2, 2, 2), 3.0)
    t = np.full((1, 2, 2, 2), 1.0)
    L, dy = U.loss(y, t)
    assert L == pytest.approx(0.5 * 4.0)   # mean of (3-1)^2 / 2
    np.testing.assert_allclose(dy, 2.0 / 8)
    L0, dy0 = U.loss(y, t, np.zeros((1, 2, 2)))
    assert L0 == 0.0 and not dy0.any()


def test_adam_bias_correction_closed_forms():
    """With a constant gradient g the corrected moments are exactly g and g^2 at every step,
    so each step moves w by lr g / (|g| + eps) (Kingma & Ba, Sec. 3)."""
    g = np.array([0.3, -2.0, 1e-3])
    w = np.array([1.0, 2.0, 3.0])
    m = np.zeros(3)
    v = np.zeros(3)
    lr, eps = 0.01, 1e-8
    for step in range(1, 6):
        w_new, m, v = U.adam_step(w, g, m, v, step, lr, eps=eps)
        np.testing.assert_allclose(w - w_new, lr * g / (np.abs(g) + eps), rtol=1e-10)
        w = w_new


def test_training_reduces_loss_on_a_tiny_problem():
    rng = np.random.default_rng(7)
    levels, base, cin, cout = 2, 4, 4, 2
    p = U.init_params(rng, levels, base, cin, cout)
    x = rng.standard_normal((4, 4, 8, cin))
    t = 0.5 * x[..., :2] - 0.25 * x[..., 2:]
    m = np.zeros_like(p)
    v = np.zeros_like(p)
    L0 = None
    for step in range(1, 101):
        L, g, _ = U.loss_and_gradient(p, x, t, None, levels, base, cin, cout)
        L0 = L if L0 is None else L0
        p, m, v = U.adam_step(p, g, m, v, step, 3e-3)
    assert L < 0.5 * L0


def test_bf16_rounding_matches_the_format_and_torch():
    """Nearest BF16 value with ties to even: hand-worked bit patterns, then torch's own
    float32 -> bfloat16 conversion on random values (a library routine)."""
    import torch
    e = 2.0 ** -8
    cases = {1.0: 1.0, 1 + e: 1.0, 1 + 3 * e: 1 + 4 * e, 1 + e + 2.0 ** -20: 1 + 2 * e,
             -(1 + 3 * e): -(1 + 4 * e), 0.0: 0.0, 3.0: 3.0}
    for x, want in cases.items():
        assert U.bf16(np.array([x]))[0] == want, x
    rng = np.random.default_rng(0)
    v = (rng.standard_normal(100000) * 10.0 ** rng.uniform(-20, 20, 100000)).astype(np.float32)
    ref = torch.from_numpy(v).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(U.bf16(v), ref)
    np.testing.assert_array_equal(U.bf16(U.bf16(v)), U.bf16(v))


def test_storage_rounding_stays_near_fp64():
    """Rounding the stored operands to BF16 moves the output by about 1e-2 of itself at most
    (the envelope the GPU comparison with the plain FP64 oracle relies on)."""
    rng = np.random.default_rng(8)
    lv, b, ci, co = 3, 8, 4, 2
    p = U.init_params(rng, lv, b, ci, co)
    x = rng.standard_normal((2, 16, 24, ci))
    y0 = U.forward(p, x, lv, b, ci, co)
    y1 = U.forward(p, x, lv, b, ci, co, quantize=U.bf16)
    r = np.linalg.norm(y1 - y0) / np.linalg.norm(y0)
    assert 1e-4 < r < 2e-2
