"""Pins of the FP64 U-Net oracle: library routines for each layer, brute-force SSIM, closed forms,
and finite differences for the hand-written backward pass."""
import math

import numpy as np
import pytest
from scipy import signal

from oracle import unet as U


def test_parameter_count_of_the_denoiser():
    n = sum(int(np.prod(s)) for _, s in U.param_shapes())
    assert n == 585363


def test_conv3x3_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv3x3(x, w, b)
    for n in range(2):
        for o in range(4):
            ref = b[o] + sum(signal.correlate(x[n, :, :, c], w[o, :, :, c], mode="same") for c in range(3))
            np.testing.assert_allclose(y[n, :, :, o], ref, rtol=1e-12, atol=1e-12)


def test_transposed_conv_is_a_kronecker_paint():
    rng = np.random.default_rng(1)
    x = rng.normal(size=(1, 3, 4, 1))
    w = rng.normal(size=(1, 2, 2, 1))
    y = U.convT2(x, w, np.zeros(1))
    np.testing.assert_allclose(y[0, :, :, 0], np.kron(x[0, :, :, 0], w[0, :, :, 0]), rtol=1e-14)


def test_maxpool_values_and_tie_rule():
    rng = np.random.default_rng(2)
    x = rng.normal(size=(1, 6, 8, 2))
    y, _ = U.maxpool2(x)
    np.testing.assert_array_equal(y[0, :, :, 1], x[0, :, :, 1].reshape(3, 2, 4, 2).max(axis=(1, 3)))
    t = np.ones((1, 2, 2, 1))
    _, arg = U.maxpool2(t)
    assert arg[0, 0, 0, 0] == 0  # first element of the window on ties
    g = U.maxpool2_backward(np.ones((1, 1, 1, 1)), arg, t.shape)
    np.testing.assert_array_equal(g[0, :, :, 0], [[1, 0], [0, 0]])


def _ssim_bruteforce(x, y):
    g1 = U.gaussian11()
    g2 = np.outer(g1, g1)
    n, h, w, c = x.shape
    out = np.zeros((n, h - 10, w - 10, c))
    for a in range(n):
        for ch in range(c):
            for i in range(h - 10):
                for j in range(w - 10):
                    px, py = x[a, i:i + 11, j:j + 11, ch], y[a, i:i + 11, j:j + 11, ch]
                    mx, my = (g2 * px).sum(), (g2 * py).sum()
                    vx = (g2 * (px - mx) ** 2).sum()
                    vy = (g2 * (py - my) ** 2).sum()
                    cxy = (g2 * (px - mx) * (py - my)).sum()
                    out[a, i, j, ch] = ((2 * mx * my + U.C1) * (2 * cxy + U.C2)) / (
                        (mx * mx + my * my + U.C1) * (vx + vy + U.C2))
    return out


def test_ssim_matches_brute_force_windows_and_identity():
    rng = np.random.default_rng(3)
    x = rng.random((1, 14, 13, 2))
    y = x + 0.1 * rng.normal(size=x.shape)
    s, _ = U.ssim_map(x, y)
    np.testing.assert_allclose(s, _ssim_bruteforce(x, y), rtol=1e-10)
    s_id, _ = U.ssim_map(x, x)
    np.testing.assert_allclose(s_id, 1.0, rtol=1e-12)
    value, grad = U.loss(x, x)
    assert value == pytest.approx(0.0, abs=1e-12)
    np.testing.assert_allclose(grad, 0.0, atol=1e-12)
    assert abs(U.gaussian11().sum() - 1) < 1e-15


def test_loss_gradient_finite_differences():
    rng = np.random.default_rng(4)
    p = rng.random((1, 13, 12, 3))
    t = rng.random((1, 13, 12, 3))
    _, g = U.loss(p, t)
    eps = 1e-6
    for _ in range(25):
        idx = tuple(rng.integers(0, s) for s in p.shape)
        pp, pm = p.copy(), p.copy()
        pp[idx] += eps
        pm[idx] -= eps
        fd = (U.loss(pp, t)[0] - U.loss(pm, t)[0]) / (2 * eps)
        assert fd == pytest.approx(g[idx], rel=1e-5, abs=1e-10)


def test_network_gradients_finite_differences():
    """Tiny U-Net (2 levels, widths 4/8): d loss / d params and d loss / d input vs central differences."""
    chans = (4, 8)
    rng = np.random.default_rng(5)
    params = U.init_params(seed=1, in_ch=3, out_ch=3, chans=chans)
    for k in params:
        if k.endswith("_b"):
            params[k] = rng.normal(0, 0.1, params[k].shape)
    x = rng.random((1, 16, 16, 3))
    t = rng.random((1, 16, 16, 3))

    def f(pp, xx):
        y, _ = U.forward(pp, xx, chans)
        return U.loss(y, t)[0]

    y, cache = U.forward(params, x, chans)
    _, gy = U.loss(y, t)
    grads, gx = U.backward(params, cache, gy, chans)
    assert set(grads) == set(params)
    eps = 1e-6
    checked = 0
    for name in params:
        for _ in range(3):
            idx = tuple(rng.integers(0, s) for s in params[name].shape)
            pp = {k: v.copy() for k, v in params.items()}
            pm = {k: v.copy() for k, v in params.items()}
            pp[name][idx] += eps
            pm[name][idx] -= eps
            fd = (f(pp, x) - f(pm, x)) / (2 * eps)
            assert fd == pytest.approx(grads[name][idx], rel=1e-4, abs=1e-9), name
            checked += 1
    for _ in range(10):
        idx = tuple(rng.integers(0, s) for s in x.shape)
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert (f(params, xp) - f(params, xm)) / (2 * eps) == pytest.approx(gx[idx], rel=1e-4, abs=1e-9)
    assert checked >= 3 * len(params)


def test_adam_first_step_is_lr_times_sign():
    p = {"w": np.array([1.0, -2.0, 3.0])}
    g = {"w": np.array([0.5, -4.0, 1e-3])}
    m = {"w": np.zeros(3)}
    v = {"w": np.zeros(3)}
    U.adam_step(p, g, m, v, 1, lr=0.01)
    np.testing.assert_allclose(p["w"], [1.0 - 0.01, -2.0 + 0.01, 3.0 - 0.01], rtol=1e-6)


def test_bf16_rounding():
    x = np.array([1.0, 1.0 + 2 ** -8, 1.0 + 3 * 2 ** -9, -3.140625, 65504.0])
    r = U.bf16(x)
    # 8 significant bits: 1 + 2^-8 rounds to even (1.0); 1 + 3*2^-9 rounds up to 1 + 2^-7
    np.testing.assert_array_equal(r[:3], [1.0, 1.0, 1.0 + 2 ** -7])
    assert r[3] == -3.140625  # exactly representable
    assert r[4] == 65536.0  # 65504 = 1.1111111111b x 2^15 rounds up to 2^16


def test_bce_loss_closed_forms_and_finite_differences():
    """Binary cross-entropy with logits: y = 0 gives log 2 whatever the label; a confident right
    answer costs ~0, a confident wrong one ~|y|; the gradient matches central differences and
    channels 1, 2 carry none."""
    shape = (2, 5, 7, 3)
    zero = np.zeros(shape)
    t = np.zeros(shape)
    t[..., 0] = (np.arange(2 * 5 * 7).reshape(2, 5, 7) % 3 == 0)
    v, _ = U.loss_bce(zero, t)
    assert abs(v - np.log(2.0)) < 1e-15
    y = np.zeros(shape)
    y[..., 0] = np.where(t[..., 0] > 0, 30.0, -30.0)
    assert U.loss_bce(y, t)[0] < 1e-12
    assert abs(U.loss_bce(-y, t)[0] - 30.0) < 1e-9
    rng = np.random.default_rng(3)
    p = rng.normal(0, 2, shape)
    tt = rng.random(shape)
    v, g = U.loss_bce(p, tt)
    assert (g[..., 1:] == 0).all()
    for idx in [(0, 1, 2, 0), (1, 4, 6, 0), (0, 0, 0, 1)]:
        e = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += e
        pm[idx] -= e
        fd = (U.loss_bce(pp, tt)[0] - U.loss_bce(pm, tt)[0]) / (2 * e)
        assert abs(fd - g[idx]) < 1e-8


def test_linear_l2_loss_closed_forms_mean_minimiser_and_finite_differences():
    """Squared error in linear radiance on log1p-domain values: zero at the target, 1 where every
    linear value is off by 1, minimised over one prediction by the linear mean of noisy targets
    (not their log-domain median), gradient equal to central differences."""
    shape = (2, 3, 4, 3)
    rng = np.random.default_rng(5)
    t = np.log1p(rng.random(shape) * 4.0)
    assert U.loss_l2_linear(t, t)[0] == 0.0
    assert abs(U.loss_l2_linear(np.log1p(np.expm1(t) + 1.0), t)[0] - 1.0) < 1e-12
    # sparse, bright samples of one pixel: the linear mean minimises the loss
    samples = np.array([0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 0.0, 20.0])
    tt = np.log1p(samples).reshape(-1, 1)
    grid = np.linspace(0.0, 5.0, 5001)
    losses = [U.loss_l2_linear(np.full_like(tt, np.log1p(v)), tt)[0] for v in grid]
    assert abs(grid[int(np.argmin(losses))] - samples.mean()) <= 1e-3
    assert abs(grid[int(np.argmin(losses))] - np.median(samples)) > 2.0
    p = rng.normal(0.5, 0.8, shape)
    v, g = U.loss_l2_linear(p, t)
    for idx in [(0, 1, 2, 0), (1, 2, 3, 2), (0, 0, 0, 1)]:
        e = 1e-6
        pp, pm = p.copy(), p.copy()
        pp[idx] += e
        pm[idx] -= e
        fd = (U.loss_l2_linear(pp, t)[0] - U.loss_l2_linear(pm, t)[0]) / (2 * e)
        assert abs(fd - g[idx]) < 1e-8 * max(1.0, abs(fd))
