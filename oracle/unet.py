"""FP64 NumPy oracle of the U-Net denoiser (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU baseline use this module.  It
is the plain definition of the network the CUDA kernels implement, written with explicit loops
over the 3x3 taps and numpy contractions, and its backward pass derived by hand (checked against
finite differences in tests/test_oracle_unet.py).

Network (a U-Net in the family the paper trains, Sec. IV-A, after Ronneberger et al. 2015), for
channel widths c_0 .. c_{L-1}:
  encoder level l: [2x2 max-pool if l > 0] -> conv3x3 + ReLU -> conv3x3 + ReLU  (skip e_l)
  decoder level l (deepest first): 2x2 stride-2 transposed conv (c_{l+1} -> c_l, no ReLU)
      -> concat [upsampled, e_l] -> conv3x3 + ReLU -> conv3x3 + ReLU
  output: 1x1 conv c_0 -> out channels.
Zero padding, NHWC tensors, max-pool ties go to the first element of the window in row-major
order.  Loss: 0.16 * mean|p - t| + 0.84 * (1 - mean SSIM(p, t)), SSIM of Wang et al. (2004) with
an 11x11 Gaussian window (sigma 1.5), C1 = 0.01^2, C2 = 0.03^2, valid windows, mean over channels.
Optimiser: Adam (Kingma & Ba 2015), beta1 0.9, beta2 0.999, eps 1e-8, bias-corrected.
"""
from __future__ import annotations

import math

import numpy as np

L1_WEIGHT, SSIM_WEIGHT = 0.16, 0.84
C1, C2 = 0.01 ** 2, 0.03 ** 2


# ------------------------------------------------------------------------------------------
# parameters
# ------------------------------------------------------------------------------------------

def param_shapes(in_ch=11, out_ch=3, chans=(32, 48, 64, 128)):
    """Ordered (name, shape): conv weights (Cout, 3, 3, Cin), transposed-conv weights
    (Cin, 2, 2, Cout), output weights (Cout, Cin), biases (Cout,)."""
    L = len(chans)
    out = []
    cin = in_ch
    for l in range(L):
        out += [(f"enc{l}_c1_w", (chans[l], 3, 3, cin)), (f"enc{l}_c1_b", (chans[l],)),
                (f"enc{l}_c2_w", (chans[l], 3, 3, chans[l])), (f"enc{l}_c2_b", (chans[l],))]
        cin = chans[l]
    for l in reversed(range(L - 1)):
        out += [(f"up{l}_w", (chans[l + 1], 2, 2, chans[l])), (f"up{l}_b", (chans[l],)),
                (f"dec{l}_c1_w", (chans[l], 3, 3, 2 * chans[l])), (f"dec{l}_c1_b", (chans[l],)),
                (f"dec{l}_c2_w", (chans[l], 3, 3, chans[l])), (f"dec{l}_c2_b", (chans[l],))]
    out += [("out_w", (out_ch, chans[0])), ("out_b", (out_ch,))]
    return out


def init_params(seed=0, in_ch=11, out_ch=3, chans=(32, 48, 64, 128)):
    """He-normal weights, zero biases (seeded)."""
    rng = np.random.default_rng(seed)
    p = {}
    for name, shape in param_shapes(in_ch, out_ch, chans):
        if name.endswith("_b"):
            p[name] = np.zeros(shape)
        else:
            fan_in = int(np.prod(shape[1:])) if not name.startswith("up") else shape[0]
            p[name] = rng.normal(0.0, math.sqrt(2.0 / fan_in), shape)
    return p


# ------------------------------------------------------------------------------------------
# layers (forward and backward)
# ------------------------------------------------------------------------------------------

def conv3x3(x, w, b):
    """y[n,i,j,o] = b[o] + sum_{dy,dx,c} x[n,i+dy-1,j+dx-1,c] w[o,dy,dx,c], zero padded."""
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    y = np.zeros((n, h, wd, w.shape[0])) + b
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("nijc,oc->nijo", xp[:, dy:dy + h, dx:dx + wd, :], w[:, dy, dx, :])
    return y


def conv3x3_backward(x, w, gy):
    n, h, wd, _ = x.shape
    xp = np.pad(x, ((0, 0), (1, 1), (1, 1), (0, 0)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(3):
        for dx in range(3):
            gw[:, dy, dx, :] = np.einsum("nijo,nijc->oc", gy, xp[:, dy:dy + h, dx:dx + wd, :])
            gxp[:, dy:dy + h, dx:dx + wd, :] += np.einsum("nijo,oc->nijc", gy, w[:, dy, dx, :])
    return gxp[:, 1:h + 1, 1:wd + 1, :], gw, gy.sum(axis=(0, 1, 2))


def relu(x):
    return np.maximum(x, 0.0)


def maxpool2(x):
    """2x2 stride-2 max pool; returns the pooled tensor and the winning index 0..3 (row-major)."""
    n, h, w, c = x.shape
    v = x.reshape(n, h // 2, 2, w // 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(n, h // 2, w // 2, 4, c)
    arg = np.argmax(v, axis=3)  # first maximum on ties
    return np.take_along_axis(v, arg[:, :, :, None, :], axis=3)[:, :, :, 0, :], arg


def maxpool2_backward(gy, arg, shape):
    n, h, w, c = shape
    g = np.zeros((n, h // 2, w // 2, 4, c))
    np.put_along_axis(g, arg[:, :, :, None, :], gy[:, :, :, None, :], axis=3)
    return g.reshape(n, h // 2, w // 2, 2, 2, c).transpose(0, 1, 3, 2, 4, 5).reshape(n, h, w, c)


def convT2(x, w, b):
    """y[n,2i+a,2j+e,o] = b[o] + sum_c x[n,i,j,c] w[c,a,e,o]."""
    n, h, wd, _ = x.shape
    co = w.shape[3]
    y = np.zeros((n, 2 * h, 2 * wd, co)) + b
    for a in range(2):
        for e in range(2):
            y[:, a::2, e::2, :] += np.einsum("nijc,co->nijo", x, w[:, a, e, :])
    return y


def convT2_backward(x, w, gy):
    gx = np.zeros_like(x)
    gw = np.zeros_like(w)
    for a in range(2):
        for e in range(2):
            g = gy[:, a::2, e::2, :]
            gx += np.einsum("nijo,co->nijc", g, w[:, a, e, :])
            gw[:, a, e, :] = np.einsum("nijc,nijo->co", x, g)
    return gx, gw, gy.sum(axis=(0, 1, 2))


# ------------------------------------------------------------------------------------------
# network
# ------------------------------------------------------------------------------------------

def forward(p, x, chans):
    L = len(chans)
    cache = {"x": x}
    h = x
    for l in range(L):
        if l > 0:
            cache[f"pool{l}_in"] = h
            h, cache[f"pool{l}_arg"] = maxpool2(h)
        cache[f"enc{l}_c1_in"] = h
        h = relu(conv3x3(h, p[f"enc{l}_c1_w"], p[f"enc{l}_c1_b"]))
        cache[f"enc{l}_c2_in"] = h
        h = relu(conv3x3(h, p[f"enc{l}_c2_w"], p[f"enc{l}_c2_b"]))
        cache[f"enc{l}_out"] = h
    for l in reversed(range(L - 1)):
        cache[f"up{l}_in"] = h
        u = convT2(h, p[f"up{l}_w"], p[f"up{l}_b"])
        c = np.concatenate([u, cache[f"enc{l}_out"]], axis=-1)
        cache[f"dec{l}_c1_in"] = c
        h = relu(conv3x3(c, p[f"dec{l}_c1_w"], p[f"dec{l}_c1_b"]))
        cache[f"dec{l}_c2_in"] = h
        h = relu(conv3x3(h, p[f"dec{l}_c2_w"], p[f"dec{l}_c2_b"]))
        cache[f"dec{l}_out"] = h
    cache["out_in"] = h
    y = np.einsum("nijc,oc->nijo", h, p["out_w"]) + p["out_b"]
    return y, cache


def backward(p, cache, gy, chans):
    """Gradients of a scalar whose gradient w.r.t. the output is gy; returns (grads, grad of input)."""
    L = len(chans)
    g = {}
    h = cache["out_in"]
    g["out_w"] = np.einsum("nijo,nijc->oc", gy, h)
    g["out_b"] = gy.sum(axis=(0, 1, 2))
    gh = np.einsum("nijo,oc->nijc", gy, p["out_w"])
    skip_grad = {}
    for l in range(L - 1):
        gz = gh * (cache[f"dec{l}_out"] > 0)
        gh, g[f"dec{l}_c2_w"], g[f"dec{l}_c2_b"] = conv3x3_backward(cache[f"dec{l}_c2_in"], p[f"dec{l}_c2_w"], gz)
        gz = gh * (cache[f"dec{l}_c2_in"] > 0)
        gc, g[f"dec{l}_c1_w"], g[f"dec{l}_c1_b"] = conv3x3_backward(cache[f"dec{l}_c1_in"], p[f"dec{l}_c1_w"], gz)
        cu = chans[l]
        skip_grad[l] = gc[..., cu:]
        gh, g[f"up{l}_w"], g[f"up{l}_b"] = convT2_backward(cache[f"up{l}_in"], p[f"up{l}_w"], gc[..., :cu])
    for l in reversed(range(L)):
        if l < L - 1:
            gh = gh + skip_grad[l]
        gz = gh * (cache[f"enc{l}_out"] > 0)
        gh, g[f"enc{l}_c2_w"], g[f"enc{l}_c2_b"] = conv3x3_backward(cache[f"enc{l}_c2_in"], p[f"enc{l}_c2_w"], gz)
        gz = gh * (cache[f"enc{l}_c2_in"] > 0)
        gh, g[f"enc{l}_c1_w"], g[f"enc{l}_c1_b"] = conv3x3_backward(cache[f"enc{l}_c1_in"], p[f"enc{l}_c1_w"], gz)
        if l > 0:
            gh = maxpool2_backward(gh, cache[f"pool{l}_arg"], cache[f"pool{l}_in"].shape)
    return g, gh


# ------------------------------------------------------------------------------------------
# loss: L1 + (1 - SSIM)
# ------------------------------------------------------------------------------------------

def gaussian11(sigma=1.5):
    k = np.arange(11) - 5.0
    g = np.exp(-k * k / (2 * sigma * sigma))
    return g / g.sum()


def _blur(a, g):
    """Valid separable correlation of (n, h, w, c) with the 1-D kernel g along h and w."""
    k = len(g)
    n, h, w, c = a.shape
    t = sum(g[i] * a[:, i:h - k + 1 + i, :, :] for i in range(k))
    return sum(g[i] * t[:, :, i:w - k + 1 + i, :] for i in range(k))


def _blur_T(a, g, shape):
    """Adjoint of _blur: scatters (n, h-10, w-10, c) back to (n, h, w, c)."""
    k = len(g)
    n, h, w, c = shape
    t = np.zeros((n, a.shape[1], w, c))
    for i in range(k):
        t[:, :, i:w - k + 1 + i, :] += g[i] * a
    out = np.zeros(shape)
    for i in range(k):
        out[:, i:h - k + 1 + i, :, :] += g[i] * t
    return out


def ssim_map(x, y):
    g = gaussian11()
    mx, my = _blur(x, g), _blur(y, g)
    exx, eyy, exy = _blur(x * x, g), _blur(y * y, g), _blur(x * y, g)
    a1 = 2 * mx * my + C1
    a2 = 2 * (exy - mx * my) + C2
    b1 = mx * mx + my * my + C1
    b2 = (exx - mx * mx) + (eyy - my * my) + C2
    return a1 * a2 / (b1 * b2), (mx, my, a1, a2, b1, b2)


def loss(pred, target):
    """Returns (loss, d loss / d pred)."""
    s, (mx, my, a1, a2, b1, b2) = ssim_map(pred, target)
    l1 = np.abs(pred - target).mean()
    value = L1_WEIGHT * l1 + SSIM_WEIGHT * (1.0 - s.mean())
    g_l1 = np.sign(pred - target) / pred.size
    # d S / d (mu_x, E[x^2], E[xy]) per window, then the adjoint of the blur
    d_mx = (2 * my * a2 - 2 * my * a1) / (b1 * b2) - s * (2 * mx / b1 - 2 * mx / b2)
    d_exx = -s / b2
    d_exy = 2 * a1 / (b1 * b2)
    g = gaussian11()
    shp = pred.shape
    g_s = _blur_T(d_mx, g, shp) + 2 * pred * _blur_T(d_exx, g, shp) + target * _blur_T(d_exy, g, shp)
    grad = L1_WEIGHT * g_l1 - SSIM_WEIGHT * g_s / s.size
    return value, grad


def loss_bce(pred, target):
    """Segmentation loss (Sec. IV trains a U-Net to segment transparent objects and caustics):
    binary cross-entropy with the logit in channel 0 and the label in target channel 0, mean over
    pixels of -[t log s(y) + (1 - t) log(1 - s(y))], s the logistic function; channels 1 and 2 take
    no part.  Returns (loss, d loss / d pred)."""
    y = pred[..., 0].astype(np.float64)
    t = target[..., 0].astype(np.float64)
    s = 1.0 / (1.0 + np.exp(-y))
    n = y.size

    def softplus(z):  # log(1 + e^z) without overflow or cancellation
        return np.maximum(z, 0.0) + np.log1p(np.exp(-np.abs(z)))

    # log s(y) = -softplus(-y), log(1 - s(y)) = -softplus(y)
    value = float((t * softplus(-y) + (1.0 - t) * softplus(y)).sum() / n)
    grad = np.zeros(pred.shape)
    grad[..., 0] = (s - t) / n
    return value, grad


def loss_l2_linear(pred, target):
    """Squared error in linear radiance: prediction and target are in the network's log1p domain,
    the loss is the mean over pixels and the three channels of (expm1(y) - expm1(t))^2, so the
    minimiser over noisy targets is their mean in linear radiance (what an MSE against a reference
    measures), not a median in the log domain.  Returns (loss, d loss / d pred)."""
    y = pred.astype(np.float64)
    t = target.astype(np.float64)
    e = np.expm1(y) - np.expm1(t)
    n = y.size
    return float((e * e).sum() / n), 2.0 * e * np.exp(y) / n


# ------------------------------------------------------------------------------------------
# Adam
# ------------------------------------------------------------------------------------------

def adam_step(p, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One bias-corrected Adam step (t starts at 1); updates p, m, v in place."""
    for k in p:
        m[k] = b1 * m[k] + (1 - b1) * g[k]
        v[k] = b2 * v[k] + (1 - b2) * g[k] * g[k]
        mh = m[k] / (1 - b1 ** t)
        vh = v[k] / (1 - b2 ** t)
        p[k] = p[k] - lr * mh / (np.sqrt(vh) + eps)


def bf16(a):
    """Round to bfloat16 (nearest even) and back, the precision the GPU stores weights and activations in."""
    a = np.asarray(a, np.float32)
    u = a.view(np.uint32).astype(np.uint64)
    r = ((u + 0x7FFF + ((u >> 16) & 1)) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64)
