"""Torch-facing handle of the BF16 U-Net denoiser of ``include/sc_unet.h`` (marshalling only).

Every computation (forward, loss, backward, Adam) runs in the library's CUDA kernels; this module
passes torch device pointers through the C ABI.  The network is the U-Net family the paper uses for
its downstream evaluation (Sec. IV-A), here trained to denoise low-sample renders from the tracer's
own ground-truth buffers.
"""
from __future__ import annotations

import math

import numpy as np
import torch

from . import native as N
from .renderer import Context, Frame

CHANS = (32, 48, 64, 128)
IN_CH, OUT_CH = 11, 3


def param_shapes(in_ch=IN_CH, out_ch=OUT_CH, chans=CHANS):
    """(name, shape) of the flat parameter vector, in the ABI's order (see sc_unet.h)."""
    out = []
    cin = in_ch
    for l, c in enumerate(chans):
        out += [(f"enc{l}_c1_w", (c, 3, 3, cin)), (f"enc{l}_c1_b", (c,)),
                (f"enc{l}_c2_w", (c, 3, 3, c)), (f"enc{l}_c2_b", (c,))]
        cin = c
    for l in reversed(range(len(chans) - 1)):
        c, cn = chans[l], chans[l + 1]
        out += [(f"up{l}_w", (cn, 2, 2, c)), (f"up{l}_b", (c,)),
                (f"dec{l}_c1_w", (c, 3, 3, 2 * c)), (f"dec{l}_c1_b", (c,)),
                (f"dec{l}_c2_w", (c, 3, 3, c)), (f"dec{l}_c2_b", (c,))]
    out += [("out_w", (out_ch, chans[0])), ("out_b", (out_ch,))]
    return out


def flatten(params: dict) -> np.ndarray:
    return np.concatenate([np.asarray(params[k], np.float64).ravel() for k, _ in param_shapes()])


def unflatten(flat) -> dict:
    flat = np.asarray(flat)
    out, off = {}, 0
    for k, s in param_shapes():
        n = int(np.prod(s))
        out[k] = flat[off:off + n].reshape(s)
        off += n
    return out


def he_init(seed: int = 0) -> torch.Tensor:
    """He-normal weights and zero biases as a flat FP32 vector (seeded)."""
    g = torch.Generator().manual_seed(seed)
    parts = []
    for name, shape in param_shapes():
        if name.endswith("_b"):
            parts.append(torch.zeros(int(np.prod(shape))))
        else:
            fan_in = shape[0] if name.startswith("up") else int(np.prod(shape[1:]))
            parts.append(torch.randn(int(np.prod(shape)), generator=g) * math.sqrt(2.0 / fan_in))
    return torch.cat(parts).float()


def _ptr(t: torch.Tensor | None):
    if t is None:
        return None
    if not t.is_cuda or not t.is_contiguous():
        raise ValueError("device tensors must be contiguous CUDA tensors")
    return t.data_ptr()


class UNet:
    """An ``sc_unet`` with workspace for up to ``max_batch`` images of ``height x width``."""

    def __init__(self, ctx: Context, max_batch: int, height: int, width: int):
        self.ctx, self.max_batch, self.height, self.width = ctx, max_batch, height, width
        self.n_params = N.sc_unet_param_count()
        self.h = N.sc_unet_create(ctx.handle, max_batch, height, width)
        self.dev = torch.device("cuda", ctx.device)

    def close(self):
        if self.h:
            N.sc_unet_destroy(self.ctx.handle, self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # parameters -----------------------------------------------------------------------------
    def set_params(self, flat: torch.Tensor):
        flat = flat.to(self.dev, torch.float32).contiguous()
        if flat.numel() != self.n_params:
            raise ValueError(f"expected {self.n_params} parameters, got {flat.numel()}")
        N.sc_unet_set_params(self.ctx.handle, self.h, _ptr(flat))
        self.ctx.stream.synchronize()

    def get_params(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        N.sc_unet_get_params(self.ctx.handle, self.h, _ptr(out))
        return out

    def get_grads(self) -> torch.Tensor:
        out = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        N.sc_unet_get_grads(self.ctx.handle, self.h, _ptr(out))
        return out

    def set_grads(self, flat: torch.Tensor):
        flat = flat.to(self.dev, torch.float32).contiguous()
        N.sc_unet_set_grads(self.ctx.handle, self.h, _ptr(flat))
        self.ctx.stream.synchronize()

    # training state (checkpoint / resume) ----------------------------------------------------
    def get_state(self):
        """(params, adam_m, adam_v, step): the whole training state, device tensors + the step count."""
        m = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        v = torch.empty(self.n_params, dtype=torch.float32, device=self.dev)
        step = N.sc_unet_get_state(self.ctx.handle, self.h, _ptr(m), _ptr(v))
        return self.get_params(), m, v, step

    def set_state(self, params: torch.Tensor, m: torch.Tensor, v: torch.Tensor, step: int):
        p, m, v = (t.to(self.dev, torch.float32).contiguous() for t in (params, m, v))
        N.sc_unet_set_state(self.ctx.handle, self.h, _ptr(p), _ptr(m), _ptr(v), int(step))
        self.ctx.stream.synchronize()

    def set_loss(self, kind: int):
        """N.SC_UNET_LOSS_L1_SSIM (denoising) or N.SC_UNET_LOSS_BCE (segmentation logits in channel 0)."""
        N.sc_unet_set_loss(self.ctx.handle, self.h, int(kind))

    def save(self, path: str):
        N.sc_unet_save(self.ctx.handle, self.h, path)

    def load(self, path: str):
        N.sc_unet_load(self.ctx.handle, self.h, path)

    # compute --------------------------------------------------------------------------------
    def forward(self, x: torch.Tensor, y: torch.Tensor | None = None) -> torch.Tensor:
        n = x.shape[0]
        if y is None:
            y = torch.empty((n, self.height, self.width, OUT_CH), dtype=torch.float32, device=self.dev)
        N.sc_unet_forward(self.ctx.handle, self.h, _ptr(x), n, _ptr(y))
        return y

    def loss_grad(self, x: torch.Tensor, target: torch.Tensor):
        n = x.shape[0]
        y = torch.empty((n, self.height, self.width, OUT_CH), dtype=torch.float32, device=self.dev)
        loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        N.sc_unet_loss_grad(self.ctx.handle, self.h, _ptr(x), _ptr(target), n, _ptr(y), _ptr(loss))
        return y, loss

    def adam(self, lr: float):
        N.sc_unet_adam(self.ctx.handle, self.h, float(lr))

    def train_step(self, x: torch.Tensor, target: torch.Tensor, lr: float, loss: torch.Tensor | None = None):
        if loss is None:
            loss = torch.empty(1, dtype=torch.float32, device=self.dev)
        N.sc_unet_train_step(self.ctx.handle, self.h, _ptr(x), _ptr(target), x.shape[0], float(lr), _ptr(loss))
        return loss

    def buffer(self, name: str, level: int = 0) -> torch.Tensor:
        """A dense copy of one internal tensor (``sc_unet.h`` SC_UNET_BUF_*), [n, h, w, c]."""
        bid = N.SC_UNET_BUF[name]
        info = N.sc_unet_buffer(self.h, bid, level)
        dt = torch.bfloat16 if info.dtype == 0 else torch.float32
        out = torch.empty((info.n, info.h, info.w, info.c), dtype=dt, device=self.dev)
        N.sc_unet_copy_buffer(self.ctx.handle, self.h, bid, level, _ptr(out))
        return out


def ssim_l1_loss(ctx: Context, pred: torch.Tensor, target: torch.Tensor, want_grad: bool = True):
    """(loss [1], grad or None) of 0.16 L1 + 0.84 (1 - SSIM) for [n, h, w, 3] FP32 device tensors."""
    n, h, w, _ = pred.shape
    loss = torch.empty(1, dtype=torch.float32, device=pred.device)
    grad = torch.empty_like(pred) if want_grad else None
    N.sc_ssim_l1_loss(ctx.handle, _ptr(pred), _ptr(target), n, h, w, _ptr(loss), _ptr(grad))
    return loss, grad


SOURCES = {"rgb": N.SC_UNET_SRC_RGB, "direct": N.SC_UNET_SRC_DIRECT, "caustic": N.SC_UNET_SRC_CAUSTIC}


def pack_frame(ctx: Context, frame: Frame, x: torch.Tensor, index: int = 0, source: str = "rgb"):
    """Writes the 11-channel network input of ``frame`` into image ``index`` of x [n, H, W, 11];
    ``source`` picks the radiance estimate: the full image, the camera estimator alone or the
    light-traced caustic buffer alone."""
    N.sc_unet_pack_frame(ctx.handle, frame.struct(), SOURCES[source], _ptr(x), index)
    return x


def pack_target(ctx: Context, frame: Frame, t: torch.Tensor, index: int = 0, source: str = "rgb"):
    """Writes log1p of the frame's selected estimate into image ``index`` of t [n, H, W, 3]."""
    N.sc_unet_pack_target(ctx.handle, frame.struct(), SOURCES[source], _ptr(t), index)
    return t


def output_rgb(ctx: Context, y: torch.Tensor, add: torch.Tensor | None = None,
               out: torch.Tensor | None = None) -> torch.Tensor:
    """Linear RGB (float4 per pixel, w = 1) of network outputs y [..., 3], plus ``add`` (float4
    per pixel, e.g. the light-traced caustic buffer) when given."""
    rgb = out if out is not None else torch.empty(y.shape[:-1] + (4,), dtype=torch.float32, device=y.device)
    N.sc_unet_output_rgb(ctx.handle, _ptr(y), y.numel() // 3, _ptr(add), _ptr(rgb))
    return rgb
