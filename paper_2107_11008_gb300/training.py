"""Denoiser training pairs rendered by the tracer itself, and the training / evaluation driver.

A pair is one scene rendered twice with disjoint Philox sample ranges: a low-sample render (the
network input, with the albedo / normal / depth / mask ground-truth buffers of Sec. III-D) and a
high-sample render (the target).  With ``source="direct"`` the network sees and predicts only the
camera-path estimate, and the low-sample render's light-traced caustic buffer is added back to
its output: the AOVs describe the first-hit image, not where caustics focus, and an unbiased
caustic estimate from many cheap light paths beats a learned guess of their shape.  All
rendering, packing, training and inference run in the library's CUDA kernels; this module only
orders the calls and picks crops and batches.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import torch

from . import denoiser as D
from . import renderer as R
from .scenes import Scene, guide_sphere


@dataclass
class RenderSpec:
    spp: int
    lights_per_pixel: float
    max_depth: int = 8
    n_bins: int = 1
    guided: bool = True  # light paths aimed into the sphere around the glass (scenes.guide_sphere)


CHUNK = 256  # samples (and light paths) per pixel accumulated in one float32 pass


def render(ctx: R.Context, gs: R.GpuScene, frame: R.Frame, spec: RenderSpec, seed: int, sample_offset: int = 0,
           path_offset: int = 0, scene_index: int = 0, guide=None, chunked: bool = True):
    """Camera paths + light paths + resolve into ``frame`` (accumulators cleared first); ``guide``
    is the scene's guide sphere, used when ``spec.guided``.  Budgets above CHUNK per pixel run as
    passes of consecutive sample / path ranges whose resolved estimates are averaged in float64
    (a bright caustic pixel collecting millions of splats in one float32 sum would lose the small
    ones), so the result is the same estimator as one pass.  ``chunked=False`` always runs one pass
    (timing a frame as a user would render it)."""
    w, h = frame.width, frame.height
    n_light = int(round(spec.lights_per_pixel * w * h))
    g = guide if spec.guided else None

    def one(spp, soff, nl, poff):
        frame.zero_accumulators()
        if spp > 0:
            R.trace_camera(ctx, gs, frame, spp, spec.max_depth, spec.n_bins, seed, soff, scene_index)
        if nl > 0:
            R.trace_lights(ctx, gs, frame, nl, spec.max_depth, spec.n_bins, seed, poff, scene_index, guide=g)
        R.resolve(ctx, gs, frame, max(spp, 1), max(nl, 1))

    if not chunked or (spec.spp <= CHUNK and spec.lights_per_pixel <= CHUNK):
        one(spec.spp, sample_offset, n_light, path_offset)
        return
    direct = torch.zeros((h, w, 3), dtype=torch.float64, device=frame["rgb"].device)
    caustic = torch.zeros_like(direct)
    done = 0
    while done < spec.spp:
        k = min(CHUNK, spec.spp - done)
        one(k, sample_offset + done, 0, 0)
        direct += frame["direct"][..., :3].double() * k
        done += k
    done, step = 0, CHUNK * w * h
    while done < n_light:
        k = min(step, n_light - done)
        one(0, 0, k, path_offset + done)
        caustic += frame["caustic"][..., :3].double() * k
        done += k
    if spec.spp > 0:
        direct /= spec.spp
    if n_light > 0:
        caustic /= n_light
    frame["direct"][..., :3] = direct.float()
    frame["caustic"][..., :3] = caustic.float()
    frame["rgb"][..., :3] = (direct + caustic).float()


@dataclass
class Pairs:
    x: torch.Tensor          # [n, H, W, 11] network input of the low-sample renders
    target: torch.Tensor     # [n, H, W, 3] log1p of the high-sample renders' selected estimate
    rgb_lo: torch.Tensor     # [n, H, W, 4] low-sample linear RGB (full image)
    rgb_hi: torch.Tensor     # [n, H, W, 4] high-sample linear RGB (full image)
    caustic_lo: torch.Tensor  # [n, H, W, 4] low-sample caustic buffer (added back for source "direct")
    source: str = "rgb"

    def add(self):
        return self.caustic_lo if self.source == "direct" else None



def make_pairs(ctx: R.Context, scenes: list[Scene], lo: RenderSpec, hi: RenderSpec, seed: int = 0,
               source: str = "rgb") -> Pairs:
    h, w = scenes[0].camera.height, scenes[0].camera.width
    n = len(scenes)
    dev = torch.device("cuda", ctx.device)
    x = torch.empty((n, h, w, D.IN_CH), dtype=torch.float32, device=dev)
    t = torch.empty((n, h, w, D.OUT_CH), dtype=torch.float32, device=dev)
    rgb_lo = torch.empty((n, h, w, 4), dtype=torch.float32, device=dev)
    rgb_hi = torch.empty((n, h, w, 4), dtype=torch.float32, device=dev)
    caustic_lo = torch.empty((n, h, w, 4), dtype=torch.float32, device=dev)
    f = R.Frame(w, h, device=dev)
    n_light_lo = int(round(lo.lights_per_pixel * w * h))
    for i, sc in enumerate(scenes):
        if (sc.camera.width, sc.camera.height) != (w, h):
            raise ValueError("all scenes of a pair set share one resolution")
        gs = R.GpuScene(ctx, sc)
        guide = guide_sphere(sc)
        render(ctx, gs, f, lo, seed, 0, 0, scene_index=i, guide=guide)
        D.pack_frame(ctx, f, x, i, source)
        rgb_lo[i].copy_(f["rgb"])
        caustic_lo[i].copy_(f["caustic"])
        # the target uses the samples after the input's: independent noise, same estimator
        render(ctx, gs, f, hi, seed, lo.spp, n_light_lo, scene_index=i, guide=guide)
        D.pack_target(ctx, f, t, i, source)
        rgb_hi[i].copy_(f["rgb"])
        ctx.stream.synchronize()
        del gs
    ctx.sync_status()
    return Pairs(x, t, rgb_lo, rgb_hi, caustic_lo, source)


def train(net: D.UNet, pairs: Pairs, steps: int, batch: int, lr: float, crop: int | None = None, seed: int = 0,
          lr_final: float | None = None, log_every: int = 0):
    """Adam on random batches (and random crops of size ``crop``) of the pairs; cosine learning-rate
    decay to ``lr_final``.  Returns the logged losses."""
    g = torch.Generator(device="cpu").manual_seed(seed)
    n, h, w, _ = pairs.x.shape
    ch = cw = crop or 0
    if crop is None:
        ch, cw = h, w
    if batch > net.max_batch or ch != net.height or cw != net.width:
        raise ValueError("batch and crop must match the network's workspace")
    xb = torch.empty((batch, ch, cw, D.IN_CH), dtype=torch.float32, device=pairs.x.device)
    tb = torch.empty((batch, ch, cw, D.OUT_CH), dtype=torch.float32, device=pairs.x.device)
    loss = torch.empty(1, dtype=torch.float32, device=pairs.x.device)
    lf = lr if lr_final is None else lr_final
    logged = []
    for s in range(steps):
        idx = torch.randint(0, n, (batch,), generator=g)
        oy = torch.randint(0, h - ch + 1, (batch,), generator=g)
        ox = torch.randint(0, w - cw + 1, (batch,), generator=g)
        for b in range(batch):
            i, y0, x0 = int(idx[b]), int(oy[b]), int(ox[b])
            xb[b].copy_(pairs.x[i, y0:y0 + ch, x0:x0 + cw])
            tb[b].copy_(pairs.target[i, y0:y0 + ch, x0:x0 + cw])
        rate = lf + 0.5 * (lr - lf) * (1.0 + np.cos(np.pi * s / max(steps - 1, 1)))
        net.train_step(xb, tb, rate, loss)
        if log_every and (s % log_every == 0 or s == steps - 1):
            logged.append((s, float(loss.item())))
    return logged


def denoise(net: D.UNet, x: torch.Tensor, add: torch.Tensor | None = None, batch: int | None = None) -> torch.Tensor:
    """Linear RGB [n, H, W, 4] of the network applied to inputs x [n, H, W, 11], plus ``add``
    [n, H, W, 4] (the caustic buffer when the network denoises the camera estimate alone)."""
    n = x.shape[0]
    b = batch or net.max_batch
    out = []
    for s in range(0, n, b):
        y = net.forward(x[s:s + b].contiguous())
        out.append(D.output_rgb(net.ctx, y, None if add is None else add[s:s + b].contiguous()))
    return torch.cat(out)


def mse(a: torch.Tensor, b: torch.Tensor) -> float:
    """Mean squared error over the RGB channels (float64 on the device)."""
    return float(((a[..., :3].double() - b[..., :3].double()) ** 2).mean())


# ----------------------------------------------------------------------------------------------
# Caustic segmentation (the paper's Sec. IV-B experiment, synthetic -> synthetic): a U-Net trained
# with the segmentation loss on rendered images labelled by the caustic mask ground truth
# ----------------------------------------------------------------------------------------------

@dataclass
class SegData:
    x: torch.Tensor       # [n, H, W, 11] network input: log1p of the rendered RGB, the rest zero
    target: torch.Tensor  # [n, H, W, 3] label in channel 0: the non-local caustic mask (Sec. III-D)


def seg_data(ctx: R.Context, scenes: list[Scene], spec: RenderSpec, seed: int = 0) -> SegData:
    """Renders each scene (camera paths + guided light paths + resolve) and keeps its RGB image as
    the input (the other ten input channels zero: the network sees the image only, as a
    segmentation network deployed on photographs would) and its caustic mask as the label."""
    h, w = scenes[0].camera.height, scenes[0].camera.width
    n = len(scenes)
    dev = torch.device("cuda", ctx.device)
    x = torch.empty((n, h, w, D.IN_CH), dtype=torch.float32, device=dev)
    t = torch.zeros((n, h, w, D.OUT_CH), dtype=torch.float32, device=dev)
    f = R.Frame(w, h, device=dev)
    for i, sc in enumerate(scenes):
        gs = R.GpuScene(ctx, sc)
        render(ctx, gs, f, spec, seed, scene_index=i, guide=guide_sphere(sc))
        D.pack_frame(ctx, f, x, i, "rgb")
        x[i, ..., 3:] = 0.0
        t[i, ..., 0] = f["caustic_mask"].float()
        ctx.stream.synchronize()
        del gs
    ctx.sync_status()
    return SegData(x, t)


def predict_masks(net: D.UNet, x: torch.Tensor) -> torch.Tensor:
    """Boolean [n, H, W]: logit of output channel 0 above zero (probability above one half)."""
    out = []
    for s in range(0, x.shape[0], net.max_batch):
        out.append(net.forward(x[s:s + net.max_batch].contiguous())[..., 0] > 0.0)
    return torch.cat(out)


def iou(pred: torch.Tensor, label: torch.Tensor) -> float:
    """Intersection over union of two boolean masks over all their pixels."""
    inter = (pred & label).sum().item()
    union = (pred | label).sum().item()
    return inter / union if union else 1.0


def brightness_baseline(train: SegData, tests: list[SegData]) -> tuple[float, list[float]]:
    """The method without a network: a pixel is a caustic when its log1p luminance exceeds a
    threshold, the one (of 64 quantiles) with the best IoU on the training images."""
    def lum(x):
        return 0.2126 * x[..., 0] + 0.7152 * x[..., 1] + 0.0722 * x[..., 2]

    lt = lum(train.x)
    lab = train.target[..., 0] > 0.5
    best, best_thr = -1.0, 0.0
    for q in torch.linspace(0.5, 0.999, 64):
        thr = float(torch.quantile(lt.flatten()[::7].float(), float(q)))
        v = iou(lt > thr, lab)
        if v > best:
            best, best_thr = v, thr
    return best_thr, [iou(lum(d.x) > best_thr, d.target[..., 0] > 0.5) for d in tests]
