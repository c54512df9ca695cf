#!/usr/bin/env python
"""Benchmark of the spectral glass path/light tracer on one GB300 per rank.

Workload (one "step" = one frame of the whole hot path): the 512x512 glass scene -- four
procedural transparent meshes of ~20k triangles (sphere, hollow cylinder glass, torus,
superellipsoid) with random pose from seed 0 over a checkered floor and back wall, a 1x1 m
rect light, Cauchy glass A=1.5 B=0.004 um^2 over 8 wavelength bins, max depth 12.  Per step:
BVH build from device-resident triangles, 256 camera samples per pixel (67.1M camera paths),
4M light paths splatted as caustics, and the resolve pass with every ground-truth buffer.

Metric: Mpaths/s (camera + light paths per second, all ranks) with frames/s beside it.
Multi-GPU: each rank renders its own frame of the same scene with a disjoint sample range
(no data-path collective; weak scaling).  ``--impl reference`` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "Mpaths/s and frames/s at 512^2 glass scene"
UNIT = "Mpaths/s"
WORKLOAD = ("glass_scene_512: 4 glass meshes x ~20k tris (sphere, hollow cylinder, torus, superellipsoid; seed 0) "
            "over checkered floor+wall, 1x1 m rect light, Cauchy A=1.5 B=0.004, 8 bins, depth 12, "
            "256 spp + 4M light paths, LBVH build + resolve per frame")
# FP32 work per traversal step: a 4-wide node visit tests four child boxes, each slab test being
# 3 axes x 2 planes x (sub + mul), and loads 7 float4 (boxes + child references); a watertight
# triangle test is ~43 flops on 48 bytes.
FLOPS_PER_NODE = 48
FLOPS_PER_TRI = 43
BYTES_PER_NODE = 112
BYTES_PER_TRI = 48


def launches_per_step_base(n_tris):
    """Our kernels per step besides the camera estimator: the BVH build (bounds init, gather,
    morton, 8 x (hist, scan, scatter), reorder, PLOC init, 4 launches per grid-wide round, the
    single-block finish, depth, 4-wide collapse) + lights + resolve + outline/occlusion pass.  The
    grid-wide rounds follow the library's rule: enough to bring ~0.84^k * n below 1024 clusters."""
    rounds = 0 if n_tris <= 1024 else math.ceil(math.log(n_tris / 1024) / math.log(1 / 0.84))
    return 3 + 24 + 1 + (2 + 4 * rounds) + 2 + 3


def camera_launches(engine, width, height, spp, depth):
    """Kernel launches of one sc_trace_camera call: one persistent kernel, or per wave of whole
    pixels (at most 2^25 paths) generate + depth x (extend, dielectric, diffuse, shadow, rotate, and
    for waves of at least 2^18 paths three compactions of 3 launches each that emit the ordered
    queues) + reduce."""
    if engine == "persistent":
        return 1
    tiles = ((width + 7) // 8) * ((height + 3) // 4)
    one_tile = 32 * spp
    max_paths = max(one_tile, min(tiles * one_tile, 1 << 25))
    wave_tiles = max(1, max_paths // one_tile)
    waves = -(-tiles // wave_tiles)
    per_bounce = 14 if min(wave_tiles, tiles) * one_tile >= 1 << 18 else 5
    return waves * (2 + per_bounce * depth)
# DRAM bytes (dram__bytes_read.sum + dram__bytes_write.sum) of one full-size camera launch, from
# one ncu capture of this kernel version:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum --clock-control none \
#       -k regex:k_trace_camera -s 4 -c 1 python bench.py --steps 1 --warmup 3 --no-cpu-baseline
# (the scene stays in L2, so DRAM sees little more than the accumulators and first touches)
# wavefront: all kernels of one 256-spp camera phase, scaled by the path count (x16) from one ncu capture
# of the 16-spp frame (the traffic is path state and queues, proportional to the paths):
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
#       -k regex:k_wf_ -s 680 -c 170 python bench.py --steps 1 --warmup 3 --spp 16 --no-cpu-baseline --no-sub
CAMERA_DRAM_BYTES = {"persistent": 24.5e6, "wavefront": 16 * 8.5297e9}


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--spp", type=int, default=256)
    ap.add_argument("--light-paths", type=int, default=1 << 22)
    ap.add_argument("--res", type=int, default=512)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--camera-engine", default="wavefront", choices=["wavefront", "persistent"],
                    help="sc_trace_camera engine: event-regrouped wavefront kernels or the persistent state machine")
    ap.add_argument("--no-sub", action="store_true",
                    help="skip the sub-results (cfg1 frame, batch64, U-Net training) of the default line")
    ap.add_argument("--cpu-seconds", type=float, default=12.0)
    ap.add_argument("--den-ratio", type=int, default=16, help="denoise workload: light paths per camera sample")
    ap.add_argument("--den-steps", type=int, default=48000, help="denoise workload: training steps")
    ap.add_argument("--seg-steps", type=int, default=4000, help="caustic_seg workload: training steps")
    ap.add_argument("--workload", default="glass512",
                    choices=["glass512", "batch64", "unet_train", "denoise", "denoise_dense", "caustic_seg"],
                    help="batch64: 64 randomised scenes (1k-200k tris, 128^2..1024^2, 64 spp) in one graph-captured "
                         "persistent launch vs 64 sequential launches; unet_train: U-Net training steps on batches "
                         "of 16 x 256^2 render pairs; denoise: 4-spp render + U-Net vs the plain tracer at matched MSE")
    return ap.parse_args()


def measure_batch(steps, warmup, local, world):
    """64 randomised dataset scenes traced in one persistent CUDA-graph launch vs one launch per scene.
    Returns (batch ms per launch, sequential ms per pass, info dict)."""
    import torch

    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S

    dev = torch.device("cuda", local)
    n, spp, depth = 64, 64, 12
    t0 = time.perf_counter()
    scs = [S.random_scene(i) for i in range(n)]
    gen_s = time.perf_counter() - t0
    ctx = R.Context(local)
    arrays = [R.SceneArrays(s, dev) for s in scs]
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    gss = [R.GpuScene(ctx, a) for a in arrays]
    torch.cuda.synchronize(dev)
    build_s = time.perf_counter() - t0
    frames = [R.Frame(s.camera.width, s.camera.height, device=dev, fields=("accum_camera",)) for s in scs]
    batch = R.Batch(ctx, gss, frames, spp, depth, seed=3)
    stream = torch.cuda.current_stream(dev)
    for _ in range(warmup):
        batch.launch()
    ctx.sync_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(local)
    ev[0].record(stream)
    for _ in range(steps):
        batch.launch()
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    batch_ms = ev[0].elapsed_time(ev[1]) / steps
    # the same work as one plain launch per scene
    ev[0].record(stream)
    for _ in range(steps):
        for i, (g, f) in enumerate(zip(gss, frames)):
            R.trace_camera(ctx, g, f, spp, depth, seed=3, scene_index=i)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    seq_ms = ev[0].elapsed_time(ev[1]) / steps
    ctx.sync_status()
    paths = sum(s.camera.width * s.camera.height for s in scs) * spp
    info = {"triangles": sum(s.n_tris for s in scs), "camera_paths": paths, "scene_generation_s": gen_s,
            "lbvh_build_s": build_s, "clocks": clocks}
    batch.close()
    for g in gss:
        g.free()
    ctx.close()
    return batch_ms, seq_ms, info


BATCH_WORKLOAD = ("batch64: scenes.random_scene(0..63): 1-6 glass objects, 1k-200k tris, resolution from "
                  "{128,256,512,1024}^2, IOR U[1.33,1.9], 64 spp, depth 12")


def run_batch(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    batch_ms, seq_ms, info = measure_batch(args.steps, args.warmup, local, world)
    paths = info["camera_paths"]
    value = world * paths / (batch_ms * 1e-3) / 1e6
    if rank == 0:
        line = {"metric": "Mpaths/s of 64 randomised scenes in one graph-captured launch", "value": value,
                "unit": UNIT, "n_gpus": world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": batch_ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
                "config": {"workload": BATCH_WORKLOAD, "triangles": info["triangles"], "camera_paths": paths},
                "sequential_launches": {"ms_per_step": seq_ms, "value": world * paths / (seq_ms * 1e-3) / 1e6},
                "batch_over_sequential": seq_ms / batch_ms, "scene_generation_s": info["scene_generation_s"],
                "lbvh_build_s": info["lbvh_build_s"], "gpu_launches": args.steps, "clocks": info["clocks"]}
        print(json.dumps(line), flush=True)


# ---------------------------------------------------------------------------------------------
# U-Net denoiser workloads
# ---------------------------------------------------------------------------------------------
UNET_CHANS = (32, 48, 64, 128)
# our kernels per training step (counted from an ncu launch list of one step): forward 23 (input
# pack, 9 encoder conv launches -- the 128 -> 128 conv runs as two halves --, 3 pools, 3 x
# (transposed conv, 2 convs), output layer); loss 3; backward 41 (output layer 3, decoder 3 x 6,
# encoder 19 -- 8 weight gradients, 8 data-gradient convs, 3 pool routings --, one split-K
# reduce); Adam 1
UNET_TRAIN_LAUNCHES = 23 + 3 + 41 + 1
UNET_FWD_LAUNCHES = 23
# DRAM bytes of one training step (all its kernels, dram__bytes_read.sum + dram__bytes_write.sum
# summed over launches 1-68 = the first step; launch 0 is the parameter refresh), from one ncu
# capture of these kernel versions:
#   ncu --metrics dram__bytes_read.sum,dram__bytes_write.sum,gpu__time_duration.sum --clock-control none \
#       -k regex:"k_(gemm|conv_tma|wgrad_mn|ssim|pool|adam|wgrad_reduce|loss_final|pack_input|out_)" -c 70 \
#       --csv python bench.py --workload unet_train --steps 1 --warmup 3 --no-cpu-baseline
UNET_STEP_DRAM_BYTES = 3.95e9


def unet_macs(h, w, in_ch=11, out_ch=3):
    """Multiply-adds of one forward pass over an h x w image (algorithmic: unpadded channels)."""
    c = UNET_CHANS
    px = [(h >> l) * (w >> l) for l in range(4)]
    m, cin = 0, in_ch
    for l in range(4):
        m += px[l] * 9 * cin * c[l] + px[l] * 9 * c[l] * c[l]
        cin = c[l]
    for l in range(3):
        m += px[l + 1] * c[l + 1] * 4 * c[l] + px[l] * 9 * 2 * c[l] * c[l] + px[l] * 9 * c[l] * c[l]
    return m + px[0] * c[0] * out_ch


def unet_train_macs(h, w, in_ch=11):
    """Forward + data gradients (all layers but the first) + weight gradients."""
    first = h * w * 9 * in_ch * UNET_CHANS[0]
    return 3 * unet_macs(h, w, in_ch) - first


def unet_cpu_baseline(seconds, h=64, w=64):
    """The FP64 NumPy oracle, as it stands: forward + loss + backward of one 64 x 64 image, repeated
    for about `seconds`; reported as 256^2 images/s by pixel count."""
    import numpy as np

    from oracle import unet as U

    rng = np.random.default_rng(0)
    p = U.init_params(seed=0)
    x, t = rng.random((1, h, w, 11)), rng.random((1, h, w, 3))
    n, t0 = 0, time.perf_counter()
    while True:
        y, cache = U.forward(p, x, UNET_CHANS)
        _, gy = U.loss(y, t)
        U.backward(p, cache, gy, UNET_CHANS)
        n += 1
        el = time.perf_counter() - t0
        if el > seconds or n >= 50:
            break
    scale = (h * w) / (256 * 256)
    return {"value": n / el * scale, "unit": "images/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"{n} forward+loss+backward passes of one {h}x{w} image in FP64 NumPy ({el:.1f} s; numpy may use "
                      f"up to {os.cpu_count()} BLAS threads), scaled to 256^2 images by pixel count"}


def measure_unet_train(steps, warmup, local, world, e2e=True):
    """Training steps of the BF16 U-Net on batches of 16 render pairs at 256^2 (config-1-type scenes:
    4 spp + AOV input, 256 spp target; the step's work does not depend on the pixel values).
    Returns a dict of timings (ms per step, forward ms, e2e s per step) and sizes."""
    import torch

    from paper_2107_11008_gb300 import denoiser as D
    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S
    from paper_2107_11008_gb300 import training as T

    rank = int(os.environ.get("RANK", "0"))
    dev = torch.device("cuda", local)
    n, hw = 16, 256
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream)
    pairs = T.make_pairs(ctx, [S.denoise_scene(100 * rank + i, hw, hw) for i in range(n)], T.RenderSpec(4, 4),
                         T.RenderSpec(256, 256), seed=rank)
    net = D.UNet(ctx, n, hw, hw)
    net.set_params(D.he_init(0).to(dev))
    x, t = pairs.x.contiguous(), pairs.target.contiguous()
    loss = torch.empty(1, dtype=torch.float32, device=dev)
    lr = 1e-4
    for _ in range(max(3, warmup)):
        net.train_step(x, t, lr, loss)
    torch.cuda.synchronize(dev)
    ctx.sync_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(local)
    ev[0].record(stream)
    for _ in range(steps):
        net.train_step(x, t, lr, loss)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ctx.sync_status()
    ms = ev[0].elapsed_time(ev[1]) / steps
    # forward alone (inference throughput of the same batch)
    ev[0].record(stream)
    for _ in range(steps):
        net.forward(x)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    fwd_ms = ev[0].elapsed_time(ev[1]) / steps
    out = {"ms": ms, "forward_ms": fwd_ms, "batch": n, "hw": hw, "clocks": clocks}
    if e2e:
        # end to end: the batch from pinned host memory each step, the loss read back
        xh, th = x.cpu().pin_memory(), t.cpu().pin_memory()
        lh = torch.empty(1, dtype=torch.float32, pin_memory=True)
        torch.cuda.synchronize(dev)
        t0 = time.perf_counter()
        for _ in range(steps):
            x.copy_(xh, non_blocking=True)
            t.copy_(th, non_blocking=True)
            net.train_step(x, t, lr, loss)
            lh.copy_(loss, non_blocking=True)
            torch.cuda.synchronize(dev)
        out["e2e_s"] = (time.perf_counter() - t0) / steps
        out["h2d"] = (xh.numel() + th.numel()) * 4
    net.close()
    ctx.close()
    return out


def unet_roofline(ms, n, hw):
    flops = 2.0 * unet_train_macs(hw, hw) * n
    peak = peaks().get("bf16_tflops_sustained", 1700.0)
    achieved = flops / (ms * 1e-3) / 1e12
    return {"kernel": "all U-Net GEMMs of the step (tcgen05 BF16, FP32 accumulate)", "bound": "tensor",
            "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": UNET_STEP_DRAM_BYTES, "traffic_unit": "bytes per step (ncu)", "flops_per_step": flops,
            "peak_source": "MEASURED_PEAKS bf16_tflops_sustained (of measured)"}


def run_unet_train(args):
    import torch

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    r = measure_unet_train(args.steps, args.warmup, local, world)
    n, hw, ms = r["batch"], r["hw"], r["ms"]
    value = world * n / (ms * 1e-3)
    if rank == 0:
        cb = None if args.no_cpu_baseline or world > 1 else unet_cpu_baseline(min(args.cpu_seconds, 15.0))
        line = {"metric": "U-Net training images/s (16 x 256^2 per step)", "value": value, "unit": "images/s",
                "n_gpus": world, "steps": args.steps, "warmup": max(3, args.warmup), "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "bf16",
                "data": "synthetic (render pairs of scenes.denoise_scene)",
                "config": {"workload": UNET_WORKLOAD, "l2": "working set ~1.5 GB > L2 (no flush)",
                           "parallelism": f"replicas x{world}"},
                "forward_ms": r["forward_ms"], "forward_images_s": world * n / (r["forward_ms"] * 1e-3),
                "roofline": unet_roofline(ms, n, hw),
                "e2e": {"value": world * n / r["e2e_s"], "unit": "images/s", "h2d_bytes_per_step": r["h2d"],
                        "d2h_bytes_per_step": 4},
                "gpu_launches": UNET_TRAIN_LAUNCHES * args.steps, "clocks": r["clocks"], "cpu_baseline": cb}
        print(json.dumps(line), flush=True)


UNET_WORKLOAD = ("unet_train: U-Net 11->3, widths 32/48/64/128 (585,363 params), batch 16 of 256^2, loss 0.16 L1 "
                 "+ 0.84 (1 - SSIM 11x11), Adam")


def run_denoise(args):
    """Denoised frames vs the plain tracer at matched MSE on held-out config-1-type scenes at 256^2.

    Both pipelines spend the same ratio of light paths to camera samples (``--den-ratio``, 16),
    light paths aimed into the sphere around the glass (guided emission): the denoised frame is
    4 camera spp + 4 x ratio light paths per pixel, the U-Net removing the camera estimate's noise
    (trained --den-steps (48000) steps on 16 random 128^2 crops of 256 pairs: that estimate at 4 -> 1024 spp;
    one network with L1 + SSIM and one with the squared error in linear radiance, two validation
    scenes pick one) and the light-traced caustic buffer added back; the plain frame is N spp + N x
    ratio light paths.
    MSEs are against a reference of two independent halves (2048 spp + 8192 light paths / px
    each), with the reference's own variance, MSE(half_a, half_b) / 4, subtracted."""
    import numpy as np
    import torch

    from paper_2107_11008_gb300 import denoiser as D
    from paper_2107_11008_gb300 import native as N
    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S
    from paper_2107_11008_gb300 import training as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hw, n_train, n_test, ratio = 256, 256, 8, args.den_ratio
    lo = T.RenderSpec(4, 4 * ratio)
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream)
    t0 = time.perf_counter()
    train = T.make_pairs(ctx, [S.denoise_scene(i, hw, hw) for i in range(n_train)], lo, T.RenderSpec(1024, 0),
                         seed=1, source="direct")
    val = T.make_pairs(ctx, [S.denoise_scene(5_000 + i, hw, hw) for i in range(2)], lo, T.RenderSpec(1024, 0),
                       seed=4, source="direct")
    test_scenes = [S.denoise_scene(10_000 + i, hw, hw) for i in range(n_test)]
    test = T.make_pairs(ctx, test_scenes, lo, T.RenderSpec(0, 0), seed=2, source="direct")
    gss = [R.GpuScene(ctx, s) for s in test_scenes]
    guides = [S.guide_sphere(s) for s in test_scenes]
    f = R.Frame(hw, hw, device=dev)
    half = T.RenderSpec(2048, 8192)
    ref_a = torch.empty_like(test.rgb_lo)
    ref_b = torch.empty_like(test.rgb_lo)
    for i, g in enumerate(gss):
        for k, dst in enumerate((ref_a, ref_b)):
            T.render(ctx, g, f, half, seed=3, sample_offset=(1 << 24) + k * half.spp,
                     path_offset=(1 << 42) + k * 8192 * hw * hw, scene_index=i, guide=guides[i])
            dst[i].copy_(f["rgb"])
    ref = 0.5 * (ref_a + ref_b)
    var_ref = T.mse(ref_a, ref_b) / 4.0
    gen_s = time.perf_counter() - t0
    trainer = D.UNet(ctx, 16, 128, 128)  # 128^2 random crops of the 256^2 pairs, 16 per step
    t0 = time.perf_counter()
    # one network per loss; validation scenes (not test scenes) pick the one used
    candidates = {}
    for name, loss_kind, lr, init in (("l1_ssim", N.SC_UNET_LOSS_L1_SSIM, 1.5e-3, 0),
                                      ("l2_linear", N.SC_UNET_LOSS_L2_LINEAR, 1e-3, 1)):
        trainer.set_params(D.he_init(init).to(dev))
        trainer.set_loss(loss_kind)
        T.train(trainer, train, steps=args.den_steps, batch=16, crop=128, lr=lr, lr_final=5e-5, seed=init)
        candidates[name] = trainer.get_params()
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    ctx.sync_status()
    net = D.UNet(ctx, 8, hw, hw)
    val_mse, test_mse = {}, {}
    for name, prm in candidates.items():
        net.set_params(prm)
        val_mse[name] = T.mse(T.denoise(net, val.x, None), torch.expm1(val.target))
        test_mse[name] = T.mse(T.denoise(net, test.x, test.add()), ref) - var_ref
    chosen = min(val_mse, key=val_mse.get)
    net.set_params(candidates[chosen])
    den = T.denoise(net, test.x, test.add())
    m_den = T.mse(den, ref) - var_ref
    m_in = T.mse(test.rgb_lo, ref) - var_ref
    # plain tracer at increasing budgets, same light/camera ratio, samples disjoint from the reference's
    sweep = {}
    for spp in (4, 8, 16, 32, 64, 128):
        out = torch.empty_like(ref)
        for i, g in enumerate(gss):
            T.render(ctx, g, f, T.RenderSpec(spp, spp * ratio), seed=7, scene_index=i, guide=guides[i])
            out[i].copy_(f["rgb"])
        sweep[spp] = T.mse(out, ref) - var_ref
    ctx.sync_status()
    budgets = sorted(sweep)
    above = [s for s in budgets if sweep[s] > m_den]
    below = [s for s in budgets if sweep[s] <= m_den]
    if below and above:  # log-log interpolation between the bracketing budgets
        s_lo, s_hi = max(above), min(below)
        a, b = np.log(sweep[s_lo]), np.log(sweep[s_hi])
        spp_match = float(np.exp(np.log(s_lo) + (np.log(m_den) - a) / (b - a) * (np.log(s_hi) - np.log(s_lo))))
    elif below:
        spp_match = float(budgets[0])
    else:  # beyond the sweep: MSE ~ 1/spp from the largest budget
        spp_match = budgets[-1] * sweep[budgets[-1]] / m_den
    # timed frames on test scene 0: (a) 4 spp + caustics + denoise, (b) plain at the matched budget
    g0 = gss[0]
    x1 = torch.empty((1, hw, hw, 11), dtype=torch.float32, device=dev)
    y1 = torch.empty((1, hw, hw, 3), dtype=torch.float32, device=dev)
    rgb1 = torch.empty((1, hw, hw, 4), dtype=torch.float32, device=dev)
    net1 = D.UNet(ctx, 1, hw, hw)
    net1.set_params(net.get_params())

    def denoised_frame():
        T.render(ctx, g0, f, lo, seed=11, guide=guides[0], chunked=False)
        D.pack_frame(ctx, f, x1, 0, source="direct")
        net1.forward(x1, y1)
        D.output_rgb(ctx, y1, f["caustic"], out=rgb1)

    spp_int = max(1, int(np.ceil(spp_match)))
    plain_spec = T.RenderSpec(spp_int, spp_int * ratio)

    def plain_frame():
        T.render(ctx, g0, f, plain_spec, seed=11, guide=guides[0], chunked=False)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for fn in (denoised_frame, plain_frame):
        for _ in range(max(3, args.warmup)):
            fn()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    ev[0].record(stream)
    for _ in range(args.steps):
        denoised_frame()
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    den_ms = ev[0].elapsed_time(ev[1]) / args.steps
    ev[0].record(stream)
    for _ in range(args.steps):
        plain_frame()
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    plain_ms = ev[0].elapsed_time(ev[1]) / args.steps
    # the network alone
    ev[0].record(stream)
    for _ in range(args.steps):
        net1.forward(x1, y1)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    net_ms = ev[0].elapsed_time(ev[1]) / args.steps
    clocks = sampler.stop()
    ctx.sync_status()
    # end to end: the denoised RGB read back to pinned host memory every frame
    out_h = torch.empty((hw, hw, 4), dtype=torch.float32, pin_memory=True)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        denoised_frame()
        out_h.copy_(rgb1[0], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_ms = (time.perf_counter() - t0) * 1e3 / args.steps
    if rank == 0:
        line = {"metric": "denoised fps at the plain tracer's matched MSE (256^2 ball-on-plane scenes)",
                "value": world * 1e3 / den_ms, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": den_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic (scenes.denoise_scene)",
                "config": {"workload": "denoise: 256^2 config-1-type scenes; U-Net on the camera estimate trained "
                                       f"{args.den_steps} steps x 16 crops of 128^2 from 256 pairs (4 -> 1024 spp; L1 + "
                                       "SSIM or linear squared error, picked on 2 validation scenes), guided "
                                       "light-traced caustics added back; 8 held-out scenes; reference 2 x (2048 spp "
                                       "+ 8192 guided light paths/px)",
                           "input": f"{lo.spp} camera spp + {lo.lights_per_pixel} light paths/px",
                           "light_paths_per_camera_sample": ratio},
                "mse": {"denoised": m_den, "input": m_in, "reference_variance": var_ref, "plain_sweep": sweep,
                        "by_loss": {"validation": val_mse, "test": test_mse, "chosen": chosen}},
                "matched_spp": spp_match, "plain_frame": {"spp": spp_int, "light_paths_per_px": spp_int * ratio,
                                                          "ms": plain_ms, "fps": world * 1e3 / plain_ms},
                "fps_ratio_denoised_over_plain": plain_ms / den_ms, "unet_forward_ms": net_ms,
                "setup_s": {"pairs_and_reference": gen_s, "training": train_s},
                "e2e": {"value": world * 1e3 / e2e_ms, "unit": "frames/s", "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": hw * hw * 16},
                "gpu_launches": args.steps * ((3 + 1 + UNET_FWD_LAUNCHES + 1) + 3 + UNET_FWD_LAUNCHES),
                "clocks": clocks, "cpu_baseline": None}
        print(json.dumps(line), flush=True)


def run_denoise_dense(args):
    """The dense comparison: 1024^2 frames of 16 overlapping glass objects (~1M triangles), 16
    wavelength bins, 32M guided light paths per frame.  Denoised frame = 8 camera spp + 32M light
    paths, a U-Net on the camera estimate (trained on 128^2 crops of 1024^2 renders of other dense
    scenes, 8 -> 512 spp, so that objects have the test frames' size in pixels) and the light-traced
    caustic buffer added back.  Two networks are trained, one with L1 + SSIM in the log domain and
    one with the squared error in linear radiance (the loss the MSE comparison rewards); a
    validation scene, not a test scene, picks the one used.  Plain frames = N spp + the same light
    paths per camera sample.  MSEs against a two-half reference (2048 spp + 4x that in light paths
    per pixel each) with the reference's own variance subtracted; the plain tracer's matched spp
    interpolated from a sweep up to 1024 spp (its MSE at 1024 spp measured directly)."""
    import numpy as np
    import torch

    from paper_2107_11008_gb300 import denoiser as D
    from paper_2107_11008_gb300 import native as N
    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S
    from paper_2107_11008_gb300 import training as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hw, n_train, n_test, nb, depth = 1024, 24, 2, 16, 12
    lpp = 32e6 / (hw * hw)        # light paths per pixel of the denoised frame (32M per frame)
    ratio = lpp / 8.0             # light paths per camera sample, kept for every plain budget
    lo = T.RenderSpec(8, lpp, max_depth=depth, n_bins=nb)
    hi = T.RenderSpec(512, 0, max_depth=depth, n_bins=nb)
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream)
    t0 = time.perf_counter()
    train = T.make_pairs(ctx, [S.dense_scene(100 + i, hw, hw) for i in range(n_train)], lo, hi, seed=1,
                         source="direct")
    val = T.make_pairs(ctx, [S.dense_scene(5_000, hw, hw)], lo, hi, seed=4, source="direct")
    test_scenes = [S.dense_scene(10_000 + i, hw, hw) for i in range(n_test)]
    gss = [R.GpuScene(ctx, sc) for sc in test_scenes]
    guides = [S.guide_sphere(sc) for sc in test_scenes]
    f = R.Frame(hw, hw, device=dev)
    test_x = torch.empty((n_test, hw, hw, D.IN_CH), dtype=torch.float32, device=dev)
    test_caustic = torch.empty((n_test, hw, hw, 4), dtype=torch.float32, device=dev)
    test_rgb = torch.empty((n_test, hw, hw, 4), dtype=torch.float32, device=dev)
    for i, g in enumerate(gss):
        T.render(ctx, g, f, lo, seed=2, scene_index=i, guide=guides[i])
        D.pack_frame(ctx, f, test_x, i, "direct")
        test_caustic[i].copy_(f["caustic"])
        test_rgb[i].copy_(f["rgb"])
    glass = test_x[..., 10] > 0.5  # transparent-object pixels (the mask channel of the input)
    half = T.RenderSpec(2048, 2048 * ratio, max_depth=depth, n_bins=nb)
    ref_a = torch.empty_like(test_rgb)
    ref_b = torch.empty_like(test_rgb)
    ref_direct = torch.zeros_like(test_rgb)  # the reference's two parts (mean of the halves)
    ref_caustic = torch.zeros_like(test_rgb)
    for i, g in enumerate(gss):
        for k, dst in enumerate((ref_a, ref_b)):
            T.render(ctx, g, f, half, seed=3, sample_offset=(1 << 24) + k * half.spp,
                     path_offset=(1 << 42) + k * int(half.lights_per_pixel * hw * hw), scene_index=i, guide=guides[i])
            dst[i].copy_(f["rgb"])
            ref_direct[i] += 0.5 * f["direct"]
            ref_caustic[i] += 0.5 * f["caustic"]
    ref = 0.5 * (ref_a + ref_b)
    var_ref = T.mse(ref_a, ref_b) / 4.0
    gen_s = time.perf_counter() - t0
    trainer = D.UNet(ctx, 16, 128, 128)
    t0 = time.perf_counter()
    candidates = {}
    for name, loss_kind, lr, init in (("l1_ssim", N.SC_UNET_LOSS_L1_SSIM, 1.5e-3, 0),
                                      ("l2_linear", N.SC_UNET_LOSS_L2_LINEAR, 1e-3, 1)):
        trainer.set_params(D.he_init(init).to(dev))
        trainer.set_loss(loss_kind)
        T.train(trainer, train, steps=args.den_steps, batch=16, crop=128, lr=lr, lr_final=5e-5, seed=init)
        candidates[name] = trainer.get_params()
    torch.cuda.synchronize(dev)
    train_s = time.perf_counter() - t0
    trainer.close()
    del train
    net = D.UNet(ctx, 1, hw, hw)
    val_mse, test_mse = {}, {}
    for name, prm in candidates.items():
        net.set_params(prm)
        # validation: the network's camera estimate against the validation scene's 512-spp one
        val_mse[name] = T.mse(T.denoise(net, val.x, None, batch=1), torch.expm1(val.target))
        test_mse[name] = T.mse(T.denoise(net, test_x, test_caustic, batch=1), ref) - var_ref
    chosen = min(val_mse, key=val_mse.get)
    net.set_params(candidates[chosen])
    del val
    den = T.denoise(net, test_x, test_caustic, batch=1)
    m_den = T.mse(den, ref) - var_ref
    m_in = T.mse(test_rgb, ref) - var_ref
    # where the denoised frame's error sits: the network's camera estimate against the reference's
    # camera part, the caustic buffer (added back unchanged) against its caustic part, and the
    # transparent-object pixels against the rest (each still carries its share of the reference's
    # own variance)
    den_cam = T.denoise(net, test_x, None, batch=1)
    sq = ((den[..., :3].double() - ref[..., :3].double()) ** 2).sum(-1)
    m_parts = {"network_camera_estimate": T.mse(den_cam, ref_direct),
               "caustic_buffer": T.mse(test_caustic, ref_caustic),
               "input_camera_estimate": T.mse(test_rgb - test_caustic, ref_direct),
               "glass_pixel_share_of_squared_error": float(sq[glass].sum() / sq.sum()),
               "glass_pixel_fraction": float(glass.double().mean())}
    sweep = {}
    for spp in (8, 16, 32, 64, 128, 256, 512, 1024):
        out = torch.empty_like(ref)
        for i, g in enumerate(gss):
            T.render(ctx, g, f, T.RenderSpec(spp, spp * ratio, max_depth=depth, n_bins=nb), seed=7, scene_index=i,
                     guide=guides[i])
            out[i].copy_(f["rgb"])
        sweep[spp] = T.mse(out, ref) - var_ref
    ctx.sync_status()
    budgets = sorted(sweep)
    above = [b for b in budgets if sweep[b] > m_den]
    below = [b for b in budgets if sweep[b] <= m_den]
    if below and above:
        s_lo, s_hi = max(above), min(below)
        a, b = np.log(sweep[s_lo]), np.log(sweep[s_hi])
        spp_match = float(np.exp(np.log(s_lo) + (np.log(m_den) - a) / (b - a) * (np.log(s_hi) - np.log(s_lo))))
    elif below:
        spp_match = float(budgets[0])
    else:
        spp_match = budgets[-1] * sweep[budgets[-1]] / m_den
    g0 = gss[0]
    x1 = torch.empty((1, hw, hw, D.IN_CH), dtype=torch.float32, device=dev)
    y1 = torch.empty((1, hw, hw, D.OUT_CH), dtype=torch.float32, device=dev)
    rgb1 = torch.empty((1, hw, hw, 4), dtype=torch.float32, device=dev)

    def denoised_frame():
        T.render(ctx, g0, f, lo, seed=11, guide=guides[0], chunked=False)
        D.pack_frame(ctx, f, x1, 0, source="direct")
        net.forward(x1, y1)
        D.output_rgb(ctx, y1, f["caustic"], out=rgb1)

    spp_int = max(1, int(np.ceil(spp_match)))
    plain_spec = T.RenderSpec(spp_int, spp_int * ratio, max_depth=depth, n_bins=nb)
    spec_1024 = T.RenderSpec(1024, 1024 * ratio, max_depth=depth, n_bins=nb)

    def plain_frame(spec):
        T.render(ctx, g0, f, spec, seed=11, guide=guides[0], chunked=False)

    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    for _ in range(max(3, args.warmup)):
        denoised_frame()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)

    def timed(fn, reps):
        ev[0].record(stream)
        for _ in range(reps):
            fn()
        ev[1].record(stream)
        torch.cuda.synchronize(dev)
        return ev[0].elapsed_time(ev[1]) / reps

    den_ms = timed(denoised_frame, args.steps)
    plain_frame(plain_spec)
    plain_ms = timed(lambda: plain_frame(plain_spec), max(1, min(args.steps, 3)))
    plain1024_ms = timed(lambda: plain_frame(spec_1024), 1)
    net_ms = timed(lambda: net.forward(x1, y1), args.steps)
    clocks = sampler.stop()
    ctx.sync_status()
    if rank == 0:
        line = {"metric": "denoised fps at the plain tracer's matched MSE (dense 1024^2 scene, 16 objects, ~1M tris)",
                "value": world * 1e3 / den_ms, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
                "warmup": max(3, args.warmup), "ms_per_step": den_ms, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16+f32", "data": "synthetic (scenes.dense_scene)",
                "config": {"workload": "denoise_dense: 1024^2 scenes.dense_scene (16 glass objects, 1.08M tris), 16 bins, "
                                       "depth 12, 8 spp + 32M guided light paths; U-Net on the camera estimate trained "
                                       f"{args.den_steps} steps on 128^2 crops of {n_train} 1024^2 dense-scene pairs "
                                       "(8 -> 512 spp; L1 + SSIM or linear squared error, picked on a validation "
                                       "scene), light-traced caustics added back; 2 held-out scenes; reference "
                                       "2 x (2048 spp + 4x light paths per sample)",
                           "light_paths_per_camera_sample": ratio},
                "mse": {"denoised": m_den, "input": m_in, "reference_variance": var_ref, "plain_sweep": sweep,
                        "plain_1024spp": sweep[1024], "denoised_reaches_plain_1024": m_den <= sweep[1024],
                        "parts": m_parts, "by_loss": {"validation": val_mse, "test": test_mse,
                                                      "chosen": chosen}},
                "matched_spp": spp_match,
                "plain_frame": {"spp": spp_int, "ms": plain_ms, "fps": world * 1e3 / plain_ms},
                "plain_1024spp_frame": {"ms": plain1024_ms, "fps": world * 1e3 / plain1024_ms},
                "fps_ratio_denoised_over_plain_matched": plain_ms / den_ms,
                "fps_ratio_denoised_over_plain_1024": plain1024_ms / den_ms,
                "unet_forward_ms": net_ms, "setup_s": {"data_and_reference": gen_s, "training": train_s},
                "gpu_launches": None, "clocks": clocks, "cpu_baseline": None}
        print(json.dumps(line), flush=True)


def run_caustic_seg(args):
    """The paper's caustic-segmentation experiment (Sec. IV-B, Table II), synthetic -> synthetic: the
    BF16 U-Net trained with the segmentation loss on rendered 128^2 glass scenes labelled by their
    caustic masks, evaluated by IoU on held-out scenes of the training object families and on scenes
    of a family it never saw; against a brightness-threshold baseline."""
    import torch

    from paper_2107_11008_gb300 import denoiser as D
    from paper_2107_11008_gb300 import native as N
    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S
    from paper_2107_11008_gb300 import training as T

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    hw, n_train, n_test = 128, 256, 48
    known, novel = ("sphere", "cylinder", "torus"), ("superellipsoid",)
    spec = T.RenderSpec(16, 128, max_depth=8)
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream)
    t0 = time.perf_counter()

    def scenes(seed0, n, fams):
        return [S.glass_scene(seed0 + i, hw, hw, n_objects=3, tris_per_object=2000, families=fams) for i in range(n)]

    train = T.seg_data(ctx, scenes(20_000 + 1000 * rank, n_train, known), spec, seed=1)
    test_known = T.seg_data(ctx, scenes(30_000, n_test, known), spec, seed=2)
    test_novel = T.seg_data(ctx, scenes(40_000, n_test, novel), spec, seed=3)
    data_s = time.perf_counter() - t0
    net = D.UNet(ctx, 16, hw, hw)
    net.set_params(D.he_init(0).to(dev))
    net.set_loss(N.SC_UNET_LOSS_BCE)
    torch.cuda.synchronize(dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    sampler = ClockSampler(local)
    ev[0].record(stream)
    logged = T.train(net, train, steps=args.seg_steps, batch=16, lr=2e-3, lr_final=1e-4, seed=0, log_every=500)
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ctx.sync_status()
    train_ms = ev[0].elapsed_time(ev[1])
    lab = lambda d: d.target[..., 0] > 0.5  # noqa: E731
    iou_known = T.iou(T.predict_masks(net, test_known.x), lab(test_known))
    iou_novel = T.iou(T.predict_masks(net, test_novel.x), lab(test_novel))
    iou_train = T.iou(T.predict_masks(net, train.x), lab(train))
    thr, (b_known, b_novel) = T.brightness_baseline(train, [test_known, test_novel])
    if rank == 0:
        line = {"metric": "caustic segmentation IoU, held-out scenes of the training object families", "value": iou_known,
                "unit": "IoU", "n_gpus": world, "steps": args.seg_steps, "warmup": 0,
                "ms_per_step": train_ms / args.seg_steps, "higher_is_better": True, "scaling": "weak",
                "vs_baseline": None, "dtype": "bf16", "data": "synthetic (scenes.glass_scene)",
                "config": {"workload": f"caustic_seg: {n_train} training scenes of 128^2 ({'/'.join(known)}, 3 glass "
                                       f"objects each), labels = non-local caustic masks, input = rendered RGB "
                                       f"(16 spp + 128 guided light paths/px); tests: {n_test} scenes of the same "
                                       f"families, {n_test} of an unseen family ({novel[0]})",
                           "loss": "binary cross-entropy with logits (sc_unet_set_loss)", "batch": 16,
                           "steps": args.seg_steps},
                "iou": {"known_objects": iou_known, "novel_objects": iou_novel, "training_images": iou_train},
                "brightness_threshold_baseline": {"threshold_log1p_luminance": thr, "known_objects": b_known,
                                                  "novel_objects": b_novel},
                "caustic_pixel_fraction": {"train": float(lab(train).float().mean()),
                                           "known": float(lab(test_known).float().mean()),
                                           "novel": float(lab(test_novel).float().mean())},
                "loss_log": logged, "data_generation_s": data_s, "train_images_s": 16e3 * args.seg_steps / train_ms,
                "gpu_launches": None, "clocks": clocks, "cpu_baseline": None}
        print(json.dumps(line), flush=True)


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.lines = []
        self.proc = None
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(gpu_index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            p = [x.strip() for x in ln.split(",")]
            if len(p) < 9:
                continue
            try:
                sm.append(float(p[1]))
                mx.append(float(p[2]))
            except ValueError:
                continue
            for n, v in zip(names, p[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx), "reasons": sorted(reasons),
                "samples": len(sm)}


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f)
    except Exception:  # noqa: BLE001
        return {}


def cpu_baseline(scene, spp_full, nl_full, seconds, depth=12, nbins=8):
    """The FP64 oracle, as it stands, on a bounded sample of the same frame (rows of pixels at 4 spp
    plus light paths), on this host's cores."""
    import oracle as O

    cores = len(os.sched_getaffinity(0))
    orc = O.OracleScene(scene)
    W, H = scene.camera.width, scene.camera.height
    # calibrate on a 1-spp band of rows, then size the sample (rows x spp) to about `seconds`
    band = max(1, H // 8)
    t0 = time.perf_counter()
    orc.trace_camera(1, depth, nbins=nbins, window=(0, W, H // 2 - band // 2, H // 2 - band // 2 + band),
                     records=False, n_threads=cores)
    per_path = max(time.perf_counter() - t0, 1e-3) / (band * W)
    budget = 0.85 * seconds / per_path  # camera paths that fit
    if budget >= W * H:
        rows, spp = H, int(max(1, min(spp_full, budget // (W * H))))
    else:
        rows, spp = max(1, int(budget // W)), 1
    y0 = max(0, H // 2 - rows // 2)
    n_light = max(4096, int(0.15 * seconds / max(per_path, 1e-9)))
    t0 = time.perf_counter()
    orc.trace_camera(spp, depth, nbins=nbins, window=(0, W, y0, y0 + rows), records=False, n_threads=cores)
    t_cam = time.perf_counter() - t0
    t0 = time.perf_counter()
    orc.trace_lights(n_light, depth, nbins=nbins, records=False, n_threads=cores)
    t_light = time.perf_counter() - t0
    paths = rows * W * spp + n_light
    return {"value": paths / (t_cam + t_light) / 1e6, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"{rows} rows x {W} px x {spp} spp camera paths + {n_light} light paths of the same frame "
                      f"({t_cam + t_light:.1f} s on {cores} cores); full frame is {spp_full} spp + {nl_full} light paths",
            "seconds": t_cam + t_light}


def measure_peaks(ctx, dev, stream, repeats=5):
    """FP32 FMA throughput (TFLOP/s) and L2 read bandwidth (GB/s) on this device, best of
    `repeats` launches of the library's measurement kernels, each sized to about 20 ms."""
    import torch

    from paper_2107_11008_gb300 import native as N

    sink = torch.zeros(1, dtype=torch.float32, device=dev)
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]

    def best(launch):
        out = []
        for _ in range(repeats):
            ev[0].record(stream)
            work = launch()
            ev[1].record(stream)
            torch.cuda.synchronize(dev)
            out.append(work / (ev[0].elapsed_time(ev[1]) * 1e-3))
        return max(out)

    iters = 1 << 14
    N.sc_peak_fma(ctx.handle, iters, sink.data_ptr())  # warm-up
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    N.sc_peak_fma(ctx.handle, iters, sink.data_ptr())
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    iters = max(16, int(iters * 20.0 / max(ev[0].elapsed_time(ev[1]), 1e-3)) // 16 * 16)
    fma = best(lambda: N.sc_peak_fma(ctx.handle, iters, sink.data_ptr())) / 1e12
    nbytes = 32 << 20  # resident in the 129 MB L2
    buf = torch.ones(nbytes // 4, dtype=torch.float32, device=dev)
    reps = 64
    N.sc_peak_l2_read(ctx.handle, buf.data_ptr(), nbytes, reps, sink.data_ptr())
    torch.cuda.synchronize(dev)
    ev[0].record(stream)
    N.sc_peak_l2_read(ctx.handle, buf.data_ptr(), nbytes, reps, sink.data_ptr())
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    reps = max(1, int(reps * 20.0 / max(ev[0].elapsed_time(ev[1]), 1e-3)))
    l2 = best(lambda: N.sc_peak_l2_read(ctx.handle, buf.data_ptr(), nbytes, reps, sink.data_ptr())) / 1e9
    return {"fp32_tflops": fma, "l2_read_gbs": l2,
            "how": f"sc_peak_fma ({iters} steps x 8 chains x SMs x 2048 threads) and sc_peak_l2_read (32 MB x {reps} "
                   "passes, L1 bypassed), best of 5 launches of ~20 ms each, CUDA events, just before the timed region"}


def measure_cfg1(local, steps=20, warmup=3):
    """The 64x64 parity workload as a frame: LBVH build + 16 spp camera paths (depth 8) + resolve."""
    import torch

    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S

    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    sc = S.ball_on_plane()
    ctx = R.Context(local, stream)
    arrays = R.SceneArrays(sc, dev)
    frame = R.Frame(sc.camera.width, sc.camera.height, device=dev)
    spp, depth = 16, 8

    def frame_once():
        gs = R.GpuScene(ctx, arrays)
        frame.zero_accumulators()
        R.trace_camera(ctx, gs, frame, spp, depth)
        R.resolve(ctx, gs, frame, spp, 0)
        gs.free()

    for _ in range(warmup):
        frame_once()
    ctx.sync_status()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(2)]
    ev[0].record(stream)
    for _ in range(steps):
        frame_once()
    ev[1].record(stream)
    torch.cuda.synchronize(dev)
    ctx.sync_status()
    ms = ev[0].elapsed_time(ev[1]) / steps
    paths = sc.camera.width * sc.camera.height * spp
    ctx.close()
    return {"workload": "cfg1 ball_on_plane: 64^2, glass icosphere 1280 tris on a plane, point light, 16 spp, depth 8, "
                        "LBVH build + camera + resolve per frame (latency-bound)",
            "ms_per_frame": ms, "frames_per_s": 1e3 / ms, "camera_mpaths_s": paths / (ms * 1e-3) / 1e6,
            "steps": steps, "warmup": warmup}


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    from paper_2107_11008_gb300 import scenes as S

    sc = S.glass_scene(0, width=args.res, height=args.res)
    # each step: a bounded sample of the frame; sized so that warmup + steps stay within minutes
    # (and at most --cpu-seconds)
    per_step = max(2.0, min(20.0, 150.0 / max(1, args.steps + args.warmup), args.cpu_seconds))
    vals, secs = [], []
    cb = None
    for i in range(args.warmup + args.steps):
        r = cpu_baseline(sc, args.spp, args.light_paths, per_step)
        if i >= args.warmup:
            vals.append(r["value"])
            secs.append(r["seconds"])
            cb = r
    v = statistics.mean(vals)
    line = {"metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(secs), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": {"workload": WORKLOAD + " (oracle on a bounded sample of the frame per step)",
                       "resolution": args.res},
            "cpu_baseline": {"value": v, "unit": UNIT, "cores": cb["cores"], "kind": "oracle", "sample": cb["sample"]},
            "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
        return
    if args.workload == "batch64":
        run_batch(args)
        return
    if args.workload == "unet_train":
        run_unet_train(args)
        return
    if args.workload == "denoise":
        run_denoise(args)
        return
    if args.workload == "caustic_seg":
        run_caustic_seg(args)
        return
    if args.workload == "denoise_dense":
        run_denoise_dense(args)
        return
    import torch
    import torch.distributed as dist

    from paper_2107_11008_gb300 import renderer as R
    from paper_2107_11008_gb300 import scenes as S

    rank, world, local = dist_env()
    if world > 1:
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    res, spp, nl, depth, nbins = args.res, args.spp, args.light_paths, 12, 8
    scene = S.glass_scene(0, width=res, height=res)
    host_arrays = R.SceneArrays(scene, "cpu")
    dev_arrays = R.SceneArrays(scene, dev)
    stream = torch.cuda.current_stream(dev)
    ctx = R.Context(local, stream)
    R.N.sc_set_camera_engine(ctx.handle, {"wavefront": R.N.SC_CAMERA_WAVEFRONT,
                                          "persistent": R.N.SC_CAMERA_PERSISTENT}[args.camera_engine])
    frame = R.Frame(res, res, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)  # > 129 MB L2
    sample_offset = rank * spp  # disjoint sample ranges per rank

    def step(arrays, ev=None):
        if ev:
            ev[0].record(stream)
        gs = R.GpuScene(ctx, arrays)
        if ev:
            ev[1].record(stream)
        frame.zero_accumulators()
        R.trace_camera(ctx, gs, frame, spp, depth, nbins, seed=1, sample_offset=sample_offset)
        if ev:
            ev[2].record(stream)
        R.trace_lights(ctx, gs, frame, nl, depth, nbins, seed=2, path_offset=rank * nl)
        if ev:
            ev[3].record(stream)
        R.resolve(ctx, gs, frame, spp, nl)
        if ev:
            ev[4].record(stream)
        gs.free()

    for _ in range(args.warmup):
        step(dev_arrays)
    ctx.sync_status()

    # traversal work per launch (untimed pass with counters on)
    counters = torch.zeros(3, dtype=torch.int64, device=dev)
    gs = R.GpuScene(ctx, dev_arrays)
    R.N.sc_set_counters(ctx.handle, counters.data_ptr())
    frame.zero_accumulators()
    R.trace_camera(ctx, gs, frame, spp, depth, nbins, seed=1, sample_offset=sample_offset)
    torch.cuda.synchronize(dev)
    cam_counts = counters.cpu().tolist()
    counters.zero_()
    R.trace_lights(ctx, gs, frame, nl, depth, nbins, seed=2)
    torch.cuda.synchronize(dev)
    light_counts = counters.cpu().tolist()
    R.N.sc_set_counters(ctx.handle, None)
    gs.free()

    mp = measure_peaks(ctx, dev, stream)

    # timed region: K steps, L2 flushed between steps, CUDA events on the launching stream
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(5)] for _ in range(args.steps)]
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize(dev)
    sampler = ClockSampler(local)
    for k in range(args.steps):
        flush.zero_()
        step(dev_arrays, evs[k])
    torch.cuda.synchronize(dev)
    clocks = sampler.stop()
    ctx.sync_status()
    if world > 1:
        dist.barrier()
    step_ms = [e[0].elapsed_time(e[4]) for e in evs]
    build_ms = [e[0].elapsed_time(e[1]) for e in evs]
    cam_ms = [e[1].elapsed_time(e[2]) for e in evs]
    light_ms = [e[2].elapsed_time(e[3]) for e in evs]
    resolve_ms = [e[3].elapsed_time(e[4]) for e in evs]
    total_ms = sum(step_ms)
    if world > 1:
        t = torch.tensor([total_ms], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        total_ms = float(t.item())
    ms_per_step = total_ms / args.steps
    paths_per_step = res * res * spp + nl
    value = world * paths_per_step / (ms_per_step * 1e-3) / 1e6

    # end to end through the C ABI with host buffers: H2D of the scene, D2H of the frame outputs
    e2e_steps = min(3, args.steps)
    outs = ("rgb", "depth", "normal_world", "normal_camera", "instance_id", "mask", "caustic_mask", "albedo")
    pinned = {k: torch.empty(frame[k].shape, dtype=frame[k].dtype, pin_memory=True) for k in outs}
    d2h = sum(p.numel() * p.element_size() for p in pinned.values())
    h2d = host_arrays.nbytes()
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        step(host_arrays)
        for k in outs:
            pinned[k].copy_(frame[k], non_blocking=True)
        torch.cuda.synchronize(dev)
    e2e_s = (time.perf_counter() - t0) / e2e_steps
    if world > 1:
        t = torch.tensor([e2e_s], device=dev)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        e2e_s = float(t.item())
    e2e_value = world * paths_per_step / e2e_s / 1e6

    pk = peaks()
    cam_s = statistics.mean(cam_ms) * 1e-3
    cam_flops = cam_counts[1] * FLOPS_PER_NODE + cam_counts[2] * FLOPS_PER_TRI
    cam_bytes = cam_counts[1] * BYTES_PER_NODE + cam_counts[2] * BYTES_PER_TRI
    hbm_peak = pk.get("hbm_gbs", 6800.0)
    dram = CAMERA_DRAM_BYTES[args.camera_engine]
    bounds = {
        "fp32": {"achieved": cam_flops / cam_s / 1e12, "peak": mp["fp32_tflops"], "unit": "TFLOP/s",
                 "per_launch": cam_flops},
        "l2": {"achieved": cam_bytes / cam_s / 1e9, "peak": mp["l2_read_gbs"], "unit": "GB/s",
               "per_launch": cam_bytes},
    }
    if dram is not None:
        bounds["hbm"] = {"achieved": dram / cam_s / 1e9, "peak": hbm_peak, "unit": "GB/s", "per_launch": dram}
    for b in bounds.values():
        b["frac"] = b["achieved"] / b["peak"]
    # the attainable rate is the minimum over the three ceilings: the binding one has the largest fraction
    bind = max(bounds, key=lambda k: bounds[k]["frac"])
    cam_kernel = ("camera traversal: k_wf_extend + k_wf_shadow, timed over the whole camera phase (all its kernels)"
                  if args.camera_engine == "wavefront" else "k_trace_camera_t")
    roofline = {"kernel": cam_kernel, "bound": {"fp32": "alu", "l2": "l2", "hbm": "hbm"}[bind],
                "achieved": bounds[bind]["achieved"], "peak": bounds[bind]["peak"], "unit": bounds[bind]["unit"],
                "frac": bounds[bind]["frac"], "traffic": dram, "traffic_unit": "bytes per camera phase (ncu)",
                "bounds": bounds,
                "peak_source": "fp32 and l2: measured in this run (" + mp["how"] + "); hbm: MEASURED_PEAKS hbm_gbs "
                               "(of measured)",
                "algorithmic": f"per 4-wide node visit {BYTES_PER_NODE} B + {FLOPS_PER_NODE} flop, per triangle test "
                               f"{BYTES_PER_TRI} B + {FLOPS_PER_TRI} flop, counted live (sc_set_counters)"}
    subs = {}
    if not args.no_sub and rank == 0:
        subs["cfg1"] = measure_cfg1(local)
        bms, sms, info = measure_batch(1, 1, local, world)
        subs["batch64"] = {"workload": BATCH_WORKLOAD, "camera_paths": info["camera_paths"],
                           "triangles": info["triangles"], "ms_per_launch": bms,
                           "mpaths_s": info["camera_paths"] / (bms * 1e-3) / 1e6,
                           "sequential_ms": sms, "sequential_mpaths_s": info["camera_paths"] / (sms * 1e-3) / 1e6,
                           "batch_over_sequential": sms / bms, "steps": 1, "warmup": 1,
                           "scene_generation_s": info["scene_generation_s"], "lbvh_build_s": info["lbvh_build_s"]}
        u = measure_unet_train(10, 3, local, world, e2e=False)
        subs["unet_train"] = {"workload": UNET_WORKLOAD, "ms_per_step": u["ms"],
                              "images_s": u["batch"] / (u["ms"] * 1e-3), "forward_ms": u["forward_ms"],
                              "roofline": unet_roofline(u["ms"], u["batch"], u["hw"]), "steps": 10, "warmup": 3}
    if rank == 0:
        cb = None
        if not args.no_cpu_baseline and world == 1:
            try:
                cb = cpu_baseline(scene, spp, nl, args.cpu_seconds)
                cb.pop("seconds", None)
            except Exception as e:  # noqa: BLE001
                cb = {"value": None, "unit": UNIT, "cores": len(os.sched_getaffinity(0)), "kind": "oracle",
                      "sample": f"failed: {e}"}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "resolution": res, "spp": spp, "light_paths": nl, "max_depth": depth,
                       "wavelength_bins": nbins, "triangles": scene.n_tris, "parallelism": f"replicas x{world}",
                       "camera_engine": args.camera_engine,
                       "l2": "flushed between steps (256 MB write)"},
            "frames_per_s": world * 1e3 / ms_per_step,
            "camera_mpaths_s": world * res * res * spp / (statistics.mean(cam_ms) * 1e-3) / 1e6,
            "light_mpaths_s": world * nl / (statistics.mean(light_ms) * 1e-3) / 1e6,
            "phase_ms": {"lbvh_build": statistics.mean(build_ms), "trace_camera": statistics.mean(cam_ms),
                         "trace_lights": statistics.mean(light_ms), "resolve": statistics.mean(resolve_ms)},
            "traversal": {"camera": {"queries": cam_counts[0], "nodes": cam_counts[1], "tris": cam_counts[2]},
                          "lights": {"queries": light_counts[0], "nodes": light_counts[1], "tris": light_counts[2]},
                          "camera_grays_s": cam_counts[0] / cam_s / 1e9,
                          "camera_l2_side_gbs": cam_bytes / cam_s / 1e9},
            "roofline": roofline,
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": (launches_per_step_base(scene.n_tris) + camera_launches(args.camera_engine, res, res, spp,
                                                                                     depth)) *
                            args.steps,
            "clocks": clocks,
            "cpu_baseline": cb,
        }
        if subs:
            line["sub_results"] = subs
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
