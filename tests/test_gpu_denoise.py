"""What the learned part gains: the U-Net trained on the tracer's own low/high-sample pairs,
evaluated on held-out scenes against the plain low-sample render (both vs a high-sample target)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_11008_gb300 import denoiser as D  # noqa: E402
from paper_2107_11008_gb300 import renderer as R  # noqa: E402
from paper_2107_11008_gb300 import scenes as S  # noqa: E402
from paper_2107_11008_gb300 import training as T  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = R.Context(0)
    yield c
    c.close()


def test_pairs_use_disjoint_samples_and_same_estimator(ctx):
    sc = [S.denoise_scene(7, 32, 32)]
    lo, hi = T.RenderSpec(16, 16), T.RenderSpec(16, 16)
    p = T.make_pairs(ctx, sc, lo, hi, seed=3)
    # equal budgets, disjoint samples: different noise, same expectation
    a, b = p.rgb_lo[..., :3], p.rgb_hi[..., :3]
    assert not torch.equal(a, b)
    assert abs(float(a.mean()) - float(b.mean())) < 0.25 * float(b.mean())
    np.testing.assert_allclose(p.target.cpu().numpy(), np.log1p(np.maximum(b.cpu().numpy(), 0)), rtol=1e-6)
    np.testing.assert_allclose(p.x[..., :3].cpu().numpy(), np.log1p(np.maximum(a.cpu().numpy(), 0)), rtol=1e-6)


@pytest.mark.parametrize("source,lights", [("rgb", 4), ("direct", 1024)])
def test_trained_denoiser_beats_the_noisy_input(ctx, source, lights):
    """rgb: the network denoises the whole 4-spp image (4 light paths / px); direct: it denoises
    the 4-spp camera estimate and the caustic buffer of 1024 light paths / px is added back."""
    # rgb: uniform light emission, so that the network's input carries the noisy caustics it is
    # asked to remove; direct: guided emission (the production setting)
    guided = source == "direct"
    lo = T.RenderSpec(spp=4, lights_per_pixel=lights, guided=guided)
    hi = T.RenderSpec(spp=512, lights_per_pixel=4096, guided=guided)
    train = T.make_pairs(ctx, [S.denoise_scene(i, 64, 64) for i in range(48)], lo, hi, seed=1, source=source)
    test = T.make_pairs(ctx, [S.denoise_scene(1000 + i, 64, 64) for i in range(8)], lo, hi, seed=2, source=source)
    net = D.UNet(ctx, 8, 64, 64)
    net.set_params(D.he_init(0).cuda())
    log = T.train(net, train, steps=800, batch=8, lr=2e-3, lr_final=1e-4, log_every=100)
    ctx.sync_status()
    assert log[-1][1] < log[0][1]
    den = T.denoise(net, test.x, test.add())
    m_noisy = T.mse(test.rgb_lo, test.rgb_hi)
    m_den = T.mse(den, test.rgb_hi)
    # log-space error, which the network is trained in
    lt = torch.log1p(test.rgb_hi[..., :3].clamp_min(0))
    l_noisy = float(((torch.log1p(test.rgb_lo[..., :3].clamp_min(0)) - lt) ** 2).mean())
    l_den = float(((torch.log1p(den[..., :3]) - lt) ** 2).mean())
    print(f"[{source}, {lights} light paths/px] held-out MSE: noisy {m_noisy:.4g}, denoised {m_den:.4g} "
          f"(log space {l_noisy:.4g} -> {l_den:.4g}); losses {log}")
    # rgb: the whole-image network blurs the sharp caustics and gains little in linear MSE, which
    # it is not trained on: over eight runs on these inputs the linear ratio spread from 0.57 to
    # 0.91 (float-atomic splats and gradient reductions make each run's training differ in the
    # last bits, and 800 steps at this rate amplify that), while the log-space ratio stayed in
    # 0.41-0.53; so the linear bound only asks that it not be worse.  direct: the caustic buffer
    # added back carries its own noise, which the network does not touch and which bounds the
    # gain near 2x at this budget
    assert m_den < (1.0 if source == "rgb" else 0.6) * m_noisy
    assert l_den < (0.7 if source == "rgb" else 0.5) * l_noisy
    net.close()



def test_denoised_frame_beats_the_plain_tracer_at_several_times_its_samples(ctx):
    """The matched-MSE ordering of the denoising pipeline on held-out scenes: 4 camera spp + the
    light-traced caustics, the camera estimate denoised, against the plain tracer spending the same
    light paths per camera sample at 4, 8, 12, 16 and 32 spp; MSEs against a two-half reference
    with the reference's own variance subtracted.  The denoised frame must beat the plain one at 3x
    its samples (the full-size comparison, with its timing, is the bench's denoise workloads)."""
    hw, ratio = 128, 16
    lo = T.RenderSpec(4, 4 * ratio)
    train = T.make_pairs(ctx, [S.denoise_scene(i, hw, hw) for i in range(64)], lo, T.RenderSpec(1024, 0), seed=1,
                         source="direct")
    scenes = [S.denoise_scene(20_000 + i, hw, hw) for i in range(4)]
    test = T.make_pairs(ctx, scenes, lo, T.RenderSpec(0, 0), seed=2, source="direct")
    gss = [R.GpuScene(ctx, s) for s in scenes]
    guides = [S.guide_sphere(s) for s in scenes]
    f = R.Frame(hw, hw)
    half = T.RenderSpec(1024, 1024 * ratio)
    ref_ab = [torch.empty_like(test.rgb_lo) for _ in range(2)]
    for i, g in enumerate(gss):
        for k, dst in enumerate(ref_ab):
            T.render(ctx, g, f, half, seed=3, sample_offset=(1 << 24) + k * half.spp,
                     path_offset=(1 << 42) + k * int(half.lights_per_pixel) * hw * hw, scene_index=i, guide=guides[i])
            dst[i].copy_(f["rgb"])
    ref = 0.5 * (ref_ab[0] + ref_ab[1])
    var_ref = T.mse(ref_ab[0], ref_ab[1]) / 4.0
    # L1 + SSIM: on these single-ball scenes it beats the linear squared error (3.4e-5 against 6.8e-5
    # at this budget), the reverse of the dense scene; the bench workloads pick per scene family
    net = D.UNet(ctx, 16, 64, 64)
    net.set_params(D.he_init(0).cuda())
    T.train(net, train, steps=4000, batch=16, crop=64, lr=1.5e-3, lr_final=5e-5, seed=0)
    full = D.UNet(ctx, 4, hw, hw)
    full.set_params(net.get_params())
    m_den = T.mse(T.denoise(full, test.x, test.add()), ref) - var_ref
    sweep = {}
    for spp in (4, 8, 12, 16, 32):
        out = torch.empty_like(ref)
        for i, g in enumerate(gss):
            T.render(ctx, g, f, T.RenderSpec(spp, spp * ratio), seed=7, scene_index=i, guide=guides[i])
            out[i].copy_(f["rgb"])
        sweep[spp] = T.mse(out, ref) - var_ref
    ctx.sync_status()
    print(f"held-out MSE: denoised {m_den:.4g}; plain {', '.join(f'{s} spp {m:.4g}' for s, m in sweep.items())}; "
          f"reference variance {var_ref:.3g}")
    assert var_ref < 0.1 * sweep[32]  # the reference resolves the errors it measures
    assert sweep[4] > sweep[8] > sweep[16] > sweep[32]  # the plain tracer converges
    assert m_den < sweep[12]
    net.close()
    full.close()
