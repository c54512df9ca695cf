"""The caustic-segmentation sanity run (the paper's Sec. IV-B experiment, synthetic -> synthetic): a
U-Net trained with the segmentation loss on rendered glass scenes, labelled by their caustic masks,
segments the caustics of held-out scenes -- of the training object families and of a family it never
saw -- better than the method without it (a brightness threshold fitted on the training images)."""
import pytest

torch = pytest.importorskip("torch")

from paper_2107_11008_gb300 import denoiser as D  # noqa: E402
from paper_2107_11008_gb300 import native as N  # noqa: E402
from paper_2107_11008_gb300 import renderer as R  # noqa: E402
from paper_2107_11008_gb300 import scenes as S  # noqa: E402
from paper_2107_11008_gb300 import training as T  # noqa: E402

pytestmark = pytest.mark.gpu


def test_segmentation_network_beats_brightness_threshold():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = R.Context(0)
    hw = 64
    spec = T.RenderSpec(8, 64, max_depth=8)

    def scenes(seed0, n, fams):
        return [S.glass_scene(seed0 + i, hw, hw, n_objects=3, tris_per_object=1500, families=fams) for i in range(n)]

    train = T.seg_data(ctx, scenes(20_000, 64, ("sphere", "cylinder", "torus")), spec, seed=1)
    known = T.seg_data(ctx, scenes(30_000, 16, ("sphere", "cylinder", "torus")), spec, seed=2)
    novel = T.seg_data(ctx, scenes(40_000, 16, ("superellipsoid",)), spec, seed=3)
    lab = lambda d: d.target[..., 0] > 0.5  # noqa: E731
    assert 0.005 < float(lab(train).float().mean()) < 0.3  # the labels mark some, not most, pixels
    net = D.UNet(ctx, 16, hw, hw)
    net.set_params(D.he_init(0).cuda())
    net.set_loss(N.SC_UNET_LOSS_BCE)
    log = T.train(net, train, steps=1500, batch=16, lr=2e-3, lr_final=1e-4, seed=0, log_every=250)
    ctx.sync_status()
    assert log[-1][1] < 0.6 * log[0][1]
    iou_known = T.iou(T.predict_masks(net, known.x), lab(known))
    iou_novel = T.iou(T.predict_masks(net, novel.x), lab(novel))
    _, (b_known, b_novel) = T.brightness_baseline(train, [known, novel])
    print(f"IoU known {iou_known:.3f} (threshold {b_known:.3f}), novel {iou_novel:.3f} (threshold {b_novel:.3f})")
    assert iou_known > b_known and iou_known > 0.3
    assert iou_novel > b_novel
    net.close()
    ctx.close()
