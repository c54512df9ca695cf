"""Failure detection and training resume, through the C ABI.

Traversal limits: a query that exceeds its node-visit budget or its stack depth is abandoned, the
kernel latches a status bit and sc_sync_status returns SC_ERR_TIMEOUT / SC_ERR_STACK_OVERFLOW; the
context stays usable and the next launch with the default limits renders what it rendered before
(up to the order of its float additions).  No kernel traps: the limits only end loops early.

Tensor-core waits: every mbarrier wait of the U-Net kernels is bounded; on giving up a role raises
its CTA's abort flag, waits (bounded) for the copies and MMAs it has in flight, and the CTA frees its
TMEM and latches the watchdog bit.  A self-test CTA runs that path for real (its waits are on a
barrier nothing arrives at) and the network computes the same output afterwards.

Resume: U-Net training for N steps straight equals N/2 steps, a checkpoint written to a file and
read into a new network, and N/2 more steps -- bit for bit in parameters, Adam moments and step.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_11008_gb300 import denoiser as D  # noqa: E402
from paper_2107_11008_gb300 import native as N  # noqa: E402
from paper_2107_11008_gb300 import renderer as R  # noqa: E402
from paper_2107_11008_gb300 import scenes as S  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = R.Context(0)
    yield c
    N.sc_set_limits(c.handle, defaults=True)
    c.close()


def _frame(ctx, gs, sc, spp=2, n_light=0):
    fr = R.Frame(sc.camera.width, sc.camera.height)
    R.trace_camera(ctx, gs, fr, spp, 8)
    if n_light:
        R.trace_lights(ctx, gs, fr, n_light, 8)
    return fr


def test_default_limits_and_validation(ctx):
    lim = N.sc_get_limits(ctx.handle)
    assert (lim.max_visits, lim.stack_depth4, lim.stack_depth2) == (1 << 22, 96, 64)
    for bad in (dict(stack_depth4=97), dict(stack_depth2=65), dict(max_visits=-1)):
        with pytest.raises(N.ScError) as e:
            N.sc_set_limits(ctx.handle, **bad)
        assert e.value.code == -1
    N.sc_set_limits(ctx.handle, max_visits=1000)
    lim = N.sc_get_limits(ctx.handle)
    assert (lim.max_visits, lim.stack_depth4, lim.stack_depth2) == (1000, 96, 64)  # 0 = default
    N.sc_set_limits(ctx.handle, defaults=True)


@pytest.mark.parametrize("which", ["visits_camera", "stack4_camera", "visits_lights", "stack2_lights"])
def test_traversal_limits_report_and_recover(ctx, which):
    sc = S.ball_on_plane(32, 32)
    gs = R.GpuScene(ctx, sc)
    ref = _frame(ctx, gs, sc, n_light=4096)
    ctx.sync_status()
    limits = {"visits_camera": dict(max_visits=3), "stack4_camera": dict(stack_depth4=1),
              "visits_lights": dict(max_visits=3), "stack2_lights": dict(stack_depth2=1)}[which]
    code = -5 if "visits" in which else -4
    N.sc_set_limits(ctx.handle, **limits)
    fr = R.Frame(sc.camera.width, sc.camera.height)
    if which.endswith("camera"):
        R.trace_camera(ctx, gs, fr, 2, 8)
    else:
        R.trace_lights(ctx, gs, fr, 4096, 8)
    with pytest.raises(N.ScError) as e:
        ctx.sync_status()
    assert e.value.code == code, N.sc_last_error(ctx.handle)
    # the status is cleared once reported, and the context keeps working with the defaults
    N.sc_set_limits(ctx.handle, defaults=True)
    ctx.sync_status()
    again = _frame(ctx, gs, sc, n_light=4096)
    ctx.sync_status()
    np.testing.assert_allclose(again["accum_camera"].cpu().numpy(), ref["accum_camera"].cpu().numpy(), rtol=1e-5,
                               atol=1e-6)


def _batch(seed, n=2, h=32, w=32):
    rng = np.random.default_rng(seed)
    x = rng.random((n, h, w, 11)).astype(np.float32)
    t = rng.random((n, h, w, 3)).astype(np.float32)
    return torch.from_numpy(x).cuda(), torch.from_numpy(t).cuda()


def _train(net, batches, lr=1e-3):
    for x, t in batches:
        net.train_step(x, t, lr)


def test_training_resumes_bit_for_bit_from_a_checkpoint(ctx, tmp_path):
    batches = [_batch(s) for s in range(6)]
    init = D.he_init(3).cuda()
    straight = D.UNet(ctx, 2, 32, 32)
    straight.set_params(init)
    _train(straight, batches)
    p_ref, m_ref, v_ref, step_ref = straight.get_state()
    ctx.sync_status()
    assert step_ref == 6

    first = D.UNet(ctx, 2, 32, 32)
    first.set_params(init)
    _train(first, batches[:3])
    path = str(tmp_path / "unet.ckpt")
    first.save(path)
    first.close()
    # a network of another geometry loads the same state (it does not depend on the workspace)
    resumed = D.UNet(ctx, 4, 32, 32)
    resumed.load(path)
    assert resumed.get_state()[3] == 3
    _train(resumed, batches[3:])
    p, m, v, step = resumed.get_state()
    ctx.sync_status()
    assert step == 6
    for a, b in ((p, p_ref), (m, m_ref), (v, v_ref)):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    assert float((m_ref != 0).float().mean()) > 0.5  # the moments are really part of the state


def test_state_round_trip_and_bad_checkpoints(ctx, tmp_path):
    net = D.UNet(ctx, 2, 32, 32)
    net.set_params(D.he_init(1).cuda())
    _train(net, [_batch(9), _batch(10)])
    p, m, v, step = net.get_state()
    other = D.UNet(ctx, 2, 32, 32)
    other.set_state(p, m, v, step)
    p2, m2, v2, step2 = other.get_state()
    ctx.sync_status()
    assert step2 == step == 2
    for a, b in ((p, p2), (m, m2), (v, v2)):
        np.testing.assert_array_equal(a.cpu().numpy(), b.cpu().numpy())
    # missing, truncated and foreign files are rejected and leave the network unchanged
    path = tmp_path / "good.ckpt"
    net.save(str(path))
    data = path.read_bytes()
    (tmp_path / "short.ckpt").write_bytes(data[: len(data) // 2])
    (tmp_path / "foreign.ckpt").write_bytes(b"NOTACKPT" + data[8:])
    for bad in ("missing.ckpt", "short.ckpt", "foreign.ckpt"):
        with pytest.raises(N.ScError) as e:
            other.load(str(tmp_path / bad))
        assert e.value.code == -1
    np.testing.assert_array_equal(other.get_params().cpu().numpy(), p.cpu().numpy())
    assert other.get_state()[3] == 2
    with pytest.raises(N.ScError):
        net.save(str(tmp_path / "no_such_dir" / "x.ckpt"))


@pytest.mark.parametrize("limit", [1 << 8, 1 << 14])
def test_tensor_core_wait_gives_up_and_the_context_recovers(ctx, limit):
    net = D.UNet(ctx, 2, 32, 32)
    net.set_params(D.he_init(5).cuda())
    x, _ = _batch(11)
    before = net.forward(x).clone()
    ctx.sync_status()
    out = N.sc_unet_wait_selftest(ctx.handle, limit)
    # every role gave up, the copy and the MMA in flight completed before the CTA freed its TMEM
    assert out[:7] == [1, 1, 1, 1, 1, 2, 1], out
    print(f"{limit} polls of an abandoned wait: {out[7] / 1e3:.1f} us")
    assert out[7] > 0
    with pytest.raises(N.ScError) as e:
        ctx.sync_status()
    assert e.value.code == -5, N.sc_last_error(ctx.handle)
    ctx.sync_status()  # reported once, then cleared
    after = net.forward(x)
    ctx.sync_status()
    torch.testing.assert_close(after, before, rtol=0, atol=0)
    net.close()


def test_tensor_core_wait_selftest_rejects_bad_limits(ctx):
    for bad in (0, (1 << 24) + 1):
        with pytest.raises(N.ScError) as e:
            N.sc_unet_wait_selftest(ctx.handle, bad)
        assert e.value.code == -1
