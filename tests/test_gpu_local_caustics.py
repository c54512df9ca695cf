"""Local caustics on the GPU (caustics seen through glass; Sec. III-D local caustic mask) against
the oracle: photons per light path, the gather per camera path, the closed form of a collimated
beam through a glass slab, and the resolve pass's local-caustic buffer and mask."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import oracle as O  # noqa: E402
from paper_2107_11008_gb300 import native as N  # noqa: E402
from paper_2107_11008_gb300 import renderer as R  # noqa: E402
from paper_2107_11008_gb300 import scenes as S  # noqa: E402

from .parity import REL, rel_close, split_ambiguous  # noqa: E402
from .test_oracle_local_caustics import E0, R_BEAM, RADIUS, RHO, _beam_through_slab  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    c = R.Context(0)
    yield c
    c.close()


def fp32_point_err(sc):
    """Bound on the FP32 hit point's distance from the FP64 one, in metres: the point is the
    barycentric interpolation of the hit triangle's vertices, so its error scales with their
    coordinates V, not with the point: about 3u*V from the barycentrics' own rounding, u*V from
    b0 = 1 - b1 - b2 and 4u*V from the three products and two sums (u = 2^-24).  With the floors
    of these scenes at +-10 m that is 4.8e-6 m, 1.6e-4 of the slab's gather radius."""
    return 8 * 2.0 ** -24 * float(np.abs(sc.positions).max())


def _glass(width=40, height=32):
    return S.glass_scene(seed=1, width=width, height=height, n_objects=3, tris_per_object=2000)


def _run(ctx, sc, n_light, spp, nbins, flags, radius, guide=None, seed=4):
    gs = R.GpuScene(ctx, sc)
    pm = R.PhotonMap(ctx, gs, n_light, radius, 8, n_bins=nbins, seed=seed + 1, flags=flags, guide=guide)
    fr = R.Frame(sc.camera.width, sc.camera.height)
    fr.alloc_path_records(spp)
    pm.gather(gs, fr, spp, 8, n_bins=nbins, seed=seed, flags=flags)
    R.resolve(ctx, gs, fr, spp, 0)
    ctx.sync_status()
    return gs, pm, fr


@pytest.mark.parametrize("which", ["slab", "glass"])
def test_photons_match_oracle_light_records(ctx, which):
    sc = _beam_through_slab() if which == "slab" else _glass()
    flags = O.FLAG_FORCE_TRANSMIT if which == "slab" else 0
    guide = None if which == "slab" else S.guide_sphere(sc)
    nb, n = (1, 1 << 15) if which == "slab" else (8, 1 << 15)
    gs = R.GpuScene(ctx, sc)
    pm = R.PhotonMap(ctx, gs, n, RADIUS, 8, n_bins=nb, seed=5, flags=flags, guide=guide)
    ph = pm.export()
    ctx.sync_status()
    _, rec = O.OracleScene(sc).trace_lights(n, 8, nbins=nb, seed=5, flags=flags, guide=guide)
    grazing, sensitive = split_ambiguous(rec["amb"])
    ok = ~grazing & ~sensitive
    np.testing.assert_array_equal(ph["photon"][ok], rec["photon"][ok] != 0)
    dep = ok & ph["photon"]
    assert dep.sum() > 100
    np.testing.assert_array_equal(ph["bin"][dep], rec["bin"][dep])
    # positions and normals at the end of FP32 glass chains: within 1e-4 (relative to max(1, |x|)),
    # the scale at which the splat pixels of the same paths already agree
    scale = 1e-4 * np.maximum(1.0, np.abs(rec["x"][dep]).max(axis=1, keepdims=True))
    assert (np.abs(ph["x"][dep] - rec["x"][dep]) <= scale).all()
    assert (np.abs(ph["n"][dep] - rec["n"][dep]) <= 1e-4).all()
    assert rel_close(ph["beta"][dep], rec["beta"][dep], REL).all()


@pytest.mark.parametrize("which", ["slab", "slab_bins", "glass"])
def test_gather_matches_oracle_with_the_same_photons(ctx, which):
    """The gather kernel against the oracle's density estimate on the GPU's own photons, per camera
    path: signatures of the prefix bit for bit and radiance within 1e-4, away from grazing prefixes and
    from gather points with a photon within FP32_POINT_ERR of the gather sphere."""
    if which.startswith("slab"):
        sc, flags, guide = _beam_through_slab(), O.FLAG_FORCE_TRANSMIT, None
        nb = 4 if which == "slab_bins" else 1
    else:
        sc, flags, guide, nb = _glass(), 0, None, 8
        guide = S.guide_sphere(sc)
    # the slab's photons are dense (r = 0.03 over a uniform beam): 2^15 of them keep the share of
    # gather points with a photon near the sphere small at this margin
    n_light = (1 << 15) if which.startswith("slab") else (1 << 17)
    spp, radius = (2 if which.startswith("slab") else 4), (RADIUS if which.startswith("slab") else 0.1)
    _, pm, fr = _run(ctx, sc, n_light, spp, nb, flags, radius, guide=guide)
    ph = pm.export()
    g = R.path_records_numpy(fr.path_records)
    orc = O.OracleScene(sc)
    gr = orc.trace_gather(spp, 8, nbins=nb, seed=4, flags=flags)
    L, margin = O.local_caustic_gather(gr, {k: ph[k] for k in ("x", "n", "beta", "bin")} | {"photon": ph["photon"]},
                                       radius, n_light, nb)
    grazing = (gr["amb"] != 0)
    ok = ~grazing & (margin * radius > fp32_point_err(sc))
    assert ok.mean() > 0.9
    np.testing.assert_array_equal(g["signature"][ok], gr["signature"][ok])
    assert rel_close(g["L"][ok], L[ok], REL, floor=1e-7).all()
    lit = ok & (L.max(axis=1) > 0)
    assert lit.sum() > 20
    # the accumulator holds each pixel's samples
    acc = g["L"].reshape(sc.camera.height, sc.camera.width, spp, 3).sum(axis=2)
    np.testing.assert_allclose(fr["accum_local_caustic"][..., :3].cpu().numpy(), acc, rtol=1e-6, atol=1e-9)


def test_beam_through_slab_closed_form_on_the_gpu(ctx):
    sc = _beam_through_slab()
    _, _, fr = _run(ctx, sc, 1 << 18, 2, 1, O.FLAG_FORCE_TRANSMIT, RADIUS)
    g = R.path_records_numpy(fr.path_records)
    gr = O.OracleScene(sc).trace_gather(2, 8, seed=4, flags=O.FLAG_FORCE_TRANSMIT)
    rr = np.hypot(gr["x"][:, 0], gr["x"][:, 2])
    inside, outside = rr < R_BEAM - 2 * RADIUS, rr > R_BEAM + 2 * RADIUS
    ratio = g["L"][inside][:, 0] / ((RHO / math.pi) * E0)
    assert abs(ratio.mean() - 1.0) < 4 * ratio.std() / math.sqrt(inside.sum()) + 2e-3
    assert (g["L"][outside] == 0).all()


def test_resolve_local_caustic_buffer_and_mask(ctx):
    sc = _beam_through_slab(24, 24)
    _, _, fr = _run(ctx, sc, 1 << 17, 4, 1, O.FLAG_FORCE_TRANSMIT, RADIUS)
    acc = fr["accum_local_caustic"][..., :3].cpu().numpy().astype(np.float64)
    np.testing.assert_allclose(fr["local_caustic"][..., :3].cpu().numpy(), acc / 4, rtol=1e-6)
    out = O.OracleScene(sc).resolve(np.zeros((24, 24, 3)), None, 4, 0, acc_local=acc)
    yl = out["local_caustic"] @ np.array([0.2126, 0.7152, 0.0722])
    clear = np.abs(yl - 0.25e-3) > 1e-6
    np.testing.assert_array_equal(fr["local_caustic_mask"].cpu().numpy()[clear], out["local_caustic_mask"][clear])
    assert fr["local_caustic_mask"].cpu().numpy().sum() > 50
    np.testing.assert_allclose(fr["rgb"][..., :3].cpu().numpy(), out["rgb"], rtol=1e-5, atol=1e-7)


def test_photon_map_arguments_are_checked(ctx):
    sc = S.ball_on_plane(16, 16)
    gs = R.GpuScene(ctx, sc)
    for bad in (dict(n_paths=0, radius=0.1), dict(n_paths=100, radius=0.0), dict(n_paths=100, radius=float("inf"))):
        with pytest.raises(N.ScError):
            R.PhotonMap(ctx, gs, bad["n_paths"], bad["radius"], 8)
    pm = R.PhotonMap(ctx, gs, 1000, 0.1, 8, n_bins=2)
    with pytest.raises(N.ScError):  # gathering with other bins than the map's
        pm.gather(gs, R.Frame(16, 16), 1, 8, n_bins=1)
    ctx.sync_status()
