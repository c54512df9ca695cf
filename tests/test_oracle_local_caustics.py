"""Pins of the local-caustic oracle (caustics seen through glass, Sec. III-D "Local & Non-local
Caustics Mask"): photons of light paths that passed glass, gathered at the first diffuse vertex of
camera paths that passed glass.  A collimated beam of irradiance E0 through a glass slab lights a
disk of the floor uniformly; a camera looking at the floor through the slab must then see
(rho / pi) E0 there and nothing outside.  No GPU."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2107_11008_gb300 import scenes as S

E0, RHO, R_BEAM, RADIUS = 3.0, 0.5, 0.6, 0.03


def _beam_through_slab(width=32, height=32, nbins=1, side_light=False):
    b = S.SceneBuilder()
    b.add(S.quad((-10, 0, -10), (0, 0, 20), (20, 0, 0)), b.material(S.Material(S.MAT_DIFFUSE, albedo=(RHO,) * 3)))
    b.add(S.box((-3, 0.3, -3), (3, 0.5, 3)), b.material(S.Material(S.MAT_DIELECTRIC, cauchy_a=1.5)))
    b.lights.append(S.Light(S.LIGHT_DISK, (0.0, 2.0, 0.0), (0.0, -1.0, 0.0), power=(E0,) * 3, radius=R_BEAM))
    if side_light:  # a second beam that reaches the floor without passing glass
        b.lights.append(S.Light(S.LIGHT_DISK, (4.5, 2.0, 0.0), (0.0, -1.0, 0.0), power=(E0,) * 3, radius=0.3))
    cam = S.Camera((0.0, 3.0, 0.0), (0.0, 0.0, 0.0), (0.0, 0.0, -1.0), 30.0, width, height)
    return b.build(cam)


def _local(sc, nbins, n_light=1 << 18, spp=2, seed=4):
    o = O.OracleScene(sc)
    g = o.trace_gather(spp, 8, nbins=nbins, seed=seed, flags=O.FLAG_FORCE_TRANSMIT)
    _, ph = o.trace_lights(n_light, 8, nbins=nbins, seed=seed + 1, flags=O.FLAG_FORCE_TRANSMIT)
    L, margin = O.local_caustic_gather(g, ph, RADIUS, n_light, nbins)
    return g, ph, L, margin


@pytest.mark.parametrize("nbins", [1, 4])
def test_uniform_beam_through_slab_gives_rho_over_pi_e0(nbins):
    sc = _beam_through_slab(nbins=nbins)
    g, ph, L, _ = _local(sc, nbins)
    assert (g["valid"] == 1).all() and (g["n_specular"] == 2).all()  # every pixel sees the floor through glass
    rr = np.hypot(g["x"][:, 0], g["x"][:, 2])
    w, _ = O.spectral_weights(nbins)
    expect = w[g["bin"]] * (RHO / math.pi) * E0  # per channel, this path's bin weight
    inside = rr < R_BEAM - 2 * RADIUS
    outside = rr > R_BEAM + 2 * RADIUS
    assert inside.sum() > 300 and outside.sum() > 100
    ratio = L[inside] / expect[inside]
    m, se = ratio.mean(axis=0), ratio.std(axis=0) / math.sqrt(inside.sum())
    assert np.all(np.abs(m - 1.0) < 4 * se + 2e-3), (m, se)
    assert (L[outside] == 0).all()
    # photons: every light path passed the slab and was deposited
    assert (ph["photon"] == 1).all()


def test_only_photons_that_passed_glass_are_deposited():
    sc = _beam_through_slab(side_light=True)
    # with direct splats on, paths without glass also reach the receiver code: still no photon
    _, ph = O.OracleScene(sc).trace_lights(1 << 14, 8, seed=9, flags=O.FLAG_FORCE_TRANSMIT | O.FLAG_SPLAT_DIRECT)
    direct = ph["n_specular"] == 0
    assert direct.mean() > 0.2
    assert (ph["photon"][direct] == 0).all() and (ph["photon"][~direct] == 1).all()
    # the photon's throughput is the beam's flux per path: pi R^2 E0 x 2 lights
    np.testing.assert_allclose(ph["beta"][~direct], math.pi * R_BEAM ** 2 * E0 * 2, rtol=1e-6)


def test_local_caustic_mask_marks_glass_pixels_over_the_caustic():
    sc = _beam_through_slab(width=24, height=24)
    g, _, L, _ = _local(sc, 1, spp=4)
    acc_local = L.reshape(24, 24, 4, 3).sum(axis=2)
    out = O.OracleScene(sc).resolve(np.zeros((24, 24, 3)), None, 4, 0, acc_local=acc_local)
    rr = np.hypot(g["x"][:, 0], g["x"][:, 2]).reshape(24, 24, 4).mean(axis=2)
    np.testing.assert_allclose(out["local_caustic"], acc_local / 4)
    np.testing.assert_allclose(out["rgb"], out["direct"] + out["caustic"] + out["local_caustic"])
    assert (out["mask"] == 1).all()  # the slab covers the view
    assert (out["local_caustic_mask"][rr < R_BEAM - 0.1] == 1).all()
    assert (out["local_caustic_mask"][rr > R_BEAM + 0.1] == 0).all()
    assert (out["caustic_mask"] == 0).all()  # non-local caustics are those on non-glass pixels
