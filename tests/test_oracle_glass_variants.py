"""Pins of the oracle's glass variants (paper Sec. III-C varies the glass's colour, roughness and
the spectrum it disperses): Beer-Lambert absorption, sub-bin wavelength jitter and the GGX rough
dielectric, against closed forms, library quadrature and the rough BSDF integrated directly.
No GPU."""
import math

import numpy as np
import pytest

import oracle as O
from paper_2107_11008_gb300 import scenes as S

THICK = 0.4


def _slab(absorption, cauchy_a=1.5, cauchy_b=0.0, roughness=0.0, width=24, height=24):
    """A 12 x 0.4 x 12 m glass slab (top face y = 0.2) under a camera looking down at ~35 degrees;
    environment radiance 1, nothing else: every path through the slab ends in the environment."""
    b = S.SceneBuilder()
    b.add(S.box((-6, -0.5 * THICK, -6), (6, 0.5 * THICK, 6)),
          b.material(S.Material(S.MAT_DIELECTRIC, cauchy_a=cauchy_a, cauchy_b=cauchy_b, absorption=absorption,
                                roughness=roughness)))
    cam = S.Camera((0.3, 3.0, 2.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 30.0, width, height)
    return b.build(cam, env=(1.0, 1.0, 1.0))


def _through_slab(p0, n, eye):
    """Length of the refracted segment inside the slab for primary rays hitting its top at p0: the
    refracted ray starts 1e-4 max(1, |p0|inf) below the face (the self-intersection offset) and
    runs to the bottom face."""
    d = p0 - eye
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    cos_i = np.abs(d[:, 1])
    cos_t = np.sqrt(1.0 - (1.0 - cos_i ** 2) / n ** 2)
    eps = 1e-4 * np.maximum(1.0, np.abs(p0).max(axis=1))
    bottom = -float(O.f32(0.5 * THICK))
    return (p0[:, 1] - eps - bottom) / cos_t


def test_beer_lambert_slab_closed_form():
    """Per path: radiance = exp(-sigma t) per channel, t = the refracted path length inside."""
    sigma = np.array([0.3, 0.9, 1.7])
    sc = _slab(tuple(sigma))
    _, rec = O.OracleScene(sc).trace_camera(spp=4, max_depth=4, flags=O.FLAG_FORCE_TRANSMIT)
    hit = rec["first_tri"] >= 0
    assert hit.all()
    eye = O.f32([0.3, 3.0, 2.0])
    t = _through_slab(rec["p0"], 1.5, eye)
    expect = np.exp(-np.outer(t, O.f32(sigma)))
    np.testing.assert_allclose(rec["L"], expect, rtol=1e-9)
    assert (rec["n_specular"] == 2).all()
    # colourless glass: exactly the environment
    _, rec0 = O.OracleScene(_slab((0.0, 0.0, 0.0))).trace_camera(spp=2, max_depth=4, flags=O.FLAG_FORCE_TRANSMIT)
    np.testing.assert_array_equal(rec0["L"], 1.0)


def _rgb(lam):
    return O.xyz_to_rgb(O.cie_xyz(lam))


def test_jitter_normaliser_matches_library_quadrature():
    from scipy import integrate

    # the fit's lobes change width at their means: integrate piecewise across those kinks
    kinks = [437.0, 442.0, 459.0, 501.1, 530.9, 568.8, 599.8]
    ref = np.array([integrate.quad(lambda l, c=c: _rgb(l)[c], 400.0, 700.0, points=kinks, epsabs=0, epsrel=1e-12,
                                   limit=200)[0] for c in range(3)]) / 300.0
    np.testing.assert_allclose(O.jitter_mean(), ref, rtol=1e-9)


@pytest.mark.parametrize("jitter", [False, True])
def test_dispersion_and_absorption_per_path_wavelength(jitter):
    """A dispersive, coloured slab with 8 bins: each path's radiance is W(lambda) exp(-sigma t(n(lambda)))
    with lambda from its own Philox bin draw u (tag 0, word 2): the bin centre, or 400 + 300 u with
    jitter (W the normalised CIE-fit sRGB there)."""
    sigma = np.array([1.0, 2.0, 3.0])
    A, B, nb, seed = 1.5, 0.02, 8, 7
    sc = _slab(tuple(sigma), cauchy_a=A, cauchy_b=B)
    flags = O.FLAG_FORCE_TRANSMIT | (O.FLAG_WAVELENGTH_JITTER if jitter else 0)
    spp = 4
    _, rec = O.OracleScene(sc).trace_camera(spp=spp, max_depth=4, nbins=nb, seed=seed, flags=flags)
    W, H = sc.camera.width, sc.camera.height
    pix = np.repeat(np.arange(W * H), spp)
    smp = np.tile(np.arange(spp), W * H)
    ctr = np.stack([pix, smp, np.zeros_like(pix), np.zeros_like(pix)], axis=1).astype(np.uint32)
    u = (O.philox(ctr, seed)[:, 2] >> 8).astype(np.float64) * 2.0 ** -24
    b = np.minimum((u * nb).astype(int), nb - 1)
    np.testing.assert_array_equal(rec["bin"], b)
    if jitter:
        lam = 400.0 + 300.0 * u
        w = np.array([_rgb(x) for x in lam]) / O.jitter_mean()
    else:
        lam = 400.0 + (b + 0.5) * 300.0 / nb
        cw, _ = O.spectral_weights(nb)
        w = cw[b]
    n = float(O.f32(A)) + float(O.f32(B)) / (lam * 1e-3) ** 2
    t = _through_slab(rec["p0"], n, O.f32([0.3, 3.0, 2.0]))
    expect = w * np.exp(-t[:, None] * O.f32(sigma)[None, :])
    np.testing.assert_allclose(rec["L"], expect, rtol=1e-9, atol=1e-12)
    if jitter:  # a flat spectrum stays white in expectation
        m = w.mean(axis=0)
        assert np.all(np.abs(m - 1.0) < 4 * w.std(axis=0) / math.sqrt(len(w)))


# ------------------------------------------------------------------------------------------
# Rough dielectric (Walter, Marschner, Li, Torrance, EGSR 2007; GGX)
# ------------------------------------------------------------------------------------------

def _ggx_d(cos_m, alpha):
    """GGX normal distribution (Walter et al. eq. 33), zero for back-facing m."""
    c2 = cos_m * cos_m
    tan2 = (1.0 - c2) / np.maximum(c2, 1e-300)
    d = alpha ** 2 / (math.pi * c2 * c2 * (alpha ** 2 + tan2) ** 2)
    return np.where(cos_m > 0, d, 0.0)


def _ggx_g1(v_dot_n, v_dot_m, alpha):
    """Smith masking of GGX (eq. 34) with its sign condition chi+(v.m / v.n)."""
    c2 = v_dot_n ** 2
    tan2 = (1.0 - c2) / np.maximum(c2, 1e-300)
    g = 2.0 / (1.0 + np.sqrt(1.0 + alpha ** 2 * tan2))
    return np.where(v_dot_m * v_dot_n > 0, g, 0.0)


def _fresnel(c, eta_i, eta_t):
    """Unpolarised dielectric Fresnel reflectance for cosine c on the incident side (TIR -> 1)."""
    s2 = (eta_i / eta_t) ** 2 * (1.0 - c * c)
    ct = np.sqrt(np.maximum(0.0, 1.0 - s2))
    rs = (eta_i * c - eta_t * ct) / (eta_i * c + eta_t * ct)
    rp = (eta_i * ct - eta_t * c) / (eta_i * ct + eta_t * c)
    return np.where(s2 >= 1.0, 1.0, 0.5 * (rs * rs + rp * rp))


def _albedos_by_quadrature(i, eta_i, eta_t, alpha, n_th=600, n_ph=600):
    """Reflected and transmitted directional albedo of the rough dielectric BSDF, integrating
    f |o.n| over each hemisphere (Walter et al. eqs. 20 and 21 with h_r = unit(i + o),
    h_t = -unit(eta_i i + eta_t o)); n = +z, i on the +z side."""
    x, wx = np.polynomial.legendre.leggauss(n_th)
    phi = (np.arange(n_ph) + 0.5) * 2 * math.pi / n_ph
    out = []
    for side in (1.0, -1.0):
        ct = 0.5 * (x + 1.0)  # cos theta_o in (0, 1)
        wt = 0.5 * wx
        CT, PH = np.meshgrid(ct, phi, indexing="ij")
        ST = np.sqrt(1.0 - CT ** 2)
        o = np.stack([ST * np.cos(PH), ST * np.sin(PH), side * CT], axis=-1)
        on = o[..., 2]
        i_n = i[2]
        if side > 0:
            h = i[None, None, :] + o
            h /= np.linalg.norm(h, axis=-1, keepdims=True)
            ih = h @ i
            f = (_fresnel(ih, eta_i, eta_t) * _ggx_g1(i_n, ih, alpha) * _ggx_g1(on, (o * h).sum(-1), alpha) *
                 _ggx_d(h[..., 2], alpha) / (4 * abs(i_n) * np.abs(on)))
        else:
            h = -(eta_i * i[None, None, :] + eta_t * o)
            h /= np.linalg.norm(h, axis=-1, keepdims=True)
            h *= np.sign(h[..., 2])[..., None]  # the microfacet normal on the incident side
            ih, oh = h @ i, (o * h).sum(-1)
            den = (eta_i * ih + eta_t * oh) ** 2
            f = (np.abs(ih) * np.abs(oh) / (abs(i_n) * np.abs(on)) * eta_t ** 2 * (1 - _fresnel(ih, eta_i, eta_t)) *
                 _ggx_g1(i_n, ih, alpha) * _ggx_g1(on, oh, alpha) * _ggx_d(h[..., 2], alpha) / den)
        integrand = f * np.abs(on)
        out.append(float((integrand * wt[:, None]).sum() * (2 * math.pi / n_ph)))
    return out


def test_ggx_distribution_is_normalised():
    x, wx = np.polynomial.legendre.leggauss(2000)
    for alpha in (0.1, 0.3, 0.7):
        c = 0.5 * (x + 1.0)
        assert abs(float((_ggx_d(c, alpha) * c * 0.5 * wx).sum() * 2 * math.pi) - 1.0) < 1e-6


@pytest.mark.parametrize("alpha,theta_deg,entering", [(0.3, 30.0, True), (0.6, 55.0, True), (0.3, 20.0, False)])
def test_rough_scatter_weights_integrate_the_walter_bsdf(alpha, theta_deg, entering):
    """E[weight * 1{reflect}] and E[weight * 1{refract}] over the sampler's draws equal the reflected and
    transmitted albedos of the rough BSDF integrated directly (4 standard errors)."""
    n_glass = 1.5
    th = math.radians(theta_deg)
    rng = np.random.default_rng(1)
    ng = np.array([0.0, 0.0, 1.0]) if entering else np.array([0.0, 0.0, -1.0])
    d = np.array([math.sin(th), 0.0, -math.cos(th)])  # travelling toward the surface from +z
    eta_i, eta_t = (1.0, n_glass) if entering else (n_glass, 1.0)
    m = 160
    g1, g2 = np.meshgrid((np.arange(m) + rng.random()) / m, (np.arange(m) + rng.random()) / m, indexing="ij")
    wr, wt = [], []
    for a, b in zip(g1.ravel(), g2.ravel()):
        ok, o, w, refl = O.rough_scatter(d, ng, ng, n_glass, alpha, rng.random(), a, b)
        w = w if ok else 0.0
        wr.append(w if (ok and refl) else 0.0)
        wt.append(w if (ok and not refl) else 0.0)
    wr, wt = np.array(wr), np.array(wt)
    rho_r, rho_t = _albedos_by_quadrature(-d, eta_i, eta_t, alpha)
    for est, ref in ((wr, rho_r), (wt, rho_t)):
        se = est.std() / math.sqrt(len(est))
        assert abs(est.mean() - ref) <= 4 * se + 2e-4, (est.mean(), ref, se)
    assert rho_r + rho_t < 1.0 + 1e-6  # the single-scattering model loses, never gains, energy


def test_rough_scatter_tends_to_the_smooth_dielectric():
    """alpha -> 0: Snell / mirror directions and weight 1."""
    for th in (10.0, 40.0, 70.0):
        t = math.radians(th)
        d = np.array([math.sin(t), 0.0, -math.cos(t)])
        n = np.array([0.0, 0.0, 1.0])
        for u0 in (0.999, 0.0):
            ok, o, w, refl = O.rough_scatter(d, n, n, 1.5, 1e-7, u0, 0.37, 0.81)
            assert ok
            if refl:
                np.testing.assert_allclose(o, d - 2 * d.dot(n) * n, atol=1e-6)
            else:
                np.testing.assert_allclose(o, O.refract(d, n, 1 / 1.5), atol=1e-6)
            assert abs(w - 1.0) < 1e-6
