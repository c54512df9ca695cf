"""Python side of the FP64 CPU oracle (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline leg import this
package.  The product path (``paper_2107_11008_gb300``) never does.  The oracle is compiled
from ``oracle/sc_oracle.c`` with gcc; it shares nothing with the CUDA library except the scene
arrays produced by ``paper_2107_11008_gb300.scenes``.
"""
from __future__ import annotations

import ctypes as C
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sc_oracle.c")
_LIB = os.path.join(_HERE, "libsc_oracle.so")

FLAG_FORCE_TRANSMIT = 1
FLAG_SPLAT_DIRECT = 2
FLAG_EMITTER_AFTER_DS = 4
FLAG_WAVELENGTH_JITTER = 8

AMB_NAMES = {1: "edge", 2: "tgap", 4: "graze", 8: "fresnel", 16: "tir", 32: "shadow", 64: "splat",
             128: "checker", 256: "fixup", 512: "sensitive"}


def build(force: bool = False) -> str:
    """Compile the oracle shared library (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-D_GNU_SOURCE", "-fPIC", "-shared", "-fno-fast-math",
                               "-ffp-contract=off", "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB)
    return _LIB


class Tolerances(C.Structure):
    """Base tolerances of the ambiguity classifier; each specular event before a decision
    multiplies its tolerance by ``growth`` (FP32 error compounds along glass chains)."""
    _fields_ = [("pos", C.c_double), ("t", C.c_double), ("cosg", C.c_double), ("fres", C.c_double),
                ("tir", C.c_double), ("px", C.c_double), ("growth", C.c_double), ("sens_delta", C.c_double),
                ("sens_rel", C.c_double)]


# sens_delta: every recorded path is re-traced twice with its ray nudged by +-1e-6 (relative) after
# each scattering event; a path whose signature or radiance (beyond sens_rel) moves is flagged
# "sensitive" -- float32 cannot be expected to follow it decision for decision.
DEFAULT_TOL = dict(pos=2e-5, t=1e-5, cosg=1e-4, fres=1e-4, tir=1e-5, px=1e-4, growth=1.0, sens_delta=1e-6,
                   sens_rel=5e-5)


def default_tol(**kw) -> Tolerances:
    d = dict(DEFAULT_TOL)
    d.update(kw)
    return Tolerances(**d)


class CamParams(C.Structure):
    _fields_ = [("spp", C.c_int32), ("sample_offset", C.c_int32), ("max_depth", C.c_int32), ("nbins", C.c_int32),
                ("seed", C.c_uint64), ("scene_index", C.c_int32), ("flags", C.c_int32),
                ("x0", C.c_int32), ("x1", C.c_int32), ("y0", C.c_int32), ("y1", C.c_int32),
                ("n_threads", C.c_int32), ("brute", C.c_int32), ("tol", Tolerances)]


class PathRec(C.Structure):
    _fields_ = [("L", C.c_double * 3), ("p0", C.c_double * 3), ("first_tri", C.c_int32), ("n_queries", C.c_int32),
                ("signature", C.c_uint32), ("amb", C.c_int32), ("bin", C.c_int32), ("n_specular", C.c_int32),
                ("min_ratio", C.c_double), ("ratio_nspec", C.c_int32), ("ratio_kind", C.c_int32),
                ("kmin", C.c_double * 9), ("knspec", C.c_int32 * 9), ("pad2", C.c_int32)]


class LightParams(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("path_offset", C.c_int64), ("max_depth", C.c_int32), ("nbins", C.c_int32),
                ("seed", C.c_uint64), ("scene_index", C.c_int32), ("flags", C.c_int32),
                ("n_threads", C.c_int32), ("brute", C.c_int32), ("tol", Tolerances), ("guide", C.c_double * 4)]


class LightRec(C.Structure):
    _fields_ = [("C", C.c_double * 3), ("x", C.c_double * 3), ("pixel", C.c_int32), ("amb", C.c_int32),
                ("signature", C.c_uint32), ("n_specular", C.c_int32), ("bin", C.c_int32), ("pad", C.c_int32),
                ("min_ratio", C.c_double), ("ratio_nspec", C.c_int32), ("ratio_kind", C.c_int32),
                ("kmin", C.c_double * 9), ("knspec", C.c_int32 * 9), ("pad2", C.c_int32),
                ("beta", C.c_double * 3), ("n", C.c_double * 3), ("photon", C.c_int32), ("pad3", C.c_int32)]


class GatherRec(C.Structure):
    _fields_ = [("x", C.c_double * 3), ("n", C.c_double * 3), ("w", C.c_double * 3), ("valid", C.c_int32),
                ("bin", C.c_int32), ("amb", C.c_int32), ("n_specular", C.c_int32), ("signature", C.c_uint32),
                ("pad", C.c_uint32)]


class ResolveParams(C.Structure):
    _fields_ = [("spp_total", C.c_double), ("light_paths_total", C.c_double), ("depth_range", C.c_double),
                ("tau_rel", C.c_double), ("brute", C.c_int32), ("pad", C.c_int32)]


class PixelOut(C.Structure):
    _fields_ = [("rgb", C.c_double * 3), ("direct", C.c_double * 3), ("caustic", C.c_double * 3),
                ("depth", C.c_double), ("depth_norm", C.c_double), ("n_world", C.c_double * 3),
                ("n_cam", C.c_double * 3), ("albedo", C.c_double * 3), ("instance", C.c_int32), ("tri", C.c_int32),
                ("mask", C.c_int32), ("caustic_mask", C.c_int32), ("local_caustic_mask", C.c_int32),
                ("amb", C.c_int32), ("local_caustic", C.c_double * 3)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(build())
        P = C.POINTER
        L.orc_philox.argtypes = [P(C.c_uint32), C.c_uint64, C.c_int64, P(C.c_uint32)]
        L.orc_spectral_weights.argtypes = [C.c_int, P(C.c_double), P(C.c_double)]
        L.orc_cie_xyz.argtypes = [C.c_double, P(C.c_double)]
        L.orc_xyz_to_rgb.argtypes = [P(C.c_double), P(C.c_double)]
        L.orc_fresnel.argtypes = [C.c_double, C.c_double, C.c_double]
        L.orc_fresnel.restype = C.c_double
        L.orc_refract.argtypes = [P(C.c_double), P(C.c_double), C.c_double, P(C.c_double)]
        L.orc_jitter_mean.argtypes = [P(C.c_double)]
        L.orc_rough_scatter.argtypes = [P(C.c_double), P(C.c_double), P(C.c_double), C.c_double, C.c_double,
                                        C.c_double, C.c_double, C.c_double, C.c_int, P(C.c_double), P(C.c_double),
                                        P(C.c_int)]
        L.orc_rough_scatter.restype = C.c_int
        L.orc_scene_create.argtypes = [C.c_int, P(C.c_float), P(C.c_float), P(C.c_float), C.c_int, P(C.c_int),
                                       P(C.c_int), C.c_int, P(C.c_int), C.c_int, P(C.c_double), C.c_int,
                                       P(C.c_double), P(C.c_double), C.c_int, C.c_int, P(C.c_double)]
        L.orc_scene_create.restype = C.c_void_p
        L.orc_scene_destroy.argtypes = [C.c_void_p]
        L.orc_intersect.argtypes = [C.c_void_p, C.c_int64, P(C.c_double), C.c_int, P(C.c_double), P(C.c_int),
                                    P(C.c_double), P(C.c_int)]
        L.orc_occluded.argtypes = [C.c_void_p, C.c_int64, P(C.c_double), P(C.c_double), C.c_int, P(C.c_int),
                                   P(C.c_int)]
        L.orc_trace_camera.argtypes = [C.c_void_p, P(CamParams), P(C.c_double), P(PathRec)]
        L.orc_trace_lights.argtypes = [C.c_void_p, P(LightParams), P(C.c_double), P(LightRec)]
        L.orc_resolve.argtypes = [C.c_void_p, P(ResolveParams), P(C.c_double), P(C.c_double), P(C.c_double),
                                  P(PixelOut)]
        L.orc_sizes.argtypes = [P(C.c_int)]
        sizes = (C.c_int * 8)()
        L.orc_sizes(sizes)
        want = [C.sizeof(t) for t in (CamParams, PathRec, LightParams, LightRec, ResolveParams, PixelOut, Tolerances,
                                      GatherRec)]
        if list(sizes[:8]) != want:
            raise RuntimeError(f"oracle struct layout mismatch: C {list(sizes[:8])} vs Python {want}")
        L.orc_trace_gather.argtypes = [C.c_void_p, P(CamParams), P(GatherRec)]
        _lib = L
    return _lib


def _p(a, ctype):
    return a.ctypes.data_as(C.POINTER(ctype)) if a is not None else None


def f32(x) -> np.ndarray:
    """Round inputs through float32 so the oracle sees exactly what the FP32 library sees."""
    return np.asarray(x, dtype=np.float32).astype(np.float64)


class OracleScene:
    """An FP64 copy of a ``scenes.Scene`` with the oracle's own median-split BVH."""

    def __init__(self, scene):
        self.scene = scene
        s = scene
        self._keep = [np.ascontiguousarray(s.positions, np.float32), np.ascontiguousarray(s.normals, np.float32),
                      np.ascontiguousarray(s.uvs, np.float32), np.ascontiguousarray(s.indices, np.int32),
                      np.ascontiguousarray(s.tri_object, np.int32), np.ascontiguousarray(s.object_material, np.int32),
                      np.ascontiguousarray(f32(s.materials_flat())), np.ascontiguousarray(f32(s.lights_flat())),
                      np.ascontiguousarray(f32(s.camera.flat())), np.ascontiguousarray(f32(s.env))]
        pos, nrm, uv, idx, obj, om, mats, lights, cam, env = self._keep
        self.W, self.H = s.camera.width, s.camera.height
        self.h = lib().orc_scene_create(pos.shape[0], _p(pos, C.c_float), _p(nrm, C.c_float), _p(uv, C.c_float),
                                        idx.shape[0], _p(idx, C.c_int), _p(obj, C.c_int), om.shape[0],
                                        _p(om, C.c_int), mats.shape[0], _p(mats, C.c_double), lights.shape[0],
                                        _p(lights, C.c_double), _p(cam, C.c_double), self.W, self.H,
                                        _p(env, C.c_double))

    def __del__(self):
        if getattr(self, "h", None):
            lib().orc_scene_destroy(self.h)
            self.h = None

    # -- queries ------------------------------------------------------------------------------
    def intersect(self, origins, dirs, brute=False):
        rays = np.ascontiguousarray(np.concatenate([np.asarray(origins, np.float64), np.asarray(dirs, np.float64)], 1))
        n = rays.shape[0]
        t = np.empty(n)
        tri = np.empty(n, np.int32)
        b = np.empty((n, 2))
        amb = np.empty(n, np.int32)
        lib().orc_intersect(self.h, n, _p(rays, C.c_double), int(brute), _p(t, C.c_double), _p(tri, C.c_int),
                            _p(b, C.c_double), _p(amb, C.c_int))
        return t, tri, b, amb

    def occluded(self, origins, dirs, tmax, brute=False):
        rays = np.ascontiguousarray(np.concatenate([np.asarray(origins, np.float64), np.asarray(dirs, np.float64)], 1))
        n = rays.shape[0]
        tm = np.ascontiguousarray(np.broadcast_to(np.asarray(tmax, np.float64), (n,)))
        occ = np.empty(n, np.int32)
        amb = np.empty(n, np.int32)
        lib().orc_occluded(self.h, n, _p(rays, C.c_double), _p(tm, C.c_double), int(brute), _p(occ, C.c_int),
                           _p(amb, C.c_int))
        return occ, amb

    # -- estimators ---------------------------------------------------------------------------
    def trace_camera(self, spp, max_depth, nbins=1, seed=0, sample_offset=0, scene_index=0, flags=0, window=None,
                     records=True, accum=None, n_threads=0, brute=False, tol=None):
        x0, x1, y0, y1 = window if window is not None else (0, self.W, 0, self.H)
        tol = tol or default_tol()
        if not records:
            tol.sens_delta = 0.0  # the re-traces only classify recorded paths
        P = CamParams(spp, sample_offset, max_depth, nbins, seed, scene_index, flags, x0, x1, y0, y1, n_threads,
                      int(brute), tol)
        if accum is None:
            accum = np.zeros((self.H, self.W, 3))
        recs = (PathRec * ((y1 - y0) * (x1 - x0) * spp))() if records else None
        lib().orc_trace_camera(self.h, C.byref(P), _p(accum, C.c_double), recs)
        return accum, (records_to_numpy(recs, PathRec) if records else None)

    def trace_lights(self, n_paths, max_depth, nbins=1, seed=0, path_offset=0, scene_index=0, flags=0,
                     records=True, accum=None, n_threads=0, brute=False, tol=None, guide=None):
        """guide: (cx, cy, cz, r) sphere around the dielectric triangles for guided emission, or None."""
        tol = tol or default_tol()
        if not records:
            tol.sens_delta = 0.0
        g = (C.c_double * 4)(*(guide if guide is not None else (0.0, 0.0, 0.0, 0.0)))
        P = LightParams(n_paths, path_offset, max_depth, nbins, seed, scene_index, flags, n_threads, int(brute), tol, g)
        if accum is None:
            accum = np.zeros((self.H, self.W, 3))
        recs = (LightRec * n_paths)() if records else None
        lib().orc_trace_lights(self.h, C.byref(P), _p(accum, C.c_double), recs)
        return accum, (records_to_numpy(recs, LightRec) if records else None)

    def trace_gather(self, spp, max_depth, nbins=1, seed=0, sample_offset=0, scene_index=0, flags=0, window=None,
                     brute=False):
        """Gather points of the local-caustic estimate: per (pixel, sample) of the window, the first
        diffuse vertex of the camera path's prefix if reached through glass (valid), its normal, bin
        and camera-side weight beta * albedo / pi * W(lambda)."""
        x0, x1, y0, y1 = window if window is not None else (0, self.W, 0, self.H)
        tol = default_tol()
        tol.sens_delta = 0.0
        P = CamParams(spp, sample_offset, max_depth, nbins, seed, scene_index, flags, x0, x1, y0, y1, 1, int(brute), tol)
        recs = (GatherRec * ((y1 - y0) * (x1 - x0) * spp))()
        lib().orc_trace_gather(self.h, C.byref(P), recs)
        return records_to_numpy(recs, GatherRec)

    def resolve(self, acc_cam, acc_caus, spp_total, light_paths_total, depth_range=10.0, tau_rel=0.25, brute=False,
                acc_local=None):
        P = ResolveParams(float(spp_total), float(light_paths_total), depth_range, tau_rel, int(brute), 0)
        out = (PixelOut * (self.W * self.H))()
        a = None if acc_cam is None else np.ascontiguousarray(acc_cam, np.float64)
        b = None if acc_caus is None else np.ascontiguousarray(acc_caus, np.float64)
        c = None if acc_local is None else np.ascontiguousarray(acc_local, np.float64)
        lib().orc_resolve(self.h, C.byref(P), _p(a, C.c_double), _p(b, C.c_double), _p(c, C.c_double), out)
        r = records_to_numpy(out, PixelOut)
        return {k: v.reshape((self.H, self.W) + v.shape[1:]) for k, v in r.items()}


def records_to_numpy(arr, struct) -> dict:
    """Column view of a ctypes record array as a dict of numpy arrays."""
    n = len(arr)
    dt = np.dtype({"names": [f[0] for f in struct._fields_],
                   "formats": [_np_fmt(f[1]) for f in struct._fields_],
                   "offsets": [getattr(struct, f[0]).offset for f in struct._fields_],
                   "itemsize": C.sizeof(struct)})
    buf = np.frombuffer(arr, dtype=dt, count=n)
    return {name: np.array(buf[name]) for name in dt.names}


def _np_fmt(t):
    if hasattr(t, "_length_"):
        return (_np_fmt(t._type_), (t._length_,))
    return {C.c_double: np.float64, C.c_float: np.float32, C.c_int32: np.int32, C.c_uint32: np.uint32,
            C.c_int64: np.int64, C.c_uint64: np.uint64}[t]


def local_caustic_gather(gather: dict, photons: dict, radius: float, n_light_paths: int, nbins: int):
    """Photon density estimate at the gather points (Jensen's photon map with a constant kernel):
    L = w * B * sum(beta_i) / (N_L * pi * r^2) over the photons i of the gather point's bin within
    distance r whose normal faces the same side (n_i . n > 0); B = bins (each photon's bin has
    probability 1/B), N_L = light paths traced.  gather: trace_gather records; photons: trace_lights
    records.  Returns (L [n, 3], margin [n]): margin = the smallest | |x_i - x| - r | / r over the
    candidate photons, small where an FP32 evaluation may count a photon differently."""
    from scipy.spatial import cKDTree

    have = photons["photon"] != 0
    px, pn, pb, pbin = photons["x"][have], photons["n"][have], photons["beta"][have], photons["bin"][have]
    n = len(gather["valid"])
    L = np.zeros((n, 3))
    margin = np.full(n, np.inf)
    if len(px) == 0:
        return L, margin
    tree = cKDTree(px)
    valid = np.flatnonzero(gather["valid"] != 0)
    lists = tree.query_ball_point(gather["x"][valid], r=radius * (1.0 + 1e-3))
    norm = max(nbins, 1) / (n_light_paths * math.pi * radius * radius)
    for i, cand in zip(valid, lists):
        if not cand:
            continue
        cand = np.asarray(cand)
        dist = np.linalg.norm(px[cand] - gather["x"][i], axis=1)
        margin[i] = float(np.min(np.abs(dist - radius)) / radius)
        sel = cand[(dist < radius) & (pbin[cand] == gather["bin"][i]) & (pn[cand] @ gather["n"][i] > 0)]
        if len(sel):
            L[i] = gather["w"][i] * pb[sel].sum(axis=0) * norm
    return L, margin


def philox(counters: np.ndarray, key: int) -> np.ndarray:
    c = np.ascontiguousarray(counters, dtype=np.uint32).reshape(-1, 4)
    out = np.empty_like(c)
    lib().orc_philox(_p(c, C.c_uint32), C.c_uint64(key), c.shape[0], _p(out, C.c_uint32))
    return out


def spectral_weights(nbins: int):
    w = np.empty((max(nbins, 1), 3))
    lam = np.empty(max(nbins, 1))
    lib().orc_spectral_weights(nbins, _p(w, C.c_double), _p(lam, C.c_double))
    return w, lam


def cie_xyz(lam: float) -> np.ndarray:
    out = np.empty(3)
    lib().orc_cie_xyz(lam, _p(out, C.c_double))
    return out


def xyz_to_rgb(xyz) -> np.ndarray:
    a = np.ascontiguousarray(xyz, np.float64)
    out = np.empty(3)
    lib().orc_xyz_to_rgb(_p(a, C.c_double), _p(out, C.c_double))
    return out


def jitter_mean() -> np.ndarray:
    """Mean linear sRGB of the CIE fit over 400-700 nm (the weight normaliser of wavelength jitter)."""
    out = np.empty(3)
    lib().orc_jitter_mean(_p(out, C.c_double))
    return out


def rough_scatter(d, ns, ng, n_lambda, alpha, u0, u1, u2, flags=0):
    """One rough-dielectric scatter: (ok, new direction, weight, reflected)."""
    d, ns, ng = (np.ascontiguousarray(v, np.float64) for v in (d, ns, ng))
    out = np.empty(3)
    w = C.c_double()
    refl = C.c_int()
    ok = lib().orc_rough_scatter(_p(d, C.c_double), _p(ns, C.c_double), _p(ng, C.c_double), n_lambda, alpha, u0, u1,
                                 u2, flags, _p(out, C.c_double), C.byref(w), C.byref(refl))
    return bool(ok), out, w.value, bool(refl.value)


def fresnel(cos_i: float, n_i: float, n_t: float) -> float:
    return lib().orc_fresnel(cos_i, n_i, n_t)


def refract(d, n, eta):
    d = np.ascontiguousarray(d, np.float64)
    n = np.ascontiguousarray(n, np.float64)
    out = np.empty(3)
    ok = lib().orc_refract(_p(d, C.c_double), _p(n, C.c_double), eta, _p(out, C.c_double))
    return out if ok else None
