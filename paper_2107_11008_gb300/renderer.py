"""Python-side handles for the C ABI: a context on a torch stream, scenes built from
``scenes.Scene`` and frames whose buffers are torch tensors.

This is marshalling only: building the BVH, tracing and resolving all happen in the CUDA
library.  PyTorch provides device memory (its caching allocator backs the library's scratch)
and streams.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import native as N
from .scenes import Scene


class Context:
    """An ``sc_ctx`` bound to one CUDA device and stream; library scratch comes from torch."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None, torch_allocator: bool = True):
        if not torch.cuda.is_available():
            raise RuntimeError("supercaustics needs a CUDA device")
        self.device = device
        self.stream = stream if stream is not None else torch.cuda.current_stream(device)
        self._alloc_cb = self._free_cb = None
        if torch_allocator:
            dev, st = device, self.stream

            def _alloc(nbytes, _user):
                try:
                    return torch.cuda.caching_allocator_alloc(int(nbytes), dev, st)
                except Exception:  # noqa: BLE001 - an OOM is reported to the library as NULL
                    return None

            def _free(ptr, _user):
                if ptr:
                    torch.cuda.caching_allocator_delete(ptr)

            self._alloc_cb, self._free_cb = N.ALLOC_FN(_alloc), N.FREE_FN(_free)
        self.handle = N.sc_create(device, self.stream.cuda_stream, self._alloc_cb, self._free_cb, None)

    def sync_status(self):
        N.sc_sync_status(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            N.sc_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def _materials(scene: Scene):
    arr = (N.sc_material * max(1, len(scene.materials)))()
    for i, m in enumerate(scene.materials):
        a = arr[i]
        a.kind = m.kind
        a.albedo[:] = [float(x) for x in m.albedo]
        a.albedo2[:] = [float(x) for x in m.albedo2]
        a.checker_scale = m.checker_scale
        a.cauchy_a, a.cauchy_b = m.cauchy_a, m.cauchy_b
        a.emission[:] = [float(x) for x in m.emission]
        a.absorption[:] = [float(x) for x in getattr(m, "absorption", (0.0, 0.0, 0.0))]
        a.roughness = float(getattr(m, "roughness", 0.0))
    return arr


def _lights(scene: Scene):
    arr = (N.sc_light * max(1, len(scene.lights)))()
    for i, l in enumerate(scene.lights):
        a = arr[i]
        a.kind = l.kind
        a.p[:], a.u[:], a.v[:] = ([float(x) for x in l.p], [float(x) for x in l.u], [float(x) for x in l.v])
        a.power[:] = [float(x) for x in l.power]
        a.radius = l.radius
    return arr


def camera_struct(cam) -> N.sc_camera:
    c = N.sc_camera()
    c.eye[:], c.look[:], c.up[:] = ([float(x) for x in cam.eye], [float(x) for x in cam.look],
                                    [float(x) for x in cam.up])
    c.vfov_deg = cam.vfov_deg
    c.width, c.height = cam.width, cam.height
    return c


class SceneArrays:
    """The geometry of a ``Scene`` as torch tensors (host or device) plus the small host tables."""

    def __init__(self, scene: Scene, device: str | torch.device = "cpu"):
        self.scene = scene
        self.positions = torch.from_numpy(np.ascontiguousarray(scene.positions, np.float32)).to(device)
        self.normals = torch.from_numpy(np.ascontiguousarray(scene.normals, np.float32)).to(device)
        self.uvs = torch.from_numpy(np.ascontiguousarray(scene.uvs, np.float32)).to(device)
        self.indices = torch.from_numpy(np.ascontiguousarray(scene.indices, np.int32)).to(device)
        self.tri_object = torch.from_numpy(np.ascontiguousarray(scene.tri_object, np.int32)).to(device)
        self.object_material = np.ascontiguousarray(scene.object_material, np.int32)
        self.mats = _materials(scene)
        self.lights = _lights(scene)

    @property
    def on_device(self) -> bool:
        return self.positions.is_cuda

    def nbytes(self) -> int:
        return sum(t.numel() * t.element_size() for t in (self.positions, self.normals, self.uvs, self.indices,
                                                          self.tri_object))

    def desc(self) -> N.sc_scene_desc:
        s = self.scene
        d = N.sc_scene_desc()
        d.n_verts = int(self.positions.shape[0])
        d.n_tris = int(self.indices.shape[0])
        d.positions = self.positions.data_ptr()
        d.normals = self.normals.data_ptr()
        d.uvs = self.uvs.data_ptr()
        d.indices = self.indices.data_ptr()
        d.tri_object = self.tri_object.data_ptr()
        d.n_objects = int(self.object_material.shape[0])
        d.object_material = self.object_material.ctypes.data
        d.n_materials = len(s.materials)
        d.materials = C.cast(self.mats, C.POINTER(N.sc_material))
        d.n_lights = len(s.lights)
        d.lights = C.cast(self.lights, C.POINTER(N.sc_light))
        d.env[:] = [float(x) for x in s.env]
        d.camera = camera_struct(s.camera)
        d.geometry_on_device = 1 if self.on_device else 0
        return d


class GpuScene:
    """A scene built on the device (LBVH) by ``sc_build_scene``."""

    def __init__(self, ctx: Context, scene: Scene | SceneArrays):
        self.ctx = ctx
        self.arrays = scene if isinstance(scene, SceneArrays) else SceneArrays(scene)
        self.scene = self.arrays.scene
        self.width, self.height = self.scene.camera.width, self.scene.camera.height
        desc = self.arrays.desc()
        self.handle = N.sc_build_scene(ctx.handle, desc)

    def info(self) -> N.sc_scene_info:
        return N.sc_scene_get_info(self.handle)

    def export_bvh(self):
        info = self.info()
        nodes = np.empty((info.n_nodes, 16), np.float32)
        tris = np.empty((max(info.n_tris, 1), 12), np.float32)
        N.sc_scene_export_bvh(self.ctx.handle, self.handle, nodes.ctypes.data, tris.ctypes.data)
        return nodes, tris[: info.n_tris]

    def export_bvh4(self):
        """The 4-wide records [n_nodes, 32] float32 (children boxes SoA, int32 child references in
        columns 24..27; see sc_scene_export_bvh4)."""
        info = self.info()
        nodes4 = np.empty((max(info.n_nodes, 1), 32), np.float32)
        N.sc_scene_export_bvh4(self.ctx.handle, self.handle, nodes4.ctypes.data)
        return nodes4[: info.n_nodes]

    def free(self):
        if getattr(self, "handle", None):
            N.sc_free_scene(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.free()
        except Exception:  # noqa: BLE001
            pass


FLOAT4_FIELDS = ("accum_camera", "accum_caustic", "rgb", "direct", "caustic", "normal_world", "normal_camera",
                 "albedo", "accum_local_caustic", "local_caustic")


class Frame:
    """Frame buffers as CUDA tensors; ``fields`` selects which outputs are produced."""

    ALL = ("accum_camera", "accum_caustic", "rgb", "direct", "caustic", "instance_id", "tri_id", "mask",
           "caustic_mask", "local_caustic_mask", "depth", "depth_norm", "normal_world", "normal_camera", "albedo",
           "outline", "occlusion", "accum_local_caustic", "local_caustic")

    def __init__(self, width: int, height: int, device="cuda", fields=ALL):
        self.width, self.height = width, height
        self.t = {}
        for f in fields:
            if f in FLOAT4_FIELDS:
                self.t[f] = torch.zeros((height, width, 4), dtype=torch.float32, device=device)
            elif f in ("instance_id", "tri_id"):
                self.t[f] = torch.zeros((height, width), dtype=torch.int32, device=device)
            elif f in ("mask", "caustic_mask", "local_caustic_mask", "outline", "occlusion"):
                self.t[f] = torch.zeros((height, width), dtype=torch.uint8, device=device)
            else:
                self.t[f] = torch.zeros((height, width), dtype=torch.float32, device=device)
        self.path_records = None
        self.light_records = None

    def __getitem__(self, k):
        return self.t[k]

    def zero_accumulators(self):
        for k in ("accum_camera", "accum_caustic", "accum_local_caustic"):
            if k in self.t:
                self.t[k].zero_()

    def alloc_path_records(self, spp: int):
        n = self.width * self.height * spp
        self.path_records = torch.zeros((n, C.sizeof(N.sc_path_record) // 4), dtype=torch.int32, device="cuda")
        return self.path_records

    def alloc_light_records(self, n_paths: int):
        self.light_records = torch.zeros((n_paths, C.sizeof(N.sc_light_record) // 4), dtype=torch.int32,
                                         device="cuda")
        return self.light_records

    def struct(self) -> N.sc_frame:
        f = N.sc_frame()
        for k, v in self.t.items():
            setattr(f, k, v.data_ptr())
        f.path_records = self.path_records.data_ptr() if self.path_records is not None else None
        f.light_records = self.light_records.data_ptr() if self.light_records is not None else None
        f.width, f.height = self.width, self.height
        return f


def path_records_numpy(rec: torch.Tensor) -> dict:
    a = rec.cpu().numpy()
    return {"L": a[:, 0:3].view(np.float32), "first_tri": a[:, 3].view(np.int32), "signature": a[:, 4].view(np.uint32),
            "n_queries": a[:, 5].view(np.int32), "bin": a[:, 6].view(np.int32), "n_specular": a[:, 7].view(np.int32)}


def light_records_numpy(rec: torch.Tensor) -> dict:
    a = rec.cpu().numpy()
    return {"C": a[:, 0:3].view(np.float32), "pixel": a[:, 3].view(np.int32), "x": a[:, 4:7].view(np.float32),
            "signature": a[:, 7].view(np.uint32), "n_specular": a[:, 8].view(np.int32), "bin": a[:, 9].view(np.int32)}


def trace_camera(ctx: Context, gs: GpuScene, frame: Frame, spp: int, max_depth: int, n_bins: int = 1, seed: int = 0,
                 sample_offset: int = 0, scene_index: int = 0, flags: int = 0):
    p = N.sc_trace_params(spp, sample_offset, max_depth, n_bins, seed, scene_index, flags)
    N.sc_trace_camera(ctx.handle, gs.handle, p, frame.struct())


def trace_lights(ctx: Context, gs: GpuScene, frame: Frame, n_paths: int, max_depth: int, n_bins: int = 1,
                 seed: int = 0, path_offset: int = 0, scene_index: int = 0, flags: int = 0, guide=None):
    """guide: (cx, cy, cz, r) from scenes.guide_sphere for guided emission, or None."""
    g = (C.c_float * 4)(*(guide if guide is not None else (0.0, 0.0, 0.0, 0.0)))
    p = N.sc_light_params(n_paths, path_offset, max_depth, n_bins, seed, scene_index, flags, g)
    N.sc_trace_lights(ctx.handle, gs.handle, p, frame.struct())


def resolve(ctx: Context, gs: GpuScene, frame: Frame, spp_total: float, light_paths_total: float,
            depth_range: float = 10.0, tau_rel: float = 0.25, outline_px: int = 1, depth_jump_rel: float = 0.05):
    p = N.sc_resolve_params(float(spp_total), float(light_paths_total), depth_range, tau_rel, int(outline_px),
                            float(depth_jump_rel))
    N.sc_resolve(ctx.handle, gs.handle, p, frame.struct())


class PhotonMap:
    """Photons of the light paths that reach a diffuse surface through glass, hashed for gathering
    (sc_photon_map_create); ``gather`` adds the local caustics of camera paths to a frame."""

    def __init__(self, ctx: Context, gs: GpuScene, n_paths: int, radius: float, max_depth: int, n_bins: int = 1,
                 seed: int = 0, path_offset: int = 0, scene_index: int = 0, flags: int = 0, guide=None):
        g = (0.0, 0.0, 0.0, 0.0) if guide is None else tuple(float(x) for x in guide)
        p = N.sc_light_params(int(n_paths), int(path_offset), max_depth, n_bins, seed, scene_index, flags, g)
        self.ctx, self.n_paths, self.radius = ctx, int(n_paths), float(radius)
        self.handle = N.sc_photon_map_create(ctx.handle, gs.handle, p, float(radius))

    def export(self):
        """Photons in light-path order: dict of position (n,3), bin (n,), normal (n,3), deposited (n,),
        throughput (n,3)."""
        ph = np.empty((self.n_paths, 12), np.float32)
        order = np.empty(self.n_paths, np.uint32)
        N.sc_photon_map_export(self.ctx.handle, self.handle, ph.ctypes.data, order.ctypes.data)
        out = np.empty_like(ph)
        out[order] = ph
        return {"x": out[:, 0:3], "bin": out[:, 3].view(np.int32), "n": out[:, 4:7], "photon": out[:, 7] != 0,
                "beta": out[:, 8:11]}

    def gather(self, gs: GpuScene, frame: Frame, spp: int, max_depth: int, n_bins: int = 1, seed: int = 0,
               sample_offset: int = 0, scene_index: int = 0, flags: int = 0):
        p = N.sc_trace_params(spp, sample_offset, max_depth, n_bins, seed, scene_index, flags)
        N.sc_gather_local_caustics(self.ctx.handle, gs.handle, self.handle, p, frame.struct())

    def close(self):
        if getattr(self, "handle", None):
            N.sc_photon_map_destroy(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass


def intersect(ctx: Context, gs: GpuScene, origins: torch.Tensor, dirs: torch.Tensor, tmax: float = 3.0e38):
    """Closest hits of rays given as (n,3) CUDA tensors: returns (t, tri, b1, b2) tensors."""
    n = origins.shape[0]
    rays = torch.zeros((n, 8), dtype=torch.float32, device=origins.device)
    rays[:, 0:3] = origins
    rays[:, 3] = tmax
    rays[:, 4:7] = dirs
    hits = torch.empty((n, 4), dtype=torch.float32, device=origins.device)
    N.sc_intersect(ctx.handle, gs.handle, rays.data_ptr(), n, hits.data_ptr())
    return hits[:, 0], hits[:, 1].contiguous().view(torch.int32), hits[:, 2], hits[:, 3]


def occluded(ctx: Context, gs: GpuScene, origins: torch.Tensor, dirs: torch.Tensor, tmax: torch.Tensor):
    n = origins.shape[0]
    rays = torch.zeros((n, 8), dtype=torch.float32, device=origins.device)
    rays[:, 0:3] = origins
    rays[:, 3] = tmax
    rays[:, 4:7] = dirs
    occ = torch.empty((n,), dtype=torch.int32, device=origins.device)
    N.sc_occluded(ctx.handle, gs.handle, rays.data_ptr(), n, occ.data_ptr())
    return occ


def philox(ctx: Context, counters: torch.Tensor, key: int) -> torch.Tensor:
    c = counters.contiguous().view(torch.int32)
    out = torch.empty_like(c)
    N.sc_philox4x32_10(ctx.handle, c.data_ptr(), key, c.shape[0], out.data_ptr())
    return out


def trace_batch(ctx: Context, scenes, frames, spp: int, max_depth: int, n_bins: int = 1, seed: int = 0,
                sample_offset: int = 0, scene_index: int = 0, flags: int = 0):
    """Camera paths of many scenes in one persistent launch (scene i uses scene index scene_index + i)."""
    p = N.sc_trace_params(spp, sample_offset, max_depth, n_bins, seed, scene_index, flags)
    N.sc_trace_batch(ctx.handle, [g.handle for g in scenes], [f.struct() for f in frames], p)


class Batch:
    """The batched launch captured once as a CUDA graph; ``launch()`` replays it."""

    def __init__(self, ctx: Context, scenes, frames, spp: int, max_depth: int, n_bins: int = 1, seed: int = 0,
                 sample_offset: int = 0, scene_index: int = 0, flags: int = 0):
        self.ctx, self.scenes, self.frames = ctx, list(scenes), list(frames)
        p = N.sc_trace_params(spp, sample_offset, max_depth, n_bins, seed, scene_index, flags)
        self.handle = N.sc_batch_create(ctx.handle, [g.handle for g in self.scenes], [f.struct() for f in self.frames], p)

    def launch(self):
        N.sc_batch_launch(self.ctx.handle, self.handle)

    def close(self):
        if getattr(self, "handle", None):
            N.sc_batch_destroy(self.ctx.handle, self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001
            pass
