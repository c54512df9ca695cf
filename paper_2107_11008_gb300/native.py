"""ctypes binding of ``include/supercaustics.h`` (argument marshalling only).

Every function here forwards to the entry point of the same name in ``libsupercaustics.so`` and
raises ``ScError`` on a negative status.  No step of the renderer runs in Python: if the library
is missing the import of this module fails.
"""
from __future__ import annotations

import ctypes as C
import os

from . import build as _build

P = C.POINTER

SC_OK = 0
ERRORS = {-1: "SC_ERR_INVALID_ARG", -2: "SC_ERR_CUDA", -3: "SC_ERR_OOM", -4: "SC_ERR_STACK_OVERFLOW",
          -5: "SC_ERR_TIMEOUT", -6: "SC_ERR_QUEUE_OVERFLOW", -7: "SC_ERR_UNSUPPORTED", -8: "SC_ERR_BOUNDS"}
SC_FLAG_FORCE_TRANSMIT = 1
SC_FLAG_SPLAT_DIRECT = 2
SC_FLAG_EMITTER_AFTER_DS = 4
SC_FLAG_WAVELENGTH_JITTER = 8


class ScError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"{ERRORS.get(code, code)}: {msg}")
        self.code = code


class sc_material(C.Structure):
    _fields_ = [("kind", C.c_int32), ("albedo", C.c_float * 3), ("albedo2", C.c_float * 3),
                ("checker_scale", C.c_float), ("cauchy_a", C.c_float), ("cauchy_b", C.c_float),
                ("emission", C.c_float * 3), ("absorption", C.c_float * 3), ("roughness", C.c_float)]


class sc_light(C.Structure):
    _fields_ = [("kind", C.c_int32), ("p", C.c_float * 3), ("u", C.c_float * 3), ("v", C.c_float * 3),
                ("power", C.c_float * 3), ("radius", C.c_float)]


class sc_camera(C.Structure):
    _fields_ = [("eye", C.c_float * 3), ("look", C.c_float * 3), ("up", C.c_float * 3), ("vfov_deg", C.c_float),
                ("width", C.c_int32), ("height", C.c_int32)]


class sc_scene_desc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("positions", C.c_void_p), ("normals", C.c_void_p),
                ("uvs", C.c_void_p), ("indices", C.c_void_p), ("tri_object", C.c_void_p),
                ("n_objects", C.c_int32), ("object_material", C.c_void_p), ("n_materials", C.c_int32),
                ("materials", P(sc_material)), ("n_lights", C.c_int32), ("lights", P(sc_light)),
                ("env", C.c_float * 3), ("camera", sc_camera), ("geometry_on_device", C.c_int32)]


class sc_trace_params(C.Structure):
    _fields_ = [("spp", C.c_int32), ("sample_offset", C.c_int32), ("max_depth", C.c_int32), ("n_bins", C.c_int32),
                ("seed", C.c_uint64), ("scene_index", C.c_int32), ("flags", C.c_int32)]


class sc_light_params(C.Structure):
    _fields_ = [("n_paths", C.c_int64), ("path_offset", C.c_int64), ("max_depth", C.c_int32), ("n_bins", C.c_int32),
                ("seed", C.c_uint64), ("scene_index", C.c_int32), ("flags", C.c_int32), ("guide", C.c_float * 4)]


class sc_resolve_params(C.Structure):
    _fields_ = [("spp_total", C.c_double), ("light_paths_total", C.c_double), ("depth_range", C.c_float),
                ("tau_rel", C.c_float), ("outline_px", C.c_int32), ("depth_jump_rel", C.c_float)]


class sc_path_record(C.Structure):
    _fields_ = [("L", C.c_float * 3), ("first_tri", C.c_uint32), ("signature", C.c_uint32),
                ("n_queries", C.c_uint32), ("bin", C.c_uint32), ("n_specular", C.c_uint32)]


class sc_light_record(C.Structure):
    _fields_ = [("C", C.c_float * 3), ("pixel", C.c_int32), ("x", C.c_float * 3), ("signature", C.c_uint32),
                ("n_specular", C.c_uint32), ("bin", C.c_uint32), ("pad", C.c_uint32 * 2)]


FRAME_FIELDS = ["accum_camera", "accum_caustic", "rgb", "direct", "caustic", "instance_id", "tri_id", "mask",
                "caustic_mask", "local_caustic_mask", "depth", "depth_norm", "normal_world", "normal_camera",
                "albedo", "outline", "occlusion", "accum_local_caustic", "local_caustic", "path_records",
                "light_records"]


class sc_frame(C.Structure):
    _fields_ = [(n, C.c_void_p) for n in FRAME_FIELDS] + [("width", C.c_int32), ("height", C.c_int32)]


class sc_scene_info(C.Structure):
    _fields_ = [("n_tris", C.c_int32), ("n_nodes", C.c_int32), ("n_materials", C.c_int32), ("n_lights", C.c_int32),
                ("bvh_bytes", C.c_int64), ("max_depth", C.c_int32), ("bvh_width", C.c_int32)]


class sc_unet_buffer_info(C.Structure):
    _fields_ = [("dtype", C.c_int32), ("n", C.c_int32), ("h", C.c_int32), ("w", C.c_int32), ("c", C.c_int32)]


STRUCTS = [sc_material, sc_light, sc_camera, sc_scene_desc, sc_trace_params, sc_light_params, sc_resolve_params,
           sc_path_record, sc_light_record, sc_frame, sc_scene_info]

ALLOC_FN = C.CFUNCTYPE(C.c_void_p, C.c_size_t, C.c_void_p)
FREE_FN = C.CFUNCTYPE(None, C.c_void_p, C.c_void_p)

# exported entry points and their signatures
SIGNATURES = {
    "sc_abi_version": (C.c_int, []),
    "sc_struct_sizes": (C.c_int, [P(C.c_int32), C.c_int32]),
    "sc_create": (C.c_int, [C.c_int, C.c_void_p, ALLOC_FN, FREE_FN, C.c_void_p, P(C.c_void_p)]),
    "sc_destroy": (C.c_int, [C.c_void_p]),
    "sc_set_stream": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_last_error": (C.c_char_p, [C.c_void_p]),
    "sc_sync_status": (C.c_int, [C.c_void_p]),
    "sc_set_counters": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_build_scene": (C.c_int, [C.c_void_p, P(sc_scene_desc), P(C.c_void_p)]),
    "sc_free_scene": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_scene_get_info": (C.c_int, [C.c_void_p, P(sc_scene_info)]),
    "sc_scene_export_bvh": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_scene_export_bvh4": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_build_bvh_noalloc": (C.c_int, [C.c_void_p] + [C.c_void_p] * 6 + [C.c_int32, C.c_int32] + [C.c_void_p] * 5),
    "sc_intersect": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "sc_occluded": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p]),
    "sc_philox4x32_10": (C.c_int, [C.c_void_p, C.c_void_p, C.c_uint64, C.c_int64, C.c_void_p]),
    "sc_trace_camera": (C.c_int, [C.c_void_p, C.c_void_p, P(sc_trace_params), P(sc_frame)]),
    "sc_trace_lights": (C.c_int, [C.c_void_p, C.c_void_p, P(sc_light_params), P(sc_frame)]),
    "sc_resolve": (C.c_int, [C.c_void_p, C.c_void_p, P(sc_resolve_params), P(sc_frame)]),
    "sc_trace_batch": (C.c_int, [C.c_void_p, P(C.c_void_p), P(sc_frame), C.c_int32, P(sc_trace_params)]),
    "sc_batch_create": (C.c_int, [C.c_void_p, P(C.c_void_p), P(sc_frame), C.c_int32, P(sc_trace_params),
                                  P(C.c_void_p)]),
    "sc_batch_launch": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_batch_destroy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_set_limits": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_set_camera_engine": (C.c_int, [C.c_void_p, C.c_int32]),
    "sc_get_camera_engine": (C.c_int, [C.c_void_p, P(C.c_int32)]),
    "sc_get_limits": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_unet_get_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, P(C.c_int64)]),
    "sc_unet_set_state": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64]),
    "sc_unet_save": (C.c_int, [C.c_void_p, C.c_void_p, C.c_char_p]),
    "sc_unet_set_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32]),
    "sc_unet_wait_selftest": (C.c_int, [C.c_void_p, C.c_uint32, C.c_void_p]),
    "sc_unet_load": (C.c_int, [C.c_void_p, C.c_void_p, C.c_char_p]),
    "sc_photon_map_create": (C.c_int, [C.c_void_p, C.c_void_p, P(sc_light_params), C.c_float, P(C.c_void_p)]),
    "sc_photon_map_destroy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_photon_map_export": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_gather_local_caustics": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, P(sc_trace_params), P(sc_frame)]),
    "sc_peak_fma": (C.c_int, [C.c_void_p, C.c_int64, C.c_void_p, P(C.c_int64)]),
    "sc_peak_l2_read": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p, P(C.c_int64)]),
    # sc_unet.h
    "sc_unet_param_count": (C.c_int, [P(C.c_int64)]),
    "sc_unet_create": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, P(C.c_void_p)]),
    "sc_unet_destroy": (C.c_int, [C.c_void_p, C.c_void_p]),
    "sc_unet_set_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_unet_get_params": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_unet_get_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_unet_set_grads": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sc_unet_forward": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]),
    "sc_unet_loss_grad": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p,
                                    C.c_void_p]),
    "sc_unet_adam": (C.c_int, [C.c_void_p, C.c_void_p, C.c_float]),
    "sc_unet_train_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_float,
                                     C.c_void_p]),
    "sc_ssim_l1_loss": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_void_p,
                                  C.c_void_p]),
    "sc_unet_pack_frame": (C.c_int, [C.c_void_p, P(sc_frame), C.c_int32, C.c_void_p, C.c_int32]),
    "sc_unet_pack_target": (C.c_int, [C.c_void_p, P(sc_frame), C.c_int32, C.c_void_p, C.c_int32]),
    "sc_unet_output_rgb": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p]),
    "sc_unet_buffer": (C.c_int, [C.c_void_p, C.c_int32, C.c_int32, P(sc_unet_buffer_info)]),
    "sc_unet_copy_buffer": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int32, C.c_int32, C.c_void_p]),
}

_lib = None


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True):
    """Load libsupercaustics.so (building it first if asked); raises if it cannot be loaded."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if not os.path.exists(path):
        if not build_if_missing:
            raise ImportError(f"libsupercaustics.so not built ({path}); run paper_2107_11008_gb300.build")
        _build.build_library()
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    sizes = (C.c_int32 * len(STRUCTS))()
    k = lib.sc_struct_sizes(sizes, len(STRUCTS))
    want = [C.sizeof(s) for s in STRUCTS]
    if k != len(STRUCTS) or list(sizes) != want:
        raise ImportError(f"supercaustics ABI layout mismatch: library {list(sizes)} vs binding {want}")
    _lib = lib
    return lib


def check(code: int, ctx=None):
    if code != SC_OK:
        msg = load().sc_last_error(ctx).decode() if ctx else ""
        raise ScError(code, msg)
    return code


# --- thin wrappers, same names as the C entry points ------------------------------------------
def sc_abi_version() -> int:
    return load().sc_abi_version()


def sc_create(device, stream, alloc=None, free=None, user=None):
    out = C.c_void_p()
    a = alloc if alloc is not None else ALLOC_FN()
    f = free if free is not None else FREE_FN()
    check(load().sc_create(device, stream, a, f, user, C.byref(out)))
    return out.value


def sc_destroy(ctx):
    return check(load().sc_destroy(ctx))


def sc_set_stream(ctx, stream):
    return check(load().sc_set_stream(ctx, stream), ctx)


def sc_last_error(ctx) -> str:
    return load().sc_last_error(ctx).decode()


def sc_sync_status(ctx):
    return check(load().sc_sync_status(ctx), ctx)


def sc_set_counters(ctx, counters_dev):
    return check(load().sc_set_counters(ctx, counters_dev), ctx)


def sc_build_scene(ctx, desc: sc_scene_desc):
    out = C.c_void_p()
    check(load().sc_build_scene(ctx, C.byref(desc), C.byref(out)), ctx)
    return out.value


def sc_free_scene(ctx, scene):
    return check(load().sc_free_scene(ctx, scene), ctx)


def sc_scene_get_info(scene) -> sc_scene_info:
    info = sc_scene_info()
    check(load().sc_scene_get_info(scene, C.byref(info)))
    return info


def sc_scene_export_bvh(ctx, scene, nodes_host, tris_host):
    return check(load().sc_scene_export_bvh(ctx, scene, nodes_host, tris_host), ctx)


def sc_scene_export_bvh4(ctx, scene, nodes4_host):
    return check(load().sc_scene_export_bvh4(ctx, scene, nodes4_host), ctx)


def sc_intersect(ctx, scene, rays_dev, n, hits_dev):
    return check(load().sc_intersect(ctx, scene, rays_dev, n, hits_dev), ctx)


def sc_occluded(ctx, scene, rays_dev, n, occ_dev):
    return check(load().sc_occluded(ctx, scene, rays_dev, n, occ_dev), ctx)


def sc_philox4x32_10(ctx, ctr_dev, key, n, out_dev):
    return check(load().sc_philox4x32_10(ctx, ctr_dev, key, n, out_dev), ctx)


def sc_trace_camera(ctx, scene, params: sc_trace_params, frame: sc_frame):
    return check(load().sc_trace_camera(ctx, scene, C.byref(params), C.byref(frame)), ctx)


def sc_trace_lights(ctx, scene, params: sc_light_params, frame: sc_frame):
    return check(load().sc_trace_lights(ctx, scene, C.byref(params), C.byref(frame)), ctx)


def sc_resolve(ctx, scene, params: sc_resolve_params, frame: sc_frame):
    return check(load().sc_resolve(ctx, scene, C.byref(params), C.byref(frame)), ctx)


def _tables(scenes, frames):
    n = len(scenes)
    if len(frames) != n:
        raise ValueError("one frame per scene")
    sa = (C.c_void_p * n)(*scenes)
    fa = (sc_frame * n)(*frames)
    return n, sa, fa


def sc_trace_batch(ctx, scenes, frames, params: sc_trace_params):
    n, sa, fa = _tables(scenes, frames)
    return check(load().sc_trace_batch(ctx, sa, fa, n, C.byref(params)), ctx)


def sc_batch_create(ctx, scenes, frames, params: sc_trace_params):
    n, sa, fa = _tables(scenes, frames)
    out = C.c_void_p()
    check(load().sc_batch_create(ctx, sa, fa, n, C.byref(params), C.byref(out)), ctx)
    return out.value


def sc_batch_launch(ctx, batch):
    return check(load().sc_batch_launch(ctx, batch), ctx)


class sc_limits(C.Structure):
    _fields_ = [("max_visits", C.c_int64), ("stack_depth4", C.c_int32), ("stack_depth2", C.c_int32)]


def sc_set_limits(ctx, max_visits=0, stack_depth4=0, stack_depth2=0, defaults=False):
    if defaults:
        check(load().sc_set_limits(ctx, None), ctx)
    else:
        lim = sc_limits(max_visits, stack_depth4, stack_depth2)
        check(load().sc_set_limits(ctx, C.byref(lim)), ctx)


SC_CAMERA_WAVEFRONT = 0
SC_CAMERA_PERSISTENT = 1


def sc_set_camera_engine(ctx, engine: int):
    check(load().sc_set_camera_engine(ctx, engine), ctx)


def sc_get_camera_engine(ctx) -> int:
    e = C.c_int32()
    check(load().sc_get_camera_engine(ctx, C.byref(e)), ctx)
    return e.value


def sc_get_limits(ctx) -> sc_limits:
    lim = sc_limits()
    check(load().sc_get_limits(ctx, C.byref(lim)), ctx)
    return lim


def sc_unet_get_state(ctx, net, m_dev, v_dev) -> int:
    step = C.c_int64()
    check(load().sc_unet_get_state(ctx, net, m_dev, v_dev, C.byref(step)), ctx)
    return step.value


def sc_unet_set_state(ctx, net, params_dev, m_dev, v_dev, step):
    check(load().sc_unet_set_state(ctx, net, params_dev, m_dev, v_dev, step), ctx)


SC_UNET_LOSS_L1_SSIM = 0
SC_UNET_LOSS_BCE = 1
SC_UNET_LOSS_L2_LINEAR = 2


def sc_unet_set_loss(ctx, net, kind: int):
    check(load().sc_unet_set_loss(ctx, net, kind), ctx)


def sc_unet_wait_selftest(ctx, poll_limit: int):
    """Runs the tensor-core kernels' abort path once (see sc_unet.h); returns the 8 outcome words."""
    out = (C.c_int64 * 8)()
    check(load().sc_unet_wait_selftest(ctx, poll_limit, out), ctx)
    return list(out)


def sc_unet_save(ctx, net, path: str):
    check(load().sc_unet_save(ctx, net, os.fsencode(path)), ctx)


def sc_unet_load(ctx, net, path: str):
    check(load().sc_unet_load(ctx, net, os.fsencode(path)), ctx)


def sc_photon_map_create(ctx, scene, params: sc_light_params, radius: float):
    out = C.c_void_p()
    check(load().sc_photon_map_create(ctx, scene, C.byref(params), radius, C.byref(out)), ctx)
    return out.value


def sc_photon_map_destroy(ctx, pm):
    check(load().sc_photon_map_destroy(ctx, pm), ctx)


def sc_photon_map_export(ctx, pm, photons_host, order_host):
    check(load().sc_photon_map_export(ctx, pm, photons_host, order_host), ctx)


def sc_gather_local_caustics(ctx, scene, pm, params: sc_trace_params, frame: sc_frame):
    check(load().sc_gather_local_caustics(ctx, scene, pm, C.byref(params), C.byref(frame)), ctx)


def sc_peak_fma(ctx, iters, sink_dev) -> int:
    flops = C.c_int64()
    check(load().sc_peak_fma(ctx, iters, sink_dev, C.byref(flops)), ctx)
    return flops.value


def sc_peak_l2_read(ctx, buf_dev, nbytes, reps, sink_dev) -> int:
    nread = C.c_int64()
    check(load().sc_peak_l2_read(ctx, buf_dev, nbytes, reps, sink_dev, C.byref(nread)), ctx)
    return nread.value


def sc_batch_destroy(ctx, batch):
    return check(load().sc_batch_destroy(ctx, batch), ctx)


# --- sc_unet.h ---------------------------------------------------------------------------------
SC_UNET_BUF = dict(INPUT=0, ENC1=1, ENC2=2, POOL=3, UP=4, DEC1=5, DEC2=6, OUT=7, GOUT=8, GDEC2=9, GDEC1=10,
                   GUP=11, GSKIP=12, GENC2=13, GENC1=14)


def sc_unet_param_count() -> int:
    n = C.c_int64()
    check(load().sc_unet_param_count(C.byref(n)))
    return n.value


def sc_unet_create(ctx, max_batch, height, width):
    out = C.c_void_p()
    check(load().sc_unet_create(ctx, max_batch, height, width, C.byref(out)), ctx)
    return out.value


def sc_unet_destroy(ctx, net):
    return check(load().sc_unet_destroy(ctx, net), ctx)


def sc_unet_set_params(ctx, net, params_dev):
    return check(load().sc_unet_set_params(ctx, net, params_dev), ctx)


def sc_unet_get_params(ctx, net, params_dev):
    return check(load().sc_unet_get_params(ctx, net, params_dev), ctx)


def sc_unet_get_grads(ctx, net, grads_dev):
    return check(load().sc_unet_get_grads(ctx, net, grads_dev), ctx)


def sc_unet_set_grads(ctx, net, grads_dev):
    return check(load().sc_unet_set_grads(ctx, net, grads_dev), ctx)


def sc_unet_forward(ctx, net, x_dev, n, y_dev):
    return check(load().sc_unet_forward(ctx, net, x_dev, n, y_dev), ctx)


def sc_unet_loss_grad(ctx, net, x_dev, target_dev, n, y_dev=None, loss_dev=None):
    return check(load().sc_unet_loss_grad(ctx, net, x_dev, target_dev, n, y_dev, loss_dev), ctx)


def sc_unet_adam(ctx, net, lr):
    return check(load().sc_unet_adam(ctx, net, lr), ctx)


def sc_unet_train_step(ctx, net, x_dev, target_dev, n, lr, loss_dev=None):
    return check(load().sc_unet_train_step(ctx, net, x_dev, target_dev, n, lr, loss_dev), ctx)


def sc_ssim_l1_loss(ctx, pred_dev, target_dev, n, h, w, loss_dev=None, grad_dev=None):
    return check(load().sc_ssim_l1_loss(ctx, pred_dev, target_dev, n, h, w, loss_dev, grad_dev), ctx)


SC_UNET_SRC_RGB, SC_UNET_SRC_DIRECT, SC_UNET_SRC_CAUSTIC = 0, 1, 2


def sc_unet_pack_frame(ctx, frame: sc_frame, source, x_dev, index):
    return check(load().sc_unet_pack_frame(ctx, C.byref(frame), source, x_dev, index), ctx)


def sc_unet_buffer(net, buf_id, level) -> sc_unet_buffer_info:
    info = sc_unet_buffer_info()
    check(load().sc_unet_buffer(net, buf_id, level, C.byref(info)))
    return info


def sc_unet_copy_buffer(ctx, net, buf_id, level, dst_dev):
    return check(load().sc_unet_copy_buffer(ctx, net, buf_id, level, dst_dev), ctx)


def sc_unet_pack_target(ctx, frame: sc_frame, source, t_dev, index):
    return check(load().sc_unet_pack_target(ctx, C.byref(frame), source, t_dev, index), ctx)


def sc_unet_output_rgb(ctx, y_dev, n_px, add_dev, rgb_dev):
    return check(load().sc_unet_output_rgb(ctx, y_dev, n_px, add_dev, rgb_dev), ctx)
