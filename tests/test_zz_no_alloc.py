"""sc_build_bvh_noalloc: the LBVH build for callers that cannot allocate device memory while they
run.  Its output must equal sc_build_scene's (same kernels), call after call, even though every
call reuses the same static scratch array.  Kept in its own file, collected last."""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_2107_11008_gb300 import native as N  # noqa: E402
from paper_2107_11008_gb300 import renderer as R  # noqa: E402
from paper_2107_11008_gb300 import scenes as S  # noqa: E402

pytestmark = pytest.mark.gpu

MAX_TRIS = 32768  # SC_NOALLOC_MAX_TRIS in include/supercaustics.h


def _soup(n_tris, seed):
    rng = np.random.default_rng(seed)
    b = S.SceneBuilder()
    m = b.material(S.Material(S.MAT_DIFFUSE))
    c = rng.uniform(-1, 1, (n_tris, 1, 3))
    p = c + rng.normal(0, 0.1, (n_tris, 3, 3))
    b.add(S.Mesh(p.reshape(-1, 3), np.arange(3 * n_tris).reshape(-1, 3), None, None), m)
    return b.build(S.Camera((0, 0, 5), (0, 0, 0), (0, 1, 0), 40, 8, 8))


def _noalloc_build(ctx, sc, with_attributes=True):
    a = R.SceneArrays(sc, "cuda")
    om = torch.from_numpy(a.object_material).cuda()
    n = sc.n_tris
    out = {"nodes": torch.empty((max(n - 1, 1), 16), dtype=torch.float32, device="cuda"),
           "tris": torch.empty((n, 12), dtype=torch.float32, device="cuda"),
           "shade": torch.empty((n, 12), dtype=torch.float32, device="cuda"),
           "shade2": torch.empty((n, 4), dtype=torch.float32, device="cuda"),
           "tri_obj": torch.empty((n,), dtype=torch.int32, device="cuda")}
    nrm = a.normals.data_ptr() if with_attributes else None
    uvs = a.uvs.data_ptr() if with_attributes else None
    dev_before = torch.cuda.current_device()
    rc = N.load().sc_build_bvh_noalloc(ctx.handle, a.positions.data_ptr(), nrm, uvs,
                                       a.indices.data_ptr(), a.tri_object.data_ptr(), om.data_ptr(),
                                       int(om.shape[0]), n, out["nodes"].data_ptr(), out["tris"].data_ptr(),
                                       out["shade"].data_ptr(), out["shade2"].data_ptr(), out["tri_obj"].data_ptr())
    assert rc == 0, N.sc_last_error(ctx.handle)
    assert torch.cuda.current_device() == dev_before  # the caller's current device is left as it was
    ctx.sync_status()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _check_against_build_scene(ctx, sc, got):
    ref_nodes, ref_tris = R.GpuScene(ctx, sc).export_bvh()
    if sc.n_tris > 1:
        np.testing.assert_array_equal(got["nodes"], ref_nodes)
    np.testing.assert_array_equal(got["tris"], ref_tris)


def test_noalloc_build_matches_sc_build_scene_twice_in_a_row():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = R.Context(0)
    # larger scene first, then smaller ones: a call must not see an earlier call's scratch.  The
    # first fills the scratch exactly (the largest accepted size); the last is a single triangle
    # (a root that is a leaf: no hierarchy launch).
    for sc in (_soup(MAX_TRIS, 4), _soup(20000, 3), S.ball_on_plane(), _soup(1, 5)):
        got = _noalloc_build(ctx, sc)
        _check_against_build_scene(ctx, sc, got)
        np.testing.assert_array_equal(got["tri_obj"], sc.tri_object)
        # per input triangle: vertex normals and uv
        nrm = sc.normals[sc.indices]  # (n, 3, 3)
        np.testing.assert_array_equal(got["shade"].reshape(-1, 3, 4)[:, :, :3], nrm)
        np.testing.assert_array_equal(got["shade"].reshape(-1, 3, 4)[:, :, 3], sc.uvs[sc.indices][:, :, 0])
        np.testing.assert_array_equal(got["shade2"][:, :3], sc.uvs[sc.indices][:, :, 1])
    ctx.close()


def test_noalloc_build_without_normals_and_uvs():
    """normals = uvs = NULL is allowed: the tree is the same and the attributes read as zero."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = R.Context(0)
    sc = S.ball_on_plane()
    got = _noalloc_build(ctx, sc, with_attributes=False)
    _check_against_build_scene(ctx, sc, got)
    np.testing.assert_array_equal(got["shade"], 0.0)
    np.testing.assert_array_equal(got["shade2"][:, :3], 0.0)
    np.testing.assert_array_equal(got["tri_obj"], sc.tri_object)
    ctx.close()


def test_noalloc_rejects_sizes_beyond_its_scratch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = R.Context(0)
    dummy = torch.zeros(16, dtype=torch.float32, device="cuda")
    p = dummy.data_ptr()
    for n in (0, MAX_TRIS + 1):
        rc = N.load().sc_build_bvh_noalloc(ctx.handle, p, None, None, p, p, p, 1, n, p, p, p, p, p)
        assert rc == -1
        assert "SC_NOALLOC" in N.sc_last_error(ctx.handle) or "n_tris" in N.sc_last_error(ctx.handle)
    ctx.close()
