"""Seeded synthetic scene generator (the inputs of the renderer).

This module builds the synthetic stand-ins for the paper's scenes: several
transparent objects over a diffuse backdrop under a point or an area light
(SuperCaustics, Sec. III-A Generator Module and Sec. III-C Data Ablation Core;
Fig. 1 and Fig. 4 show the kind of scene).  The paper's asset banks, physics
settling and HDRI maps are not available, so objects are procedural meshes
with random pose, scale and index of refraction drawn from a seeded generator.

It holds none of the renderer's arithmetic: no ray, no intersection, no
shading.  Both the CUDA library and the CPU oracle take the flat arrays this
module produces (world-space float32 triangles), so neither side depends on
the other.

Conventions shared by every consumer of a ``Scene``:

* ``positions`` (V,3) float32 world space, ``indices`` (T,3) int32 with the
  geometric normal given by the winding (v1-v0) x (v2-v0).
* ``normals`` (V,3) float32; a triangle with any all-zero vertex normal is
  flat (shaded with its geometric normal).
* ``uvs`` (V,2) float32 surface coordinates in metres, used by checker albedo.
* ``tri_object`` (T,) int32 object id; ``object_material`` (O,) int32.
* Materials: DIFFUSE (albedo or checker of two albedos), DIELECTRIC (Cauchy
  A, B in um^2), EMISSIVE (radiance, one-sided along the winding normal).
* Lights: POINT (position, intensity W/sr), RECT (corner, edge_u, edge_v,
  radiance; emits along edge_u x edge_v), DISK (a collimated beam used by
  optics tests: centre, direction, radius, irradiance).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MAT_DIFFUSE = 0
MAT_DIELECTRIC = 1
MAT_EMISSIVE = 2

LIGHT_POINT = 0
LIGHT_RECT = 1
LIGHT_DISK = 2


@dataclass
class Material:
    kind: int
    albedo: tuple = (0.5, 0.5, 0.5)
    albedo2: tuple = (0.5, 0.5, 0.5)
    checker_scale: float = 0.0  # squares per metre; 0 = plain albedo
    cauchy_a: float = 1.5
    cauchy_b: float = 0.0  # um^2
    emission: tuple = (0.0, 0.0, 0.0)
    absorption: tuple = (0.0, 0.0, 0.0)  # dielectric: Beer-Lambert coefficient per metre (glass colour)
    roughness: float = 0.0  # dielectric: GGX width alpha (0 = smooth glass)

    def flat(self) -> list:
        """17 numbers: kind, albedo[3], albedo2[3], checker_scale, A, B, emission[3], absorption[3],
        roughness."""
        return [float(self.kind), *map(float, self.albedo), *map(float, self.albedo2),
                float(self.checker_scale), float(self.cauchy_a), float(self.cauchy_b),
                *map(float, self.emission), *map(float, self.absorption), float(self.roughness)]


@dataclass
class Light:
    kind: int
    p: tuple  # point position / rect corner / disk centre
    u: tuple = (0.0, 0.0, 0.0)  # rect edge_u / disk direction
    v: tuple = (0.0, 0.0, 0.0)  # rect edge_v
    power: tuple = (1.0, 1.0, 1.0)  # I (point) / Le (rect) / E (disk)
    radius: float = 0.0  # disk radius

    def flat(self) -> list:
        """14 numbers: kind, p[3], u[3], v[3], power[3], radius."""
        return [float(self.kind), *map(float, self.p), *map(float, self.u), *map(float, self.v),
                *map(float, self.power), float(self.radius)]


@dataclass
class Camera:
    eye: tuple
    look: tuple
    up: tuple
    vfov_deg: float
    width: int
    height: int

    def flat(self) -> list:
        """10 numbers: eye[3], look[3], up[3], vfov in degrees."""
        return [*map(float, self.eye), *map(float, self.look), *map(float, self.up), float(self.vfov_deg)]


@dataclass
class Mesh:
    positions: np.ndarray  # (V,3) float64
    indices: np.ndarray  # (T,3) int64
    normals: np.ndarray | None = None  # (V,3) float64, zero rows = flat
    uvs: np.ndarray | None = None  # (V,2)

    @property
    def n_tris(self) -> int:
        return int(self.indices.shape[0])

    def transformed(self, rot: np.ndarray, scale: float, offset) -> "Mesh":
        p = (self.positions * scale) @ rot.T + np.asarray(offset, dtype=np.float64)
        n = None if self.normals is None else self.normals @ rot.T
        return Mesh(p, self.indices.copy(), n, None if self.uvs is None else self.uvs.copy())


@dataclass
class Scene:
    positions: np.ndarray
    normals: np.ndarray
    uvs: np.ndarray
    indices: np.ndarray
    tri_object: np.ndarray
    object_material: np.ndarray
    materials: list
    lights: list
    camera: Camera
    env: tuple = (0.0, 0.0, 0.0)
    name: str = "scene"

    @property
    def n_tris(self) -> int:
        return int(self.indices.shape[0])

    @property
    def n_objects(self) -> int:
        return int(self.object_material.shape[0])

    def materials_flat(self) -> np.ndarray:
        return np.asarray([m.flat() for m in self.materials], dtype=np.float64).reshape(-1, 17)

    def lights_flat(self) -> np.ndarray:
        return np.asarray([l.flat() for l in self.lights], dtype=np.float64).reshape(-1, 14)

    def nbytes(self) -> int:
        return int(self.positions.nbytes + self.normals.nbytes + self.uvs.nbytes + self.indices.nbytes
                   + self.tri_object.nbytes + self.object_material.nbytes)


class SceneBuilder:
    """Accumulates objects (one material each) into flat world-space arrays."""

    def __init__(self):
        self._pos, self._nrm, self._uv, self._idx, self._obj = [], [], [], [], []
        self._obj_mat = []
        self.materials: list = []
        self.lights: list = []
        self._nv = 0

    def material(self, m: Material) -> int:
        self.materials.append(m)
        return len(self.materials) - 1

    def add(self, mesh: Mesh, material: int) -> int:
        oid = len(self._obj_mat)
        v = mesh.positions.shape[0]
        self._pos.append(mesh.positions)
        self._nrm.append(np.zeros((v, 3)) if mesh.normals is None else mesh.normals)
        self._uv.append(np.zeros((v, 2)) if mesh.uvs is None else mesh.uvs)
        self._idx.append(mesh.indices + self._nv)
        self._obj.append(np.full(mesh.n_tris, oid))
        self._obj_mat.append(material)
        self._nv += v
        return oid

    def add_rect_light(self, corner, edge_u, edge_v, radiance) -> int:
        """A one-sided area light: an emissive quad plus the matching light record."""
        m = self.material(Material(MAT_EMISSIVE, emission=tuple(radiance)))
        self.add(quad(corner, edge_u, edge_v), m)
        self.lights.append(Light(LIGHT_RECT, tuple(corner), tuple(edge_u), tuple(edge_v), tuple(radiance)))
        return len(self.lights) - 1

    def build(self, camera: Camera, env=(0.0, 0.0, 0.0), name="scene") -> Scene:
        pos = np.concatenate(self._pos).astype(np.float32)
        nrm = np.concatenate(self._nrm).astype(np.float32)
        uv = np.concatenate(self._uv).astype(np.float32)
        idx = np.concatenate(self._idx).astype(np.int32)
        obj = np.concatenate(self._obj).astype(np.int32)
        return Scene(np.ascontiguousarray(pos), np.ascontiguousarray(nrm), np.ascontiguousarray(uv),
                     np.ascontiguousarray(idx), obj, np.asarray(self._obj_mat, dtype=np.int32),
                     list(self.materials), list(self.lights), camera, tuple(env), name)


# ----------------------------------------------------------------------------------------------
# Procedural meshes (all closed and consistently wound outward unless stated)
# ----------------------------------------------------------------------------------------------

def icosphere(subdiv: int) -> Mesh:
    """Unit icosphere with 20*4^subdiv triangles and smooth (radial) normals."""
    t = (1.0 + math.sqrt(5.0)) / 2.0
    verts = [(-1, t, 0), (1, t, 0), (-1, -t, 0), (1, -t, 0), (0, -1, t), (0, 1, t), (0, -1, -t), (0, 1, -t),
             (t, 0, -1), (t, 0, 1), (-t, 0, -1), (-t, 0, 1)]
    faces = [(0, 11, 5), (0, 5, 1), (0, 1, 7), (0, 7, 10), (0, 10, 11), (1, 5, 9), (5, 11, 4), (11, 10, 2),
             (10, 7, 6), (7, 1, 8), (3, 9, 4), (3, 4, 2), (3, 2, 6), (3, 6, 8), (3, 8, 9), (4, 9, 5),
             (2, 4, 11), (6, 2, 10), (8, 6, 7), (9, 8, 1)]
    v = [np.asarray(p, dtype=np.float64) / np.linalg.norm(p) for p in verts]
    for _ in range(subdiv):
        cache = {}

        def mid(a, b):
            key = (min(a, b), max(a, b))
            if key not in cache:
                m = v[a] + v[b]
                v.append(m / np.linalg.norm(m))
                cache[key] = len(v) - 1
            return cache[key]

        nf = []
        for a, b, c in faces:
            ab, bc, ca = mid(a, b), mid(b, c), mid(c, a)
            nf += [(a, ab, ca), (b, bc, ab), (c, ca, bc), (ab, bc, ca)]
        faces = nf
    p = np.asarray(v)
    return Mesh(p, np.asarray(faces, dtype=np.int64), p.copy(), None)


def quad(corner, edge_u, edge_v, flat=True) -> Mesh:
    """Two triangles spanning corner + s*edge_u + t*edge_v, winding normal edge_u x edge_v.

    uv = (s*|edge_u|, t*|edge_v|) in metres."""
    c, eu, ev = (np.asarray(x, dtype=np.float64) for x in (corner, edge_u, edge_v))
    p = np.stack([c, c + eu, c + eu + ev, c + ev])
    lu, lv = np.linalg.norm(eu), np.linalg.norm(ev)
    uv = np.asarray([[0, 0], [lu, 0], [lu, lv], [0, lv]], dtype=np.float64)
    idx = np.asarray([[0, 1, 2], [0, 2, 3]], dtype=np.int64)
    return Mesh(p, idx, np.zeros((4, 3)), uv)


def box(lo, hi) -> Mesh:
    """Axis-aligned closed box, flat faces, outward winding."""
    lo, hi = np.asarray(lo, dtype=np.float64), np.asarray(hi, dtype=np.float64)
    d = hi - lo
    ex, ey, ez = np.array([d[0], 0, 0]), np.array([0, d[1], 0]), np.array([0, 0, d[2]])
    faces = [quad(lo, ey, ex), quad(lo + ez, ex, ey),  # -z, +z
             quad(lo, ez, ey), quad(lo + ex, ey, ez),  # -x, +x
             quad(lo, ex, ez), quad(lo + ey, ez, ex)]  # -y, +y
    return merge(faces)


def merge(meshes) -> Mesh:
    ps, ns, us, ids, off = [], [], [], [], 0
    for m in meshes:
        ps.append(m.positions)
        ns.append(np.zeros_like(m.positions) if m.normals is None else m.normals)
        us.append(np.zeros((m.positions.shape[0], 2)) if m.uvs is None else m.uvs)
        ids.append(m.indices + off)
        off += m.positions.shape[0]
    return Mesh(np.concatenate(ps), np.concatenate(ids), np.concatenate(ns), np.concatenate(us))


def _grid_indices(nu: int, nv: int, wrap_u=True) -> np.ndarray:
    """Quads of an (nv+1) x nu vertex grid (u wraps) as triangle pairs."""
    tris = []
    for j in range(nv):
        for i in range(nu):
            i1 = (i + 1) % nu if wrap_u else i + 1
            a, b = j * nu + i, j * nu + i1
            c, d = (j + 1) * nu + i1, (j + 1) * nu + i
            tris.append((a, b, c))
            tris.append((a, c, d))
    return np.asarray(tris, dtype=np.int64)


def torus(major: float, minor: float, nu: int, nv: int) -> Mesh:
    """Torus around +y with 2*nu*nv triangles and analytic smooth normals."""
    u = np.arange(nu) * (2 * math.pi / nu)
    v = np.arange(nv + 1) * (2 * math.pi / nv)
    vv, uu = np.meshgrid(v, u, indexing="ij")
    cx, sx = np.cos(uu), np.sin(uu)
    n = np.stack([np.cos(vv) * cx, np.sin(vv), np.cos(vv) * sx], -1)
    p = np.stack([(major + minor * np.cos(vv)) * cx, minor * np.sin(vv), (major + minor * np.cos(vv)) * sx], -1)
    idx = _grid_indices(nu, nv)
    # the last ring duplicates the first (v = 2 pi); remap it onto ring 0 so the mesh is closed
    idx = np.where(idx >= nv * nu, idx - nv * nu, idx)
    p, n = p[:nv].reshape(-1, 3), n[:nv].reshape(-1, 3)
    # outward winding: flip if needed so (v1-v0)x(v2-v0) agrees with the normal of v0
    e = np.cross(p[idx[0, 1]] - p[idx[0, 0]], p[idx[0, 2]] - p[idx[0, 0]])
    if np.dot(e, n[idx[0, 0]]) < 0:
        idx = idx[:, [0, 2, 1]]
    return Mesh(p, idx, n, None)


def _revolve(profile: np.ndarray, normals2d: np.ndarray, seg: int) -> Mesh:
    """Surface of revolution about +y of a polyline profile (r, y) with per-vertex 2-D normals."""
    ang = np.arange(seg) * (2 * math.pi / seg)
    ca, sa = np.cos(ang), np.sin(ang)
    k = profile.shape[0]
    p = np.zeros((k, seg, 3))
    n = np.zeros((k, seg, 3))
    p[:, :, 0] = profile[:, :1] * ca
    p[:, :, 1] = profile[:, 1:2]
    p[:, :, 2] = profile[:, :1] * sa
    n[:, :, 0] = normals2d[:, :1] * ca
    n[:, :, 1] = normals2d[:, 1:2]
    n[:, :, 2] = normals2d[:, :1] * sa
    idx = _grid_indices(seg, k - 1)
    return Mesh(p.reshape(-1, 3), idx, n.reshape(-1, 3), None)


def _orient_outward(m: Mesh, center) -> Mesh:
    """Flip every triangle whose winding normal points toward ``center`` (star-shaped pieces only)."""
    p, idx = m.positions, m.indices
    e = np.cross(p[idx[:, 1]] - p[idx[:, 0]], p[idx[:, 2]] - p[idx[:, 0]])
    c = (p[idx[:, 0]] + p[idx[:, 1]] + p[idx[:, 2]]) / 3.0 - np.asarray(center)
    flip = np.einsum("ij,ij->i", e, c) < 0
    idx = idx.copy()
    idx[flip] = idx[flip][:, [0, 2, 1]]
    return Mesh(p, idx, m.normals, m.uvs)


def _cap(radius_in: float, radius_out: float, y: float, seg: int, up: bool) -> Mesh:
    """Flat annulus (or disk when radius_in == 0) at height y facing +y (up) or -y."""
    ang = np.arange(seg) * (2 * math.pi / seg)
    ca, sa = np.cos(ang), np.sin(ang)
    outer = np.stack([radius_out * ca, np.full(seg, y), radius_out * sa], -1)
    tris = []
    if radius_in <= 0:
        p = np.concatenate([outer, [[0.0, y, 0.0]]])
        for i in range(seg):
            tris.append((seg, i, (i + 1) % seg))
    else:
        inner = np.stack([radius_in * ca, np.full(seg, y), radius_in * sa], -1)
        p = np.concatenate([outer, inner])
        for i in range(seg):
            j = (i + 1) % seg
            tris.append((i, seg + i, seg + j))
            tris.append((i, seg + j, j))
    idx = np.asarray(tris, dtype=np.int64)
    e = np.cross(p[idx[0, 1]] - p[idx[0, 0]], p[idx[0, 2]] - p[idx[0, 0]])
    if (e[1] > 0) != up:
        idx = idx[:, [0, 2, 1]]
    return Mesh(p, idx, np.zeros_like(p), None)


def hollow_cylinder(radius: float, height: float, wall: float, base: float, seg: int, rings: int) -> Mesh:
    """Open-topped drinking glass: outer wall, outer bottom, inner bottom, inner wall, rim.

    Axis +y, bottom at y=0.  Walls carry smooth radial normals, caps are flat."""
    ri = radius * (1.0 - wall)
    ys = np.linspace(0.0, height, rings + 1)
    outer = _revolve(np.stack([np.full(rings + 1, radius), ys], -1),
                     np.stack([np.ones(rings + 1), np.zeros(rings + 1)], -1), seg)
    yi = np.linspace(base, height, rings + 1)
    inner = _revolve(np.stack([np.full(rings + 1, ri), yi], -1),
                     np.stack([-np.ones(rings + 1), np.zeros(rings + 1)], -1), seg)
    outer = _orient_outward(outer, (0.0, 0.0, 0.0))
    # interior wall faces the axis: its outward (from the glass material) normal points inward
    p, idx = inner.positions, inner.indices
    e = np.cross(p[idx[:, 1]] - p[idx[:, 0]], p[idx[:, 2]] - p[idx[:, 0]])
    c = (p[idx[:, 0]] + p[idx[:, 1]] + p[idx[:, 2]]) / 3.0
    c[:, 1] = 0.0
    flip = np.einsum("ij,ij->i", e, c) > 0
    idx = idx.copy()
    idx[flip] = idx[flip][:, [0, 2, 1]]
    inner = Mesh(p, idx, inner.normals, None)
    bottom = _cap(0.0, radius, 0.0, seg, up=False)
    floor_in = _cap(0.0, ri, base, seg, up=True)
    rim = _cap(ri, radius, height, seg, up=True)
    return merge([outer, inner, bottom, floor_in, rim])


def superellipsoid(e1: float, e2: float, nu: int, nv: int) -> Mesh:
    """Barr (1981) superellipsoid |x|^(2/e2)+|z|^(2/e2))^(e2/e1)+|y|^(2/e1)=1, axis +y.

    Rings between the poles form a grid, the poles are triangle fans; normals are the analytic ones."""
    def sp(w, e):
        return np.sign(w) * np.abs(w) ** e

    eta = -math.pi / 2 + np.arange(1, nv) * (math.pi / nv)  # exclude the poles
    om = np.arange(nu) * (2 * math.pi / nu) - math.pi
    E, O = np.meshgrid(eta, om, indexing="ij")
    ce, se, co, so = np.cos(E), np.sin(E), np.cos(O), np.sin(O)
    p = np.stack([sp(ce, e1) * sp(co, e2), sp(se, e1), sp(ce, e1) * sp(so, e2)], -1).reshape(-1, 3)
    n = np.stack([sp(ce, 2 - e1) * sp(co, 2 - e2), sp(se, 2 - e1), sp(ce, 2 - e1) * sp(so, 2 - e2)], -1)
    n = n.reshape(-1, 3)
    n /= np.maximum(np.linalg.norm(n, axis=1, keepdims=True), 1e-30)
    idx = list(map(tuple, _grid_indices(nu, nv - 2)))
    south, north = len(p), len(p) + 1
    top = (nv - 2) * nu
    for i in range(nu):
        j = (i + 1) % nu
        idx.append((south, j, i))
        idx.append((north, top + i, top + j))
    p = np.concatenate([p, [[0.0, -1.0, 0.0], [0.0, 1.0, 0.0]]])
    n = np.concatenate([n, [[0.0, -1.0, 0.0], [0.0, 1.0, 0.0]]])
    return _orient_outward(Mesh(p, np.asarray(idx, dtype=np.int64), n, None), (0.0, 0.0, 0.0))


# ----------------------------------------------------------------------------------------------
# Poses
# ----------------------------------------------------------------------------------------------

def random_rotation(rng: np.random.Generator) -> np.ndarray:
    """Uniform random rotation (Shoemake's quaternion from three uniforms)."""
    u1, u2, u3 = rng.random(3)
    a, b = math.sqrt(1 - u1), math.sqrt(u1)
    q = np.array([a * math.sin(2 * math.pi * u2), a * math.cos(2 * math.pi * u2),
                  b * math.sin(2 * math.pi * u3), b * math.cos(2 * math.pi * u3)])
    x, y, z, w = q
    return np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - z * w), 2 * (x * z + y * w)],
                     [2 * (x * y + z * w), 1 - 2 * (x * x + z * z), 2 * (y * z - x * w)],
                     [2 * (x * z - y * w), 2 * (y * z + x * w), 1 - 2 * (x * x + y * y)]])


def _family_mesh(family: str, tris: int, rng: np.random.Generator) -> Mesh:
    """One of the four transparent families with roughly ``tris`` triangles, unit-ish size."""
    if family == "sphere":
        s = max(0, int(round(math.log(max(tris, 20) / 20.0, 4))))
        return icosphere(s)
    if family == "torus":
        nv = max(8, int(round(math.sqrt(tris / 2 / 2.5))))
        nu = max(8, int(round(tris / 2 / nv)))
        return torus(0.7, 0.3, nu, nv)
    if family == "cylinder":
        seg = max(12, int(round(math.sqrt(tris / 4 * 5))))
        rings = max(1, int(round((tris - 5 * seg) / (4 * seg))))
        return hollow_cylinder(0.6, 1.6, 0.08, 0.12, seg, rings)
    if family == "superellipsoid":
        nv = max(6, int(round(math.sqrt(tris / 2 / 1.6))))
        nu = max(8, int(round(tris / 2 / nv)))
        e1, e2 = rng.uniform(0.3, 2.0, size=2)
        return superellipsoid(float(e1), float(e2), nu, nv)
    raise ValueError(family)


FAMILIES = ("sphere", "cylinder", "torus", "superellipsoid")


def _place_objects(b: SceneBuilder, meshes_mats, rng, floor_y, xz_range, scale_range, max_tries=200):
    """Random rotation, scale and xz position; rest on the floor (1 mm gap); reject 3-D overlaps
    of the objects' world-space bounding boxes."""
    placed = []  # (lo, hi) world boxes
    for mesh, mat in meshes_mats:
        for _ in range(max_tries):
            rot = random_rotation(rng)
            s = rng.uniform(*scale_range)
            m = mesh.transformed(rot, s, (0.0, 0.0, 0.0))
            lo, hi = m.positions.min(0), m.positions.max(0)
            xz = rng.uniform(-xz_range, xz_range, size=2)
            off = np.array([xz[0] - 0.5 * (lo[0] + hi[0]), floor_y + 1e-3 - lo[1], xz[1] - 0.5 * (lo[2] + hi[2])])
            wlo, whi = lo + off, hi + off
            if all(np.any(wlo > h2) or np.any(whi < l2) for l2, h2 in placed):
                placed.append((wlo, whi))
                b.add(Mesh(m.positions + off, m.indices, m.normals, None), mat)
                break
        else:
            raise RuntimeError("could not place object without overlap")


def _backdrop(b: SceneBuilder, floor_y=0.0, wall_z=-4.0, size=20.0, height=10.0):
    mat = b.material(Material(MAT_DIFFUSE, albedo=(0.25, 0.25, 0.25), albedo2=(0.75, 0.75, 0.75),
                              checker_scale=4.0))
    h = size / 2
    b.add(quad((-h, floor_y, -h), (0, 0, size), (size, 0, 0)), mat)  # floor, normal +y
    b.add(quad((-h, floor_y, wall_z), (size, 0, 0), (0, height, 0)), mat)  # back wall, normal +z


# ----------------------------------------------------------------------------------------------
# The workloads
# ----------------------------------------------------------------------------------------------

def ball_on_plane(width=64, height=64, subdiv=3, ior=1.5, light_pos=(2.0, 4.0, 2.0), intensity=20.0) -> Scene:
    """Glass icosphere (radius 1, 1280 triangles at subdiv 3, IOR 1.5) on a grey plane (albedo 0.5),
    one point light at (2,4,2), pinhole camera 64x64 from (0,1,4) looking at the origin, vfov 40 deg."""
    b = SceneBuilder()
    glass = b.material(Material(MAT_DIELECTRIC, cauchy_a=ior, cauchy_b=0.0))
    grey = b.material(Material(MAT_DIFFUSE, albedo=(0.5, 0.5, 0.5)))
    b.add(icosphere(subdiv), glass)
    b.add(quad((-10, -1, -10), (0, 0, 20), (20, 0, 0)), grey)
    b.lights.append(Light(LIGHT_POINT, tuple(light_pos), power=(intensity,) * 3))
    cam = Camera((0.0, 1.0, 4.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), 40.0, width, height)
    return b.build(cam, name=f"ball_on_plane_{width}x{height}")


def guide_sphere(scene: Scene) -> tuple:
    """(cx, cy, cz, r): a sphere enclosing every dielectric triangle, as float32 values (the
    radius rounded up so that the rounded sphere still encloses them), or a zero radius when the
    scene has no glass.  The light tracer's guided emission aims into this sphere."""
    kinds = np.array([m.kind for m in scene.materials])
    tri_mat = np.asarray(scene.object_material)[np.asarray(scene.tri_object)]
    sel = kinds[tri_mat] == MAT_DIELECTRIC
    if not sel.any():
        return (0.0, 0.0, 0.0, 0.0)
    v = np.asarray(scene.positions, np.float64)[np.asarray(scene.indices)[sel].ravel()]
    c = (v.min(axis=0) + v.max(axis=0)) * 0.5
    c32 = c.astype(np.float32).astype(np.float64)
    r = np.sqrt(((v - c32) ** 2).sum(axis=1)).max() * (1.0 + 1e-5) + 1e-6
    r32 = np.nextafter(np.float32(r), np.float32(np.inf))
    return (float(c32[0]), float(c32[1]), float(c32[2]), float(r32))


def denoise_scene(seed: int, width=64, height=64) -> Scene:
    """A ball-on-plane scene with randomised parameters, for denoiser training pairs: glass
    icosphere (1280 tris) of radius 0.6-1.2 resting on the plane y = -1 near the origin, IOR
    uniform in [1.33, 1.9], plane albedo 0.3-0.8 (checkered half the time), point light at a
    random position 3-5 m up, camera jittered around (0, 1, 4)."""
    rng = np.random.default_rng(20_000 + seed)
    b = SceneBuilder()
    ior = float(rng.uniform(1.33, 1.9))
    glass = b.material(Material(MAT_DIELECTRIC, cauchy_a=ior, cauchy_b=0.0))
    a = float(rng.uniform(0.3, 0.8))
    if rng.random() < 0.5:
        a2 = float(rng.uniform(0.1, 0.9))
        floor = b.material(Material(MAT_DIFFUSE, albedo=(a, a, a), albedo2=(a2, a2, a2),
                                    checker_scale=float(rng.uniform(1.0, 4.0))))
    else:
        floor = b.material(Material(MAT_DIFFUSE, albedo=(a, a, a)))
    r = float(rng.uniform(0.6, 1.2))
    centre = (float(rng.uniform(-0.6, 0.6)), r - 1.0, float(rng.uniform(-0.6, 0.6)))
    b.add(icosphere(3).transformed(np.eye(3), r, centre), glass)
    b.add(quad((-10, -1, -10), (0, 0, 20), (20, 0, 0)), floor)
    lp = (float(rng.uniform(-3, 3)), float(rng.uniform(3, 5)), float(rng.uniform(-3, 3)))
    power = 20.0 * (lp[0] ** 2 + (lp[1] + 1) ** 2 + lp[2] ** 2) / 29.0  # about the same irradiance at the origin
    b.lights.append(Light(LIGHT_POINT, lp, power=(power,) * 3))
    eye = (float(rng.normal(0, 0.3)), 1.0 + float(rng.normal(0, 0.2)), 4.0 + float(rng.normal(0, 0.3)))
    look = (float(rng.normal(0, 0.15)), float(rng.normal(-0.2, 0.1)), 0.0)
    cam = Camera(eye, look, (0.0, 1.0, 0.0), 40.0, width, height)
    return b.build(cam, name=f"denoise_scene_s{seed}_{width}x{height}")


def glass_scene(seed=0, width=512, height=512, n_objects=4, tris_per_object=20480, families=FAMILIES,
                cauchy=(1.5, 0.004), light_size=1.0, light_radiance=20.0) -> Scene:
    """Several transparent meshes (sphere, hollow cylinder glass, torus, superellipsoid) with random pose
    and scale over a checkered floor and back wall, lit by a downward rect light 4 m up."""
    rng = np.random.default_rng(seed)
    b = SceneBuilder()
    _backdrop(b)
    items = []
    for i in range(n_objects):
        fam = families[i % len(families)]
        mat = b.material(Material(MAT_DIELECTRIC, cauchy_a=cauchy[0], cauchy_b=cauchy[1]))
        items.append((_family_mesh(fam, tris_per_object, rng), mat))
    _place_objects(b, items, rng, floor_y=0.0, xz_range=2.0, scale_range=(0.5, 1.0))
    h = light_size / 2
    b.add_rect_light((-h, 4.0, -h), (light_size, 0, 0), (0, 0, light_size), (light_radiance,) * 3)
    cam = Camera((0.0, 2.5, 6.0), (0.0, 0.3, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return b.build(cam, name=f"glass_scene_s{seed}_{width}x{height}")


def dense_scene(seed=0, width=1024, height=1024, n_objects=16, tris_per_object=62500, cauchy=(1.5, 0.004),
                light_size=1.0, light_radiance=20.0) -> Scene:
    """The dense variant of glass_scene: n_objects transparent meshes of the four families (about 1M
    triangles at the defaults) spread over a 6 x 6 m patch of the checkered floor, smaller
    (scale 0.3-0.55) so that they crowd the view and overlap in the image, same backdrop and rect light;
    the camera stands back to frame them all."""
    rng = np.random.default_rng(50_000 + seed)
    b = SceneBuilder()
    _backdrop(b)
    items = []
    for i in range(n_objects):
        fam = FAMILIES[i % len(FAMILIES)]
        mat = b.material(Material(MAT_DIELECTRIC, cauchy_a=cauchy[0], cauchy_b=cauchy[1]))
        items.append((_family_mesh(fam, tris_per_object, rng), mat))
    _place_objects(b, items, rng, floor_y=0.0, xz_range=2.6, scale_range=(0.3, 0.55), max_tries=2000)
    h = light_size / 2
    b.add_rect_light((-h, 4.0, -h), (light_size, 0, 0), (0, 0, light_size), (light_radiance,) * 3)
    cam = Camera((0.0, 3.4, 7.0), (0.0, 0.2, 0.0), (0.0, 1.0, 0.0), 45.0, width, height)
    return b.build(cam, name=f"dense_scene_s{seed}_{width}x{height}")


def random_scene(seed: int, resolutions=(128, 256, 512, 1024), tri_range=(1000, 200000)) -> Scene:
    """A randomised dataset scene: 1-6 transparent objects, total triangles uniform in tri_range,
    random IOR in [1.33, 1.9] per object, random resolution, point or rect light."""
    rng = np.random.default_rng(10_000 + seed)
    res = int(rng.choice(resolutions))
    n_obj = int(rng.integers(1, 7))
    total = int(rng.integers(tri_range[0], tri_range[1] + 1))
    b = SceneBuilder()
    _backdrop(b)
    items = []
    for i in range(n_obj):
        fam = FAMILIES[int(rng.integers(0, 4))]
        mat = b.material(Material(MAT_DIELECTRIC, cauchy_a=float(rng.uniform(1.33, 1.9)), cauchy_b=0.0))
        items.append((_family_mesh(fam, max(20, total // n_obj), rng), mat))
    _place_objects(b, items, rng, floor_y=0.0, xz_range=2.5, scale_range=(0.4, 1.0))
    if rng.random() < 0.5:
        b.lights.append(Light(LIGHT_POINT, (float(rng.uniform(-3, 3)), 4.0, float(rng.uniform(-1, 3))),
                              power=(20.0,) * 3))
    else:
        s = float(rng.uniform(0.3, 1.5))
        b.add_rect_light((-s / 2, 4.0, -s / 2), (s, 0, 0), (0, 0, s), (20.0,) * 3)
    cam = Camera((float(rng.uniform(-1, 1)), 2.5, 6.0), (0.0, 0.3, 0.0), (0.0, 1.0, 0.0), 45.0, res, res)
    return b.build(cam, name=f"random_scene_{seed}")
