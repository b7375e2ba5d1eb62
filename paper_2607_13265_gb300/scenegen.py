"""Seeded synthetic scenes and jobs for the polarized path tracer.

This module produces INPUT DATA only: triangle meshes, spheres, materials,
quad lights, cameras, textures and render jobs, as plain numpy arrays.  It
holds none of the transport arithmetic (no Mueller matrices, no sampling, no
intersection code).  Both the CUDA library and the FP64 CPU oracle consume the
same arrays, each packing them in its own way.

Scene conventions shared by both consumers (data layout, not method):

* ``verts`` float64 [V,3], ``uvs`` float64 [V,2], ``tris`` int32 [F,3] with
  counter-clockwise winding giving the geometric normal
  ``(v1-v0) x (v2-v0)``; ``tri_mat`` int32 [F]; ``tri_light`` int32 [F] (-1 or
  the index of the quad light the triangle belongs to).
* ``spheres`` float64 [S,4] (centre, radius), ``sph_mat`` int32 [S].
* ``lights`` float64 [L,9]: parallelogram corner o, edges e1, e2; the light
  emits on the side of ``e1 x e2``.  Its two triangles are part of the mesh.
* ``cameras`` float64 [C,10]: origin, target, up, vertical field of view (deg).
* textures live in one flat parameter vector ``params['tex']``; ``tex_desc``
  int64 [T,4] = (offset, width, height, channels), row-major [h][w][ch].
* differentiable parameters: ``tex``, ``ior`` [n_ior], ``le`` [L,3,4] (Stokes
  per RGB channel in the emitter frame), ``sheet`` [n_sheet] (sheet axis
  angles, radians); per-job camera-filter angles live in the job.

Material types (``MAT_*``) name the optical elements of Sec. 3.3 / 4.1 of the
paper (ideal depolarizer, Fresnel dielectric, conductor, linear polarizer,
retarder) plus the GGX pBRDFs used by the synthetic workloads.
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

MAT_DIFFUSE = 0
MAT_SMOOTH_DIELECTRIC = 1
MAT_CONDUCTOR_GGX = 2
MAT_PLASTIC_GGX = 3
MAT_POLARIZER_SHEET = 4
MAT_RETARDER_SHEET = 5
MAT_EMITTER = 6

FILTER_NONE = 0
FILTER_POLARIZER = 1          # linear polarizer P(theta) in front of the sensor
FILTER_QWP_POLARIZER = 2      # quarter-wave plate Q(pi/2, 0) then P(theta)


@dataclass
class Material:
    type: int
    albedo_tex: int = -1
    rough_tex: int = -1
    ior_index: int = -1
    eta_re: float = 1.0
    eta_im: float = 0.0
    sheet_index: int = -1
    t1: tuple = (1.0, 0.0, 0.0)
    t2: tuple = (0.0, 1.0, 0.0)
    retard: float = 0.0
    normal_tex: int = -1      # tangent-space normal map (3 channels, n = 2 c - 1), triangles with UVs
    emission: float = 0.0     # constant unpolarized emission (both sides), not differentiable


@dataclass
class Job:
    camera: int
    width: int
    height: int
    spp: int
    max_depth: int
    seed: int = 0
    pass_id: int = 0
    stream: int = 0
    filter: int = FILTER_NONE
    thetas: list = field(default_factory=list)   # radians; one output image per angle

    @property
    def num_angles(self) -> int:
        return max(1, len(self.thetas)) if self.filter != FILTER_NONE else 1

    @property
    def num_pixels(self) -> int:
        return self.width * self.height

    @property
    def num_paths(self) -> int:
        return self.width * self.height * self.spp


class Scene:
    """Container for one seeded synthetic scene (arrays + initial parameters)."""

    def __init__(self):
        self._verts: list = []
        self._uvs: list = []
        self._tris: list = []
        self._tri_mat: list = []
        self._tri_light: list = []
        self.spheres = np.zeros((0, 4))
        self.sph_mat = np.zeros((0,), np.int32)
        self.materials: list[Material] = []
        self._lights: list = []
        self._le: list = []
        self._tex_blocks: list = []
        self._tex_desc: list = []
        self.tex_differentiable: list[bool] = []
        self.ior: list[float] = []
        self.sheet: list[float] = []
        self._cameras: list = []
        self.eps = None
        self._nv = 0

    # ---------------------------------------------------------------- builders
    def add_texture(self, data: np.ndarray, differentiable: bool = False) -> int:
        data = np.asarray(data, np.float64)
        if data.ndim == 2:
            data = data[:, :, None]
        h, w, ch = data.shape
        off = sum(b.size for b in self._tex_blocks)
        self._tex_blocks.append(data.reshape(-1))
        self._tex_desc.append((off, w, h, ch))
        self.tex_differentiable.append(bool(differentiable))
        return len(self._tex_desc) - 1

    def add_const_texture(self, value, differentiable: bool = False) -> int:
        v = np.atleast_1d(np.asarray(value, np.float64))
        return self.add_texture(v.reshape(1, 1, -1), differentiable)

    def add_material(self, m: Material) -> int:
        self.materials.append(m)
        return len(self.materials) - 1

    def add_ior(self, value: float) -> int:
        self.ior.append(float(value))
        return len(self.ior) - 1

    def add_mesh(self, verts, tris, mat: int, uvs=None, light: int = -1):
        verts = np.asarray(verts, np.float64).reshape(-1, 3)
        tris = np.asarray(tris, np.int64).reshape(-1, 3)
        if uvs is None:
            uvs = np.zeros((len(verts), 2))
        self._verts.append(verts)
        self._uvs.append(np.asarray(uvs, np.float64).reshape(-1, 2))
        self._tris.append(tris + self._nv)
        self._tri_mat.append(np.full(len(tris), mat, np.int32))
        self._tri_light.append(np.full(len(tris), light, np.int32))
        self._nv += len(verts)

    def add_quad(self, o, e1, e2, mat: int, light: int = -1, uv=True):
        """Parallelogram o, o+e1, o+e1+e2, o+e2 as two triangles; normal = e1 x e2."""
        o, e1, e2 = (np.asarray(x, np.float64) for x in (o, e1, e2))
        v = np.stack([o, o + e1, o + e1 + e2, o + e2])
        t = np.array([[0, 1, 2], [0, 2, 3]])
        uvs = np.array([[0, 0], [1, 0], [1, 1], [0, 1]], np.float64) if uv else None
        self.add_mesh(v, t, mat, uvs, light)

    def add_light(self, o, e1, e2, le) -> int:
        """Quad light: geometry as two emitter triangles, Stokes radiance le[3][4]."""
        idx = len(self._lights)
        mat = self.add_material(Material(MAT_EMITTER))
        self._lights.append(np.concatenate([o, e1, e2]).astype(np.float64))
        le = np.asarray(le, np.float64)
        if le.ndim == 0:
            le = np.array([[float(le), 0, 0, 0]] * 3)
        elif le.shape == (4,):
            le = np.tile(le, (3, 1))
        self._le.append(le.reshape(3, 4))
        self.add_quad(o, e1, e2, mat, light=idx)
        return idx

    def add_sphere(self, c, r, mat: int):
        self.spheres = np.concatenate([self.spheres, np.array([[*c, r]], np.float64)])
        self.sph_mat = np.concatenate([self.sph_mat, np.array([mat], np.int32)])

    def add_camera(self, origin, target, up=(0, 1, 0), vfov_deg=40.0) -> int:
        self._cameras.append(np.array([*origin, *target, *up, vfov_deg], np.float64))
        return len(self._cameras) - 1

    # ---------------------------------------------------------------- arrays
    @property
    def verts(self):
        return np.concatenate(self._verts) if self._verts else np.zeros((0, 3))

    @property
    def uvs(self):
        return np.concatenate(self._uvs) if self._uvs else np.zeros((0, 2))

    @property
    def tris(self):
        return (np.concatenate(self._tris) if self._tris else np.zeros((0, 3))).astype(np.int32)

    @property
    def tri_mat(self):
        return np.concatenate(self._tri_mat) if self._tri_mat else np.zeros((0,), np.int32)

    @property
    def tri_light(self):
        return np.concatenate(self._tri_light) if self._tri_light else np.zeros((0,), np.int32)

    @property
    def lights(self):
        return np.stack(self._lights) if self._lights else np.zeros((0, 9))

    @property
    def cameras(self):
        return np.stack(self._cameras)

    @property
    def tex_desc(self):
        return np.array(self._tex_desc, np.int64).reshape(-1, 4)

    def params(self) -> dict:
        """Initial differentiable parameters (float64 copies)."""
        return {
            "tex": (np.concatenate(self._tex_blocks) if self._tex_blocks else np.zeros(0)).astype(np.float64),
            "ior": np.array(self.ior, np.float64),
            "le": (np.stack(self._le) if self._le else np.zeros((0, 3, 4))).astype(np.float64),
            "sheet": np.array(self.sheet, np.float64),
        }

    def extent(self) -> float:
        pts = [self.verts] if len(self.verts) else []
        if len(self.spheres):
            c, r = self.spheres[:, :3], self.spheres[:, 3:4]
            pts += [c - r, c + r]
        allp = np.concatenate(pts)
        return float(np.max(allp.max(0) - allp.min(0)))

    def ray_eps(self) -> float:
        return self.eps if self.eps is not None else 1e-4 * self.extent()

    @property
    def num_triangles(self) -> int:
        return int(self.tris.shape[0])


# ============================================================ procedural meshes
def icosahedron():
    t = (1.0 + 5 ** 0.5) / 2.0
    v = np.array([[-1, t, 0], [1, t, 0], [-1, -t, 0], [1, -t, 0],
                  [0, -1, t], [0, 1, t], [0, -1, -t], [0, 1, -t],
                  [t, 0, -1], [t, 0, 1], [-t, 0, -1], [-t, 0, 1]], np.float64)
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    f = np.array([[0, 11, 5], [0, 5, 1], [0, 1, 7], [0, 7, 10], [0, 10, 11],
                  [1, 5, 9], [5, 11, 4], [11, 10, 2], [10, 7, 6], [7, 1, 8],
                  [3, 9, 4], [3, 4, 2], [3, 2, 6], [3, 6, 8], [3, 8, 9],
                  [4, 9, 5], [2, 4, 11], [6, 2, 10], [8, 6, 7], [9, 8, 1]], np.int64)
    return v, f


def geodesic_sphere(freq: int):
    """Class-I geodesic icosphere: 20*freq^2 triangles, 10*freq^2+2 vertices, unit radius."""
    v0, f0 = icosahedron()
    pts, faces = [], []
    base = 0
    for (a, b, c) in f0:
        A, B, C = v0[a], v0[b], v0[c]
        idx = {}
        loc = []
        for i in range(freq + 1):
            for j in range(freq + 1 - i):
                k = freq - i - j
                p = (A * k + B * i + C * j) / freq
                idx[(i, j)] = base + len(loc)
                loc.append(p)
        for i in range(freq):
            for j in range(freq - i):
                faces.append((idx[(i, j)], idx[(i + 1, j)], idx[(i, j + 1)]))
                if j < freq - i - 1:
                    faces.append((idx[(i + 1, j)], idx[(i + 1, j + 1)], idx[(i, j + 1)]))
        pts.extend(loc)
        base += len(loc)
    pts = np.array(pts)
    pts /= np.linalg.norm(pts, axis=1, keepdims=True)
    faces = np.array(faces, np.int64)
    # merge duplicated edge vertices
    key = np.round(pts * 1e9).astype(np.int64)
    _, first, inv = np.unique(key, axis=0, return_index=True, return_inverse=True)
    inv = inv.reshape(-1)
    verts = pts[first]
    faces = inv[faces]
    # orient outward
    n = np.cross(verts[faces[:, 1]] - verts[faces[:, 0]], verts[faces[:, 2]] - verts[faces[:, 0]])
    flip = np.einsum("ij,ij->i", n, verts[faces].mean(1)) < 0
    faces[flip] = faces[flip][:, [0, 2, 1]]
    return verts, faces


class Perlin:
    """Improved gradient noise (Perlin 2002) with a seeded permutation table."""

    _G = np.array([[1, 1, 0], [-1, 1, 0], [1, -1, 0], [-1, -1, 0], [1, 0, 1], [-1, 0, 1],
                   [1, 0, -1], [-1, 0, -1], [0, 1, 1], [0, -1, 1], [0, 1, -1], [0, -1, -1],
                   [1, 1, 0], [-1, 1, 0], [0, -1, 1], [0, -1, -1]], np.float64)

    def __init__(self, seed: int):
        p = np.random.default_rng(seed).permutation(256)
        self.p = np.concatenate([p, p]).astype(np.int64)

    @staticmethod
    def _fade(t):
        return t * t * t * (t * (t * 6 - 15) + 10)

    def noise(self, x):
        x = np.asarray(x, np.float64)
        fl = np.floor(x)
        i = fl.astype(np.int64) & 255
        f = x - fl
        u = self._fade(f)
        p = self.p
        out = 0.0
        res = np.zeros(len(x))
        for dx in (0, 1):
            for dy in (0, 1):
                for dz in (0, 1):
                    h = p[p[p[i[:, 0] + dx] + i[:, 1] + dy] + i[:, 2] + dz] & 15
                    g = self._G[h]
                    d = f - np.array([dx, dy, dz], np.float64)
                    dot = np.einsum("ij,ij->i", g, d)
                    wx = u[:, 0] if dx else 1 - u[:, 0]
                    wy = u[:, 1] if dy else 1 - u[:, 1]
                    wz = u[:, 2] if dz else 1 - u[:, 2]
                    res += wx * wy * wz * dot
        return res + out

    def fbm(self, x, octaves=3, base_freq=2.0):
        total = np.zeros(len(x))
        amp, freq = 1.0, base_freq
        for _ in range(octaves):
            total += amp * self.noise(np.asarray(x) * freq)
            amp *= 0.5
            freq *= 2.0
        return total


def displaced_sphere(freq: int, amplitude: float, seed: int, radius: float = 1.0,
                     center=(0, 0, 0), base_freq: float = 2.0):
    """Displaced geodesic sphere with spherical UVs.  Every triangle gets its own three
    vertices so that a triangle crossing the u = 0/1 seam can carry u values on one side
    of it (u + 1 for the small ones; textures wrap), instead of interpolating across the
    whole texture."""
    v, f = geodesic_sphere(freq)
    d = Perlin(seed).fbm(v, octaves=3, base_freq=base_freq)
    v = v * (radius * (1.0 + amplitude * d))[:, None] + np.asarray(center, np.float64)
    n = v - np.asarray(center, np.float64)
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    uv = np.stack([np.arctan2(n[:, 2], n[:, 0]) / (2 * np.pi) + 0.5,
                   np.arccos(np.clip(n[:, 1], -1, 1)) / np.pi], 1)
    tv = v[f].reshape(-1, 3)
    tuv = uv[f].copy()                       # [F, 3, 2]
    u = tuv[:, :, 0]
    seam = (u.max(1) - u.min(1)) > 0.5
    u[seam] = np.where(u[seam] < 0.5, u[seam] + 1.0, u[seam])
    tf = np.arange(3 * len(f), dtype=np.int64).reshape(-1, 3)
    return tv, tf, tuv.reshape(-1, 2)


# ============================================================ workloads
def _cornell_geometry(s: Scene, white, red, green):
    # floor, ceiling, back, left, right walls of the box [-1,1]^3 (front open), normals inward
    s.add_quad((-1, -1, -1), (0, 0, 2), (2, 0, 0), white)   # floor, normal +y
    s.add_quad((-1, 1, -1), (2, 0, 0), (0, 0, 2), white)    # ceiling, normal -y
    s.add_quad((-1, -1, -1), (2, 0, 0), (0, 2, 0), white)   # back, normal +z
    s.add_quad((-1, -1, -1), (0, 2, 0), (0, 0, 2), red)     # left, normal +x
    s.add_quad((1, -1, -1), (0, 0, 2), (0, 2, 0), green)    # right, normal -x


def cornell_box(theta_deg: float = 30.0) -> tuple[Scene, Job]:
    """Small plain workload: 10 wall triangles + a 2-triangle ceiling light, one diffuse
    and one smooth-dielectric sphere, camera behind a linear polarizer; 64x64, 16 spp, depth 4."""
    s = Scene()
    tw = s.add_const_texture([0.7, 0.7, 0.7])
    tr = s.add_const_texture([0.7, 0.1, 0.1])
    tg = s.add_const_texture([0.1, 0.7, 0.1])
    ta = s.add_const_texture([0.7, 0.7, 0.7], differentiable=True)
    white = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tw))
    red = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tr))
    green = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tg))
    _cornell_geometry(s, white, red, green)
    s.add_light((-0.3, 0.999, -0.3), (0.6, 0, 0), (0, 0, 0.6), 10.0)
    diff = s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta))
    glass = s.add_material(Material(MAT_SMOOTH_DIELECTRIC, ior_index=s.add_ior(1.5)))
    s.add_sphere((-0.45, -0.6, -0.3), 0.4, diff)
    s.add_sphere((0.45, -0.6, 0.3), 0.4, glass)
    s.add_camera((0, 0, 3.5), (0, 0, 0), (0, 1, 0), 40.0)
    job = Job(camera=0, width=64, height=64, spp=16, max_depth=4, seed=0,
              filter=FILTER_POLARIZER, thetas=[math.radians(theta_deg)])
    return s, job


def cornell_views(num_views: int = 8, num_angles: int = 64, spp: int = 16, depth: int = 8,
                  sizes=(128, 183, 238, 293, 347, 402, 457, 512)) -> tuple[Scene, list[Job]]:
    """Batched workload: the Cornell scene seen from views orbiting +-20 deg in yaw, each with
    its own square size, all behind a polarizer swept over angles in [0, 180) deg."""
    s, _ = cornell_box()
    s._cameras.clear()
    yaws = np.linspace(-20, 20, num_views)
    thetas = [math.radians(a) for a in np.linspace(0, 180, num_angles, endpoint=False)]
    jobs = []
    for k, yaw in enumerate(yaws):
        y = math.radians(yaw)
        cam = s.add_camera((3.5 * math.sin(y), 0, 3.5 * math.cos(y)), (0, 0, 0), (0, 1, 0), 40.0)
        n = sizes[k % len(sizes)]
        jobs.append(Job(camera=cam, width=n, height=n, spp=spp, max_depth=depth, seed=0,
                        stream=k, filter=FILTER_POLARIZER, thetas=list(thetas)))
    return s, jobs


def icosphere_scene(freq: int = 50, tex_res: int = 128, width: int = 256, spp: int = 64,
                    depth: int = 8) -> tuple[Scene, Job]:
    """Throughput workload: displaced geodesic icosphere (20*freq^2 triangles, Perlin fBm
    amplitude 0.1, permutation seed 1) with a rough conductor pBRDF (eta = 0.2+3.0i) on a
    rough dielectric (IOR 1.5) plane; albedo 128^2x3 ~ U[0.2,0.9] (seed 3) and roughness
    128^2 ~ U[0.05,0.5] (seed 2) maps, both differentiable; one quad light of radiance 10."""
    s = Scene()
    rough = np.random.default_rng(2).uniform(0.05, 0.5, (tex_res, tex_res))
    albedo = np.random.default_rng(3).uniform(0.2, 0.9, (tex_res, tex_res, 3))
    ta = s.add_texture(albedo, differentiable=True)
    tr = s.add_texture(rough, differentiable=True)
    cond = s.add_material(Material(MAT_CONDUCTOR_GGX, albedo_tex=ta, rough_tex=tr, eta_re=0.2, eta_im=3.0))
    plastic = s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=ta, rough_tex=tr, ior_index=s.add_ior(1.5)))
    v, f, uv = displaced_sphere(freq, 0.1, seed=1)
    s.add_mesh(v, f, cond, uv)
    s.add_quad((-4, -1.2, 4), (8, 0, 0), (0, 0, -8), plastic)
    s.add_light((-1.0, 3.0, -1.0), (2, 0, 0), (0, 0, 2), 10.0)
    s.add_camera((0, 0.6, 4.2), (0, -0.2, 0), (0, 1, 0), 40.0)
    job = Job(camera=0, width=width, height=width, spp=spp, max_depth=depth, seed=0)
    return s, job


def rocks_scene(freq: int = 25, num_rocks: int = 8, tex_res: int = 512, width: int = 512,
                spp: int = 32, depth: int = 16, theta_deg: float = 45.0) -> tuple[Scene, Job]:
    """Differentiation workload: 8 displaced geodesic rocks (20*freq^2 triangles each, Perlin
    amplitude 0.25) of rough dielectric with IOR ~ U[1.3,1.7] (seed 4) on a diffuse ground,
    a shared 512^2x3 albedo texture, a differentiable emitter Stokes vector, and a camera
    stack of a quarter-wave plate followed by a linear polarizer at 45 deg; full Stokes out."""
    s = Scene()
    rng = np.random.default_rng(4)
    iors = rng.uniform(1.3, 1.7, num_rocks)
    albedo = np.random.default_rng(5).uniform(0.2, 0.9, (tex_res, tex_res, 3))
    ta = s.add_texture(albedo, differentiable=True)
    trough = s.add_const_texture([0.3])
    tg = s.add_const_texture([0.5, 0.5, 0.5])
    ground = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tg))
    s.add_quad((-6, -1, 6), (12, 0, 0), (0, 0, -12), ground)
    pos_rng = np.random.default_rng(6)
    for r in range(num_rocks):
        m = s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=ta, rough_tex=trough,
                                    ior_index=s.add_ior(iors[r])))
        ang = 2 * math.pi * r / num_rocks
        c = (1.8 * math.cos(ang) + pos_rng.uniform(-0.2, 0.2), -0.55,
             1.8 * math.sin(ang) + pos_rng.uniform(-0.2, 0.2) - 0.5)
        v, f, uv = displaced_sphere(freq, 0.25, seed=100 + r, radius=0.5, center=c)
        s.add_mesh(v, f, m, uv)
    s.add_light((-1.5, 4.0, -1.5), (3, 0, 0), (0, 0, 3), [[8.0, 2.0, 1.0, 0.5]] * 3)
    s.add_camera((0, 2.0, 4.5), (0, -0.5, -0.5), (0, 1, 0), 50.0)
    job = Job(camera=0, width=width, height=width, spp=spp, max_depth=depth, seed=0,
              filter=FILTER_QWP_POLARIZER, thetas=[math.radians(theta_deg)])
    return s, job


def smooth_texture(res: int, lo: float, hi: float, seed: int, channels: int = 1, cells: int = 16) -> np.ndarray:
    """Seeded value noise [res][res] (or [res][res][channels]): a cells x cells grid of
    U[lo, hi] values, bilinearly interpolated with wrap-around at texel centres, so the
    texture varies smoothly (one cell spans res / cells texels) and tiles seamlessly."""
    g = np.random.default_rng(seed).uniform(lo, hi, (cells, cells, channels))
    x = (np.arange(res) + 0.5) * cells / res - 0.5
    i0 = np.floor(x).astype(np.int64)
    f = x - i0
    a, b = i0 % cells, (i0 + 1) % cells
    rows = g[a] * (1 - f)[:, None, None] + g[b] * f[:, None, None]          # [res][cells][ch]
    out = rows[:, a] * (1 - f)[None, :, None] + rows[:, b] * f[None, :, None]  # [res][res][ch]
    return out[:, :, 0] if channels == 1 else out


def large_scene(num_meshes: int = 10, freq: int = 50, tex_res: int = 1024, width: int = 1024,
                spp: int = 128, depth: int = 12, num_angles: int = 16) -> tuple[Scene, Job]:
    """Large workload: 10 displaced meshes (seeds 10..19) mixing diffuse, rough conductor and
    rough dielectric pBRDFs, 3 polarizer sheets and 1 retarder sheet, 4 unpolarized lights,
    1024^2x3 albedo (value noise in [0.2, 0.9], seed 7) + 1024^2 roughness (value noise in
    [0.05, 0.5], seed 8) maps, camera polarizer swept over 16 angles.  The maps vary smoothly
    (smooth_texture): a white-noise roughness map at this resolution changes the roughness
    by up to 0.45 between texels 4e-3 scene units apart, which makes every GGX value, and so
    the FP32 gradients, hypersensitive to the hit position."""
    s = Scene()
    albedo = smooth_texture(tex_res, 0.2, 0.9, 7, 3)
    rough = smooth_texture(tex_res, 0.05, 0.5, 8)
    ta = s.add_texture(albedo, differentiable=True)
    tr = s.add_texture(rough, differentiable=True)
    mats = [s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta)),
            s.add_material(Material(MAT_CONDUCTOR_GGX, albedo_tex=ta, rough_tex=tr, eta_re=0.2, eta_im=3.0)),
            s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=ta, rough_tex=tr, ior_index=s.add_ior(1.5)))]
    tg = s.add_const_texture([0.6, 0.6, 0.6])
    ground = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tg))
    s.add_quad((-8, -1, 8), (16, 0, 0), (0, 0, -16), ground)
    rng = np.random.default_rng(9)
    for k in range(num_meshes):
        ang = 2 * math.pi * k / num_meshes
        c = (2.6 * math.cos(ang), -0.4 + rng.uniform(-0.1, 0.1), 2.6 * math.sin(ang) - 1.0)
        v, f, uv = displaced_sphere(freq, 0.15, seed=10 + k, radius=0.6, center=c)
        s.add_mesh(v, f, mats[k % 3], uv)
    for k in range(4):
        x = -3 + 2 * k
        s.add_light((x - 0.5, 4.0, -1.5), (1, 0, 0), (0, 0, 1), 8.0)
    # thin sheets standing upright in front of some meshes
    for k in range(4):
        typ = MAT_POLARIZER_SHEET if k < 3 else MAT_RETARDER_SHEET
        sidx = len(s.sheet)
        s.sheet.append(math.radians(20.0 + 35.0 * k))
        m = s.add_material(Material(typ, sheet_index=sidx, t1=(1, 0, 0), t2=(0, 1, 0),
                                    retard=math.pi / 2))
        x = -2.4 + 1.6 * k
        s.add_quad((x - 0.6, -1.0, 0.9), (1.2, 0, 0), (0, 1.6, 0), m)
    s.add_camera((0, 1.5, 6.0), (0, -0.3, -0.5), (0, 1, 0), 50.0)
    thetas = [math.radians(a) for a in np.linspace(0, 180, num_angles, endpoint=False)]
    job = Job(camera=0, width=width, height=width, spp=spp, max_depth=depth, seed=0,
              filter=FILTER_POLARIZER, thetas=thetas)
    return s, job


def deep_stack_scene(num_sheets: int = 85, width: int = 1280, height: int = 720, spp: int = 1,
                     depth: int = 128, freq: int = 20, tex_res: int = 256, mesh: bool = True) -> tuple[Scene, Job]:
    """Deep-path workload: a closed diffuse room (every wall albedo 0.8, the floor a
    differentiable tex_res^2x3 map ~ U[0.6,0.9], seed 9) lit by a ceiling quad light of
    radiance 10, holding a rough-conductor displaced sphere (20*freq^2 triangles, eta =
    0.2+3.0i, roughness 0.2) and, between it and the camera, a stack of num_sheets linear
    polarizers (0.6 x 0.6, spacing 0.004) whose axes twist from 0 to 90 deg.  The room is
    closed, so every path runs to max_depth; a path through the stack spends num_sheets
    vertices in it.  Camera polarizer at 0 deg; 1280x720, 1 spp.  mesh=False leaves out the
    conductor (flat surfaces only: long paths then stay identical between FP32 and FP64)."""
    s = Scene()
    floor_alb = np.random.default_rng(9).uniform(0.6, 0.9, (tex_res, tex_res, 3))
    tf = s.add_texture(floor_alb, differentiable=True)
    tw = s.add_const_texture([0.8, 0.8, 0.8])
    troughness = s.add_const_texture([0.2])
    talb = s.add_const_texture([0.9, 0.9, 0.9])
    wall = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tw))
    floor = s.add_material(Material(MAT_DIFFUSE, albedo_tex=tf))
    s.add_quad((-1, -1, -1), (0, 0, 2), (2, 0, 0), floor)   # floor, normal +y
    s.add_quad((-1, 1, -1), (2, 0, 0), (0, 0, 2), wall)     # ceiling, normal -y
    s.add_quad((-1, -1, -1), (2, 0, 0), (0, 2, 0), wall)    # back, normal +z
    s.add_quad((-1, -1, -1), (0, 2, 0), (0, 0, 2), wall)    # left, normal +x
    s.add_quad((1, -1, -1), (0, 0, 2), (0, 2, 0), wall)     # right, normal -x
    s.add_quad((-1, -1, 1), (0, 2, 0), (2, 0, 0), wall)     # front, normal -z
    s.add_light((-0.3, 0.999, -0.3), (0.6, 0, 0), (0, 0, 0.6), 10.0)
    if mesh:
        cond = s.add_material(Material(MAT_CONDUCTOR_GGX, albedo_tex=talb, rough_tex=troughness, eta_re=0.2,
                                       eta_im=3.0))
        v, f, uv = displaced_sphere(freq, 0.05, seed=1, radius=0.35, center=(0.0, -0.5, -0.4))
        s.add_mesh(v, f, cond, uv)
    for k in range(num_sheets):
        s.sheet.append(0.5 * math.pi * k / max(1, num_sheets - 1))
        m = s.add_material(Material(MAT_POLARIZER_SHEET, sheet_index=k, t1=(1, 0, 0), t2=(0, 1, 0)))
        s.add_quad((-0.3, -0.4, 0.3 - 0.004 * k), (0.6, 0, 0), (0, 0.6, 0), m)
    s.add_camera((0, 0, 0.95), (0, -0.1, -1), (0, 1, 0), 60.0)
    job = Job(camera=0, width=width, height=height, spp=spp, max_depth=depth, seed=0,
              filter=FILTER_POLARIZER, thetas=[0.0])
    return s, job


def bump_normal_map(res: int, seed: int, strength: float = 0.6) -> np.ndarray:
    """Tangent-space normal map [res][res][3] of a seeded height field h(u, v) (a sum of six
    periodic waves): n = normalize(-s dh/du, -s dh/dv, 1), stored as (n + 1) / 2."""
    rng = np.random.default_rng(seed)
    u = (np.arange(res) + 0.5) / res
    U, V = np.meshgrid(u, u, indexing="xy")           # row = v, column = u
    hu = np.zeros((res, res))
    hv = np.zeros((res, res))
    for _ in range(6):
        ku, kv = rng.integers(1, 4, 2)
        ph, a = rng.uniform(0, 2 * math.pi), rng.uniform(0.02, 0.05)
        arg = 2 * math.pi * (ku * U + kv * V) + ph
        hu += a * 2 * math.pi * ku * np.cos(arg)
        hv += a * 2 * math.pi * kv * np.cos(arg)
    n = np.stack([-strength * hu, -strength * hv, np.ones_like(hu)], -1)
    n /= np.linalg.norm(n, axis=-1, keepdims=True)
    return 0.5 * (n + 1.0)


def normal_map_scene(width: int = 24, spp: int = 4, depth: int = 4, tex_res: int = 16, flat: bool = False,
                     freq: int = 3) -> tuple[Scene, Job]:
    """Normal-mapped pBRDFs: a rough-dielectric ground quad, a diffuse back wall and a
    rough-conductor geodesic sphere (20*freq^2 triangles), each with its own differentiable
    tangent-space normal map (seeded bumps; flat=True: n = (0, 0, 1) everywhere) and a
    shared differentiable 8x8 albedo texture ~ U[0.3, 0.8] (seed 43) and roughness texture
    ~ U[0.15, 0.45] (seed 44); a quad light of radiance 8 and a camera polarizer at 20 deg."""
    s = Scene()
    maps = [np.full((tex_res, tex_res, 3), (0.5, 0.5, 1.0)) if flat else bump_normal_map(tex_res, 40 + k)
            for k in range(3)]
    tn = [s.add_texture(m_, differentiable=True) for m_ in maps]
    tr = s.add_texture(np.random.default_rng(44).uniform(0.15, 0.45, (8, 8)), differentiable=True)
    ta = s.add_texture(np.random.default_rng(43).uniform(0.3, 0.8, (8, 8, 3)), differentiable=True)
    ground = s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=ta, rough_tex=tr, ior_index=s.add_ior(1.5),
                                     normal_tex=tn[0]))
    wall = s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta, normal_tex=tn[1]))
    cond = s.add_material(Material(MAT_CONDUCTOR_GGX, albedo_tex=ta, rough_tex=tr, eta_re=0.2, eta_im=3.0,
                                   normal_tex=tn[2]))
    s.add_quad((-2, -1, 2), (4, 0, 0), (0, 0, -4), ground)     # normal +y
    s.add_quad((-2, -1, -2), (4, 0, 0), (0, 3, 0), wall)       # normal +z
    v, f, uv = displaced_sphere(freq, 0.0, seed=1, radius=0.6, center=(0.0, -0.3, 0.0))
    s.add_mesh(v, f, cond, uv)
    s.add_light((-0.7, 2.0, -0.7), (1.4, 0, 0), (0, 0, 1.4), 8.0)
    s.add_camera((0.0, 0.6, 3.5), (0.0, -0.3, 0.0), (0, 1, 0), 40.0)
    job = Job(camera=0, width=width, height=width, spp=spp, max_depth=depth, seed=0,
              filter=FILTER_POLARIZER, thetas=[math.radians(20.0)])
    return s, job


# ============================================================ closed-form test scenes
def malus_scene(alpha: float, le: float = 2.0) -> tuple[Scene, Job]:
    """Camera looking down -z through a linear-polarizer sheet (axis at alpha from +x toward
    +y) at a large unpolarized quad light; tiny field of view, depth 2."""
    s = Scene()
    s.sheet.append(float(alpha))
    pol = s.add_material(Material(MAT_POLARIZER_SHEET, sheet_index=0, t1=(1, 0, 0), t2=(0, 1, 0)))
    s.add_quad((-1, -1, 0), (2, 0, 0), (0, 2, 0), pol)
    s.add_light((-2, -2, -1), (4, 0, 0), (0, 4, 0), le)   # normal +z, toward the camera
    s.add_camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=4, max_depth=2, filter=FILTER_POLARIZER, thetas=[0.0])
    return s, job


def polarizer_stack_scene(angles, le=2.0, spacing: float = 0.05) -> tuple[Scene, Job]:
    """Camera looking down -z through a stack of linear-polarizer sheets (sheet k at
    z = -k * spacing, axis at angles[k]) at a large quad light; polarizer camera filter at
    0 rad; depth len(angles) + 1 (every camera path crosses the whole stack)."""
    s = Scene()
    for k, a in enumerate(angles):
        s.sheet.append(float(a))
        m = s.add_material(Material(MAT_POLARIZER_SHEET, sheet_index=k, t1=(1, 0, 0), t2=(0, 1, 0)))
        s.add_quad((-1, -1, -k * spacing), (2, 0, 0), (0, 2, 0), m)
    s.add_light((-2, -2, -len(angles) * spacing - 1), (4, 0, 0), (0, 4, 0), le)
    s.add_camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=4, max_depth=len(angles) + 1, filter=FILTER_POLARIZER,
              thetas=[0.0])
    return s, job


def retarder_pair_scene() -> tuple[Scene, Job]:
    """A polarized emitter (Stokes 2, 0.8, 0.9, 0.3) behind a quarter-wave and a sixth-wave
    retarder sheet (axes 0.3 and 1.0 rad), polarizer camera filter at 0.2 rad: every
    operator on the path is invertible."""
    s = Scene()
    s.sheet += [0.3, 1.0]
    q = s.add_material(Material(MAT_RETARDER_SHEET, sheet_index=0, retard=math.pi / 2))
    h = s.add_material(Material(MAT_RETARDER_SHEET, sheet_index=1, retard=math.pi / 3))
    s.add_quad((-1, -1, 0), (2, 0, 0), (0, 2, 0), q)
    s.add_quad((-1, -1, -0.05), (2, 0, 0), (0, 2, 0), h)
    s.add_light((-2, -2, -1), (4, 0, 0), (0, 4, 0), np.array([2.0, 0.8, 0.9, 0.3]))
    s.add_camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=4, max_depth=3, filter=FILTER_POLARIZER, thetas=[0.2])
    return s, job


def retarder_scene(alpha: float, phi: float, le: float = 2.0) -> tuple[Scene, Job]:
    """Unpolarized light through a polarizer sheet at alpha, then a quarter-wave sheet with
    fast axis phi, seen by an unfiltered camera (depth 3)."""
    s = Scene()
    s.sheet += [float(alpha), float(phi)]
    pol = s.add_material(Material(MAT_POLARIZER_SHEET, sheet_index=0, t1=(1, 0, 0), t2=(0, 1, 0)))
    qwp = s.add_material(Material(MAT_RETARDER_SHEET, sheet_index=1, t1=(1, 0, 0), t2=(0, 1, 0),
                                  retard=math.pi / 2))
    s.add_quad((-1, -1, 0.5), (2, 0, 0), (0, 2, 0), qwp)
    s.add_quad((-1, -1, 0), (2, 0, 0), (0, 2, 0), pol)
    s.add_light((-2, -2, -1), (4, 0, 0), (0, 4, 0), le)
    s.add_camera((0, 0, 2), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=4, max_depth=3)
    return s, job


def brewster_scene(ior: float = 1.5, le: float = 1.0, dielectric: bool = True) -> tuple[Scene, Job]:
    """Camera at Brewster's angle over a smooth dielectric plane (normal +y) whose mirror
    direction sees a large unpolarized light; the camera's right vector is the s axis."""
    s = Scene()
    tb = math.atan(ior)
    glass = s.add_material(Material(MAT_SMOOTH_DIELECTRIC, ior_index=s.add_ior(ior)))
    s.add_quad((-50, 0, 50), (100, 0, 0), (0, 0, -100), glass)   # normal +y
    d = 10.0
    c = np.array([0, d * math.cos(tb), d * math.sin(tb)])        # light centre in mirror direction
    n = -c / np.linalg.norm(c)                                   # light faces the origin
    a = np.array([1.0, 0, 0])
    b = np.cross(n, a)
    b /= np.linalg.norm(b)
    # e1 x e2 must equal the emission normal n
    e1, e2 = 8 * a, 8 * b
    if np.dot(np.cross(e1, e2), n) < 0:
        e1, e2 = e2, e1
    o = c - 0.5 * e1 - 0.5 * e2
    s.add_light(o, e1, e2, le)
    s.add_camera((0, 3 * math.cos(tb), -3 * math.sin(tb)), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=64, max_depth=2)
    return s, job


def polygon_light_scene(albedo=(0.6, 0.5, 0.4), le=(5.0, 3.0), surface_emission: bool = False,
                        spp: int = 4096) -> tuple[Scene, Job]:
    """A diffuse floor (y = 0, normal +y) of constant albedo seen at the origin by a camera
    with a tiny field of view, lit by two one-sided parallelogram lights of unpolarized
    radiance le[0] and le[1]: a tilted one above the origin and a small upright one near
    the horizon, so that the cosines at the two ends of a light sample differ.  Depth 2
    (direct light only), no camera filter.  With surface_emission the lights are replaced
    by two-sided emitting diffuse quads of zero albedo at the same places: there is then no
    light to sample, and only BSDF sampling reaches them.  The light quads, as (o, e1, e2),
    are LIGHT_QUADS."""
    s = Scene()
    ta = s.add_const_texture(list(albedo), differentiable=True)
    floor = s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta))
    s.add_quad((-5, 0, 5), (10, 0, 0), (0, 0, -10), floor)          # normal +y
    black = s.add_const_texture([0.0, 0.0, 0.0])
    for (o, e1, e2), L in zip(LIGHT_QUADS, le):
        if surface_emission:
            s.add_quad(o, e1, e2, s.add_material(Material(MAT_DIFFUSE, albedo_tex=black, emission=float(L))))
        else:
            s.add_light(np.array(o, np.float64), np.array(e1, np.float64), np.array(e2, np.float64), float(L))
    s.add_camera((0, 2.0, 2.0), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=spp, max_depth=2, seed=5)
    return s, job


# (o, e1, e2) of the two lights of polygon_light_scene; each emits toward e1 x e2, which faces
# the origin: one above, tilted (normal (0, -0.6, 0.6)), one upright near the horizon (normal -x)
LIGHT_QUADS = (((-0.6, 1.5, -0.9), (1.0, 0.0, 0.0), (0.0, 0.6, 0.6)),
               ((1.5, 0.2, -0.4), (0.0, 0.0, 0.8), (0.0, 0.5, 0.0)))


def _yawed(v, yaw_deg: float) -> np.ndarray:
    """v rotated by yaw_deg about the y axis (so that no direction of a test scene lies in a
    coordinate plane, where reference-frame tangents degenerate to the axes)."""
    c, s_ = math.cos(math.radians(yaw_deg)), math.sin(math.radians(yaw_deg))
    v = np.asarray(v, np.float64)
    return np.array([c * v[0] + s_ * v[2], v[1], -s_ * v[0] + c * v[2]])


def glass_interface_scene(ior: float = 1.5, theta_deg: float = 35.0, camera_inside: bool = False,
                          slab: float = 0.0, le: float = 1.0, spp: int = 256, yaw_deg: float = 30.0
                          ) -> tuple[Scene, Job]:
    """A smooth-dielectric plane (y = 0) between a camera above it, looking at the origin at
    theta_deg from the normal in the y-z plane (its right vector is the s axis of the
    interface), and a large one-sided unpolarized light below, facing up.  The plane's
    normal faces the camera (the camera is in air) or, with camera_inside, the light (the
    camera is on the side of the medium).  slab > 0 adds a second, parallel interface of the
    same index at y = -slab whose normal faces down: a glass slab seen from air.  The
    camera's plane of incidence is turned by yaw_deg about the normal.  Depth 2 (3 with the
    slab), no camera filter."""
    s = Scene()
    glass = s.add_material(Material(MAT_SMOOTH_DIELECTRIC, ior_index=s.add_ior(ior)))
    if camera_inside:
        s.add_quad((-50, 0, 50), (0, 0, -100), (100, 0, 0), glass)    # normal -y
    else:
        s.add_quad((-50, 0, 50), (100, 0, 0), (0, 0, -100), glass)    # normal +y
    if slab > 0.0:
        s.add_quad((-50, -slab, 50), (0, 0, -100), (100, 0, 0), glass)
    s.add_light(np.array([-50.0, -1.0 - slab, 50.0]), np.array([100.0, 0, 0]), np.array([0, 0, -100.0]), le)
    t = math.radians(theta_deg)
    s.add_camera(_yawed((0, 3 * math.cos(t), -3 * math.sin(t)), yaw_deg), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=spp, max_depth=3 if slab > 0.0 else 2, seed=9)
    return s, job


def specular_limit_scene(kind: str, theta_deg: float, roughness: float = 0.01, le=(1.0, 0.3, 0.5, 0.2),
                         ior: float = 1.5, eta=(0.2, 3.0), spp: int = 1024, light_size: float = 8.0,
                         yaw_deg: float = 30.0) -> tuple[Scene, Job]:
    """A plane (y = 0, normal +y) seen at theta_deg from its normal by a camera in the y-z
    plane (right vector = the s axis), with a large quad light in the mirror direction whose
    Stokes radiance le is given in the light's frame, its x axis (the first edge) along the
    s axis.  The light is a square of side light_size at distance 10; the plane of
    incidence is turned by yaw_deg about the normal.  kind: 'conductor'
    (GGX, complex index eta, white tint), 'plastic' (GGX rough dielectric of index ior with
    a black diffuse lobe, so only the specular lobe is sampled), or 'smooth' (smooth
    dielectric of index ior).  The GGX kinds take a constant roughness.  Depth 2, no camera
    filter."""
    s = Scene()
    if kind == "smooth":
        m = s.add_material(Material(MAT_SMOOTH_DIELECTRIC, ior_index=s.add_ior(ior)))
    else:
        tr = s.add_const_texture([roughness], differentiable=True)
        if kind == "conductor":
            m = s.add_material(Material(MAT_CONDUCTOR_GGX, rough_tex=tr, eta_re=eta[0], eta_im=eta[1]))
        else:
            tb = s.add_const_texture([0.0, 0.0, 0.0])
            m = s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=tb, rough_tex=tr, ior_index=s.add_ior(ior)))
    s.add_quad((-50, 0, 50), (100, 0, 0), (0, 0, -100), m)
    t = math.radians(theta_deg)
    d = 10.0
    c = _yawed((0.0, d * math.cos(t), d * math.sin(t)), yaw_deg)
    n = -c / np.linalg.norm(c)
    sx = _yawed((1.0, 0.0, 0.0), yaw_deg)             # the s axis of the plane of incidence
    e1 = light_size * sx
    e2 = light_size * np.cross(n, sx)                 # e1 x e2 along n: the light faces the origin
    s.add_light(c - 0.5 * e1 - 0.5 * e2, e1, e2, np.asarray(le, np.float64))
    s.add_camera(_yawed((0, 3 * math.cos(t), -3 * math.sin(t)), yaw_deg), (0, 0, 0), (0, 1, 0), 0.01)
    job = Job(camera=0, width=2, height=2, spp=spp, max_depth=2, seed=13)
    return s, job


def furnace_scene(albedo: float = 0.5, emission: float = 1.0) -> tuple[Scene, Job]:
    """Closed box whose every wall is a two-sided diffuse emitter of constant unpolarized
    emission and albedo a: every path of depth d carries exactly emission * sum_{k<d} a^k."""
    s = Scene()
    ta = s.add_const_texture([albedo] * 3, differentiable=True)
    m = s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta, emission=emission))
    _cornell_geometry(s, m, m, m)
    s.add_quad((-1, -1, 1), (0, 2, 0), (2, 0, 0), m)   # front wall closes the box
    s.add_camera((0, 0, 0), (0, 0, -1), (0, 1, 0), 60.0)
    job = Job(camera=0, width=8, height=8, spp=4, max_depth=5)
    return s, job


def mixed_scene(width: int = 24, spp: int = 4, depth: int = 6) -> tuple[Scene, Job]:
    """Small scene exercising every material: a textured diffuse floor, a rough conductor
    icosphere, a rough dielectric icosphere, a glass sphere, a polarizer and a retarder
    sheet, two lights (one polarized); camera behind a quarter-wave plate and polarizer."""
    s = Scene()
    ta = s.add_texture(np.random.default_rng(11).uniform(0.2, 0.9, (8, 8, 3)), differentiable=True)
    tr = s.add_texture(np.random.default_rng(12).uniform(0.05, 0.5, (8, 8)), differentiable=True)
    floor = s.add_material(Material(MAT_DIFFUSE, albedo_tex=ta))
    cond = s.add_material(Material(MAT_CONDUCTOR_GGX, albedo_tex=ta, rough_tex=tr, eta_re=0.2, eta_im=3.0))
    plas = s.add_material(Material(MAT_PLASTIC_GGX, albedo_tex=ta, rough_tex=tr, ior_index=s.add_ior(1.45)))
    glass = s.add_material(Material(MAT_SMOOTH_DIELECTRIC, ior_index=s.add_ior(1.5)))
    s.sheet += [math.radians(25.0), math.radians(60.0)]
    pol = s.add_material(Material(MAT_POLARIZER_SHEET, sheet_index=0, t1=(1, 0, 0), t2=(0, 1, 0)))
    ret = s.add_material(Material(MAT_RETARDER_SHEET, sheet_index=1, t1=(1, 0, 0), t2=(0, 1, 0),
                                  retard=math.pi / 2))
    s.add_quad((-3, -1, 3), (6, 0, 0), (0, 0, -6), floor)
    v, f, uv = displaced_sphere(3, 0.1, seed=21, radius=0.5, center=(-0.7, -0.45, -0.3))
    s.add_mesh(v, f, cond, uv)
    v, f, uv = displaced_sphere(3, 0.1, seed=22, radius=0.5, center=(0.7, -0.45, -0.3))
    s.add_mesh(v, f, plas, uv)
    s.add_sphere((0.0, -0.6, 0.6), 0.4, glass)
    s.add_quad((-1.2, -1.0, 1.3), (1.0, 0, 0), (0, 1.2, 0), pol)
    s.add_quad((0.3, -1.0, 1.2), (1.0, 0, 0), (0, 1.2, 0), ret)
    s.add_light((-1.0, 2.5, -1.0), (2, 0, 0), (0, 0, 2), 6.0)
    s.add_light((2.5, 0.5, -1.0), (0, 0, 1.5), (0, 1.5, 0), [[3.0, 1.0, 0.5, 0.8]] * 3)
    s.add_camera((0, 0.6, 3.6), (0, -0.4, 0), (0, 1, 0), 45.0)
    job = Job(camera=0, width=width, height=width, spp=spp, max_depth=depth, seed=3,
              filter=FILTER_QWP_POLARIZER, thetas=[math.radians(30.0), math.radians(100.0)])
    return s, job
