"""FP64 CPU oracle for differentiable polarized path tracing -- TEST INFRASTRUCTURE.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The product path (the CUDA library and
its Python binding) never does, and the two share no code: this package wraps
``oracle.cpp`` (plain single-threaded double precision C++) through ctypes.

Functions follow the paper as stated in ``oracle.cpp``'s header:
  * :meth:`OracleScene.render` -- the polarized MC estimator (Eq. 2 with the
    Mueller-Stokes calculus of Sec. 3.3);
  * :meth:`OracleScene.gradient` -- its reverse-mode derivative with detached
    sampling, either by conventional taped AD (``mode='tape'``, the "Conv. AD"
    reference of Sec. 5.1) or by cached suffix replay (``mode='replay'``,
    Sec. 4.3 / Fig. 2);
  * ``gradient(..., mode='pprb')`` -- basic polarized PRB with noise-regularized
    inversion (Sec. 4.1-4.2), the baseline whose failure Sec. 4.1 analyses;
  * :meth:`OracleScene.gradient_hybrid` -- hybrid cached replay (Sec. 4.4);
  * ``render(..., params_live=...)`` -- the frozen-sampling estimator used for
    central finite differences.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SO = os.path.join(_HERE, "_build", "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile oracle.cpp with g++ (C++17, -O2, portable: no -march flags)."""
    src = os.path.join(_HERE, "oracle.cpp")
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(src):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-std=c++17", "-O2", "-shared", "-fPIC", "-o", tmp, src])
        os.replace(tmp, _SO)
    return _SO


def _configure(L):
    P = ctypes.c_void_p
    i64, dbl, i32 = ctypes.c_int64, ctypes.c_double, ctypes.c_int
    L.orc_scene_create.restype = P
    L.orc_scene_create.argtypes = [i64, P, P, i64, P, P, P, i64, P, P, i64, P, P, i64, P, i64, P, i64, P, dbl]
    L.orc_scene_destroy.argtypes = [P]
    L.orc_render.restype = i32
    L.orc_render.argtypes = [P, P, P, i64, P, P, P, P, P, P]
    L.orc_gradient.restype = i32
    L.orc_gradient.argtypes = [P, P, P, i64, P, P, P, P, i32]
    L.orc_gradient_pprb.restype = i32
    L.orc_gradient_pprb.argtypes = [P, P, P, i64, P, P, P, P, dbl, i32]
    L.orc_gradient_hybrid.restype = i32
    L.orc_gradient_hybrid.argtypes = [P, P, P, i64, P, P, P, P, i32, dbl, dbl, P]
    L.orc_philox.argtypes = [P, P, P]
    L.orc_uniforms.argtypes = [ctypes.c_uint64] * 5 + [P]
    L.orc_fresnel_reflect.argtypes = [dbl, dbl, dbl, dbl, P]
    L.orc_fresnel_transmit.argtypes = [dbl, dbl, dbl, P]
    L.orc_camera_filter.argtypes = [i32, dbl, P]
    L.orc_csqrt.argtypes = [dbl, dbl, P]
    L.orc_ggx.argtypes = [dbl, dbl, dbl, dbl, P]
    L.orc_depol_index.restype = dbl
    L.orc_depol_index.argtypes = [P]
    L.orc_tex_lookup.restype = dbl
    L.orc_tex_lookup.argtypes = [i32, i32, i32, P, i32, dbl, dbl]
    L.orc_closest.restype = i32
    L.orc_closest.argtypes = [P, P, P, i32, P]
    L.orc_stats.argtypes = [P, i32]
    return L


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            _lib = _configure(ctypes.CDLL(_SO))
    return _lib


def load(path: str):
    """A separate build of the oracle at `path` (the tests build copies of oracle.cpp with
    one planted mistake and check that the pins catch it); pass it to OracleScene."""
    return _configure(ctypes.CDLL(os.path.abspath(path)))


def _p(a):
    return a.ctypes.data_as(ctypes.c_void_p) if a is not None else None


def job_array(job) -> np.ndarray:
    return np.array([job.camera, job.width, job.height, job.spp, job.max_depth, job.seed,
                     job.pass_id, job.stream, job.filter, job.num_angles], np.int64)


def flat_params(params: dict, job) -> tuple[np.ndarray, np.ndarray]:
    """Flatten {tex, ior, le, sheet} + the job's filter angles into one vector and its layout."""
    tex = np.asarray(params["tex"], np.float64).ravel()
    ior = np.asarray(params["ior"], np.float64).ravel()
    le = np.asarray(params["le"], np.float64).ravel()
    sheet = np.asarray(params["sheet"], np.float64).ravel()
    theta = np.asarray(params.get("theta", job.thetas if job.thetas else [0.0]), np.float64).ravel()
    parts = [tex, ior, le, sheet, theta]
    offs = np.cumsum([0] + [len(p) for p in parts])
    return np.concatenate(parts), offs.astype(np.int64)


def unflat(vec: np.ndarray, layout: np.ndarray) -> dict:
    names = ["tex", "ior", "le", "sheet", "theta"]
    return {n: vec[layout[i]:layout[i + 1]].copy() for i, n in enumerate(names)}


MAT_I_FIELDS = 6
MAT_F_FIELDS = 10


class OracleScene:
    """The oracle's own copy of a scene (built from the seeded generator's arrays)."""

    def __init__(self, scene, library=None):
        L = self._lib = library if library is not None else lib()
        self._keep = []

        def arr(a, dt):
            a = np.ascontiguousarray(a, dt)
            self._keep.append(a)
            return a

        verts = arr(scene.verts, np.float64)
        uvs = arr(scene.uvs, np.float64)
        tris = arr(scene.tris, np.int32)
        tmat = arr(scene.tri_mat, np.int32)
        tlight = arr(scene.tri_light, np.int32)
        sph = arr(scene.spheres, np.float64)
        smat = arr(scene.sph_mat, np.int32)
        mi = arr([[m.type, m.albedo_tex, m.rough_tex, m.ior_index, m.sheet_index, m.normal_tex]
                  for m in scene.materials], np.int32)
        mf = arr([[m.eta_re, m.eta_im, *m.t1, *m.t2, m.retard, m.emission] for m in scene.materials], np.float64)
        lights = arr(scene.lights, np.float64)
        texd = arr(scene.tex_desc, np.int64)
        cams = arr(scene.cameras, np.float64)
        self.num_lights = len(lights)
        self.h = L.orc_scene_create(len(verts), _p(verts), _p(uvs), len(tris), _p(tris), _p(tmat), _p(tlight),
                                    len(sph), _p(sph), _p(smat), len(mi), _p(mi), _p(mf), len(lights), _p(lights),
                                    len(texd), _p(texd), len(cams), _p(cams), float(scene.ray_eps()))
        self.scene = scene

    def __del__(self):
        try:
            self._lib.orc_scene_destroy(self.h)
        except Exception:
            pass

    @staticmethod
    def _pixels(job, pixels):
        if pixels is None:
            return np.arange(job.width * job.height, dtype=np.int64)
        return np.ascontiguousarray(pixels, np.int64)

    def render(self, job, params: dict, pixels=None, params_live: dict | None = None, paths: bool = False):
        """Stokes image [angles][npix][3][4] of the listed pixels (all by default).

        With ``params_live`` the sampling uses ``params`` (detached) and the Mueller
        values use ``params_live`` (frozen-sampling estimator).  With ``paths`` also
        returns the raw sensor-frame Stokes of every path and its signature."""
        pix = self._pixels(job, pixels)
        P0, lay = flat_params(params, job)
        Pv = P0 if params_live is None else flat_params(params_live, job)[0]
        A = job.num_angles
        out = np.zeros((A, len(pix), 3, 4))
        pout = np.zeros((len(pix) * job.spp, 3, 4)) if paths else None
        sig = np.zeros(len(pix) * job.spp, np.uint32) if paths else None
        j = job_array(job)
        rc = self._lib.orc_render(self.h, _p(j), _p(pix), len(pix), _p(P0), _p(Pv), _p(lay), _p(out), _p(pout), _p(sig))
        assert rc == 0
        return (out, pout, sig) if paths else out

    def gradient(self, job, params: dict, dI: np.ndarray, pixels=None, mode: str = "replay",
                 sigma: float = 1e-3, primal_noise: bool = True, single: bool = False) -> dict:
        """Gradient of sum(dI * I) w.r.t. {tex, ior, le, sheet, theta}: mode 'tape'
        (conventional AD), 'replay' (cached suffix replay) or 'pprb' (basic polarized PRB
        with noise-regularized inversion, the failing baseline of Sec. 4.1-4.2: noise of
        deviation ``sigma`` in the primal too when ``primal_noise``, fold and recovery in
        single precision when ``single``)."""
        pix = self._pixels(job, pixels)
        P, lay = flat_params(params, job)
        dI = np.ascontiguousarray(dI, np.float64).reshape(job.num_angles, len(pix), 3, 4)
        g = np.zeros_like(P)
        j = job_array(job)
        if mode == "pprb":
            rc = self._lib.orc_gradient_pprb(self.h, _p(j), _p(pix), len(pix), _p(P), _p(lay), _p(dI), _p(g),
                                         float(sigma), int(primal_noise) | (2 if single else 0))
        else:
            rc = self._lib.orc_gradient(self.h, _p(j), _p(pix), len(pix), _p(P), _p(lay), _p(dI), _p(g),
                                    {"tape": 0, "replay": 1}[mode])
        assert rc == 0
        return unflat(g, lay)

    def gradient_hybrid(self, job, params: dict, dI: np.ndarray, k: int, gamma: float, eps: float,
                        pixels=None) -> tuple[dict, dict]:
        """Gradient by hybrid cached replay (Sec. 4.4): suffixes cached every k vertices, the
        others recovered by scalar PRB (DI < gamma), inversion (|det| > eps) or
        recomputation.  Returns (gradient, channel-vertices per route)."""
        pix = self._pixels(job, pixels)
        P, lay = flat_params(params, job)
        dI = np.ascontiguousarray(dI, np.float64).reshape(job.num_angles, len(pix), 3, 4)
        g = np.zeros_like(P)
        routes = np.zeros(4)
        j = job_array(job)
        rc = self._lib.orc_gradient_hybrid(self.h, _p(j), _p(pix), len(pix), _p(P), _p(lay), _p(dI), _p(g),
                                       int(k), float(gamma), float(eps), _p(routes))
        assert rc == 0
        return unflat(g, lay), dict(zip(["cached", "scalar", "inverse", "recompute"], routes.tolist()))

    def closest(self, o, d, brute=False):
        o = np.ascontiguousarray(o, np.float64)
        d = np.ascontiguousarray(d, np.float64)
        t = np.zeros(1)
        prim = self._lib.orc_closest(self.h, _p(o), _p(d), int(brute), _p(t))
        return prim, float(t[0])


def stats(reset: bool = True) -> dict:
    out = np.zeros(9)
    lib().orc_stats(_p(out), int(reset))
    keys = ["rays", "shadow_rays", "vertices", "bvh_nodes", "tri_tests", "sph_tests", "paths", "tape_peak_nodes",
            "tape_total_nodes"]
    return dict(zip(keys, out.tolist()))


def _lib_or(library):
    """The given oracle library (a copy built from other sources, as the tests that plant
    mistakes use), else the oracle's own."""
    return library if library is not None else lib()


def philox4x64(counter, key, library=None) -> np.ndarray:
    c = np.ascontiguousarray(counter, np.uint64)
    k = np.ascontiguousarray(key, np.uint64)
    o = np.zeros(4, np.uint64)
    _lib_or(library).orc_philox(_p(c), _p(k), _p(o))
    return o


def uniforms(seed, pass_id, stream, path, vertex, library=None) -> np.ndarray:
    u = np.zeros(8)
    _lib_or(library).orc_uniforms(seed, pass_id, stream, path, vertex, _p(u))
    return u


def fresnel_reflect(cos_i, eta_i, eta_t: complex, library=None) -> np.ndarray:
    o = np.zeros(4)
    _lib_or(library).orc_fresnel_reflect(cos_i, eta_i, complex(eta_t).real, complex(eta_t).imag, _p(o))
    return o


def fresnel_transmit(cos_i, eta_i, eta_t, library=None) -> np.ndarray:
    o = np.zeros(4)
    _lib_or(library).orc_fresnel_transmit(cos_i, eta_i, eta_t, _p(o))
    return o


def camera_filter(filter_type: int, theta: float, library=None) -> np.ndarray:
    o = np.zeros(16)
    _lib_or(library).orc_camera_filter(filter_type, theta, _p(o))
    return o.reshape(4, 4)


def ggx(cos_h: float, cos_v: float, cos_vh: float, alpha: float, library=None) -> tuple[float, float]:
    """The oracle's GGX D(cos_h) and Smith G1(cos_v, cos_vh) for roughness alpha."""
    o = np.zeros(2)
    _lib_or(library).orc_ggx(float(cos_h), float(cos_v), float(cos_vh), float(alpha), _p(o))
    return float(o[0]), float(o[1])


def depol_index(m: np.ndarray, library=None) -> float:
    """The oracle's depolarization index of a 4x4 Mueller matrix (the hybrid's scalar-route test)."""
    a = np.ascontiguousarray(m, np.float64).reshape(16)
    return float(_lib_or(library).orc_depol_index(_p(a)))


def tex_lookup(texels: np.ndarray, c: int, u: float, v: float, library=None) -> float:
    """The oracle's bilinear lookup of channel c at (u, v) in texels [h][w][ch]."""
    t = np.ascontiguousarray(texels, np.float64)
    h, w, ch = t.shape
    return float(_lib_or(library).orc_tex_lookup(w, h, ch, _p(t), c, float(u), float(v)))


def csqrt(z: complex) -> complex:
    o = np.zeros(2)
    lib().orc_csqrt(z.real, z.imag, _p(o))
    return complex(o[0], o[1])
