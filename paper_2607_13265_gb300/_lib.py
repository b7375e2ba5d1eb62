"""ctypes declarations of the C ABI in include/dppt.h (argument marshalling only).

Loading fails loudly when the CUDA library has not been built: there is no CPU
or PyTorch fallback for any step of the path.
"""
from __future__ import annotations

import ctypes
import os
import threading

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "_build", "libdppt.so")

DPPT_OK = 0
STATUS_NAMES = {0: "OK", -1: "INVALID_ARG", -2: "OUT_OF_MEMORY", -3: "CUDA", -4: "TIMEOUT", -5: "UNSUPPORTED",
                -6: "DEVICE"}

c_i32, c_i64, c_u64, c_f32, c_vp = ctypes.c_int32, ctypes.c_int64, ctypes.c_uint64, ctypes.c_float, ctypes.c_void_p


class Material(ctypes.Structure):
    _fields_ = [("type", c_i32), ("albedo_tex", c_i32), ("rough_tex", c_i32), ("ior_index", c_i32),
                ("sheet_index", c_i32), ("normal_tex", c_i32), ("eta_re", c_f32), ("eta_im", c_f32), ("t1", c_f32 * 3), ("t2", c_f32 * 3),
                ("retard", c_f32), ("emission", c_f32)]


class SceneDesc(ctypes.Structure):
    _fields_ = [("num_vertices", c_i64), ("vertices", c_vp), ("uvs", c_vp),
                ("num_triangles", c_i64), ("triangles", c_vp), ("tri_material", c_vp), ("tri_light", c_vp),
                ("num_spheres", c_i64), ("spheres", c_vp), ("sphere_material", c_vp),
                ("num_materials", c_i32), ("materials", c_vp),
                ("num_lights", c_i32), ("lights", c_vp),
                ("num_textures", c_i32), ("textures", c_vp), ("tex_size", c_i64),
                ("num_cameras", c_i32), ("cameras", c_vp),
                ("num_ior", c_i32), ("num_sheets", c_i32), ("ray_eps", c_f32)]


class Job(ctypes.Structure):
    _fields_ = [("camera", c_i32), ("width", c_i32), ("height", c_i32), ("spp", c_i32), ("max_depth", c_i32),
                ("filter", c_i32), ("num_angles", c_i32), ("theta_offset", c_i32),
                ("seed", c_u64), ("stream", c_u64), ("pass_", c_i32), ("reserved", c_i32),
                ("out_offset", c_i64), ("path_sig", c_vp)]


class Params(ctypes.Structure):
    _fields_ = [("tex", c_vp), ("ior", c_vp), ("le", c_vp), ("sheet", c_vp), ("theta", c_vp)]


class Grads(ctypes.Structure):
    _fields_ = [("tex", c_vp), ("ior", c_vp), ("le", c_vp), ("sheet", c_vp), ("theta", c_vp)]


class Launch(ctypes.Structure):
    _fields_ = [("schedule", c_i32), ("block_size", c_i32), ("blocks_per_sm", c_i32),
                ("adj_schedule", c_i32), ("adj_block_size", c_i32), ("adj_blocks_per_sm", c_i32),
                ("adj_scatter", c_i32)]


class Replay(ctypes.Structure):
    _fields_ = [("method", c_i32), ("checkpoint_interval", c_i32), ("gamma", c_f32), ("eps", c_f32),
                ("sigma", c_f32)]


# every symbol include/dppt.h declares, with (restype, argtypes)
SIGNATURES = {
    "dppt_create": (c_i32, [ctypes.POINTER(c_vp), ctypes.c_int]),
    "dppt_destroy": (None, [c_vp]),
    "dppt_last_error": (ctypes.c_char_p, [c_vp]),
    "dppt_version": (ctypes.c_char_p, []),
    "dppt_scene_upload": (c_i32, [c_vp, ctypes.POINTER(SceneDesc), ctypes.POINTER(c_vp)]),
    "dppt_scene_destroy": (None, [c_vp]),
    "dppt_scene_info": (c_i32, [c_vp, ctypes.POINTER(c_i64)]),
    "dppt_render_primal": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params), c_vp, c_vp]),
    "dppt_render_adjoint": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params), c_vp,
                                    ctypes.POINTER(Grads), c_vp]),
    "dppt_loss_l2": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params), c_vp,
                             ctypes.POINTER(c_i64), c_vp, ctypes.c_double, c_vp, c_vp]),
    "dppt_render_adjoint_l2": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params), c_vp,
                                       ctypes.POINTER(c_i64), c_vp, c_f32, ctypes.POINTER(Grads), c_vp]),
    "dppt_query_workspace": (c_i32, [c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(ctypes.c_size_t)]),
    "dppt_set_launch": (c_i32, [c_vp, ctypes.POINTER(Launch)]),
    "dppt_get_launch": (c_i32, [c_vp, ctypes.POINTER(Launch)]),
    "dppt_adjoint_footprint": (c_i32, [c_vp, c_i32, ctypes.POINTER(c_i64)]),
    "dppt_set_replay": (c_i32, [c_vp, ctypes.POINTER(Replay)]),
    "dppt_get_replay": (c_i32, [c_vp, ctypes.POINTER(Replay)]),
    "dppt_count_work": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params),
                                ctypes.POINTER(ctypes.c_uint64)]),
    "dppt_autotune": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), c_i32, ctypes.POINTER(Params), c_i32,
                              ctypes.POINTER(Launch), ctypes.POINTER(ctypes.c_float)]),
    "dppt_render_primal_noalloc": (c_i32, [c_vp, c_vp, ctypes.POINTER(Job), ctypes.POINTER(Params), c_vp, c_vp]),
    "dppt_stage_stats": (c_i32, [c_vp, c_i32, c_i32, ctypes.POINTER(c_i64), ctypes.POINTER(ctypes.c_double)]),
    "dppt_sync_status": (c_i32, [c_vp, c_vp]),
}

_lib = None
_lock = threading.Lock()


class DpptError(RuntimeError):
    pass


def load(path: str = LIB_PATH):
    """Load libdppt.so; raises if it is missing (build it with paper_2607_13265_gb300.build)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise DpptError(f"CUDA library not built: {path} is missing "
                                "(run paper_2607_13265_gb300.build.build() or __graft_entry__.build())")
            L = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                f = getattr(L, name)
                f.restype = res
                f.argtypes = args
            _lib = L
    return _lib
