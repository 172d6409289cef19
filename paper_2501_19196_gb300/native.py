"""ctypes binding of include/raysplats.h (argument marshalling only).

Loads paper_2501_19196_gb300/_lib/libraysplats.so.  There is no fallback: if the library is
missing or fails to load, `load()` raises.  Function names match the C ABI.
"""
from __future__ import annotations

import ctypes
import os

from . import build as _build

P = ctypes.c_void_p
i32, i64, f32 = ctypes.c_int32, ctypes.c_int64, ctypes.c_float

RS_OK, RS_ERR_INVALID_ARG, RS_ERR_OOM, RS_ERR_CUDA, RS_ERR_UNSUPPORTED, RS_ERR_INTERNAL, RS_ERR_TIMEOUT = \
    0, -1, -2, -3, -4, -5, -6


class RsGaussians(ctypes.Structure):
    _fields_ = [("n", i64), ("means", P), ("quats", P), ("scales", P), ("opacities", P), ("rgb", P)]


class RsCamera(ctypes.Structure):
    _fields_ = [("R_wc", f32 * 9), ("pos", f32 * 3), ("fx", f32), ("fy", f32), ("cx", f32), ("cy", f32),
                ("width", i32), ("height", i32)]


class RsRenderParams(ctypes.Structure):
    _fields_ = [("Q", f32), ("eps1", f32), ("t_near", f32), ("background", f32 * 3), ("k_max", i32),
                ("depth_mode", i32), ("sort_key", i32), ("grad_mode", i32), ("eps2", f32)]


class RsFrame(ctypes.Structure):
    _fields_ = [("rgb", P), ("alpha", P), ("depth", P)]


class RsFrameGrad(ctypes.Structure):
    _fields_ = [("d_rgb", P), ("d_alpha", P), ("d_depth", P)]


class RsGaussianGrads(ctypes.Structure):
    _fields_ = [("d_means", P), ("d_quats", P), ("d_scales", P), ("d_opacities", P), ("d_rgb", P)]


class RsMeshDesc(ctypes.Structure):
    _fields_ = [("n_tri", i64), ("verts", P), ("material", P), ("albedo", P)]


class RsSceneParams(ctypes.Structure):
    _fields_ = [("light", f32 * 3), ("max_bounces", i32), ("eps_off", f32), ("list_cap", i32), ("shadow_cap", i32)]


class RsTuneParams(ctypes.Structure):
    _fields_ = [("tile_w", i32), ("tile_h", i32), ("kbuf", i32), ("leaf_size", i32), ("morton_bits", i32),
                ("persistent", i32), ("block_warps", i32), ("traversal", i32), ("smem_nodes", i32),
                ("hit_list", i32)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


STATS_FIELDS = ("rays", "nodes_visited", "gaussians_tested", "hits_composited", "rounds", "hits_inserted",
                "rays_retraced", "hits_listed", "warp_node_fetches", "warp_leaf_iterations")

# name -> (restype, argtypes)
_SIGS = {
    "rs_abi_version": (i32, []),
    "rs_last_error": (ctypes.c_char_p, []),
    "rs_default_tune": (i32, [P]),
    "rs_build_accel": (i32, [P, f32, P, P, P]),
    "rs_render": (i32, [P, P, P, i32, P, P, P, P, P]),
    "rs_render_counted": (i32, [P, P, P, i32, P, P, P, P, P, P]),
    "rs_render_backward": (i32, [P, P, P, P, P, P, P]),
    "rs_render_backward_counted": (i32, [P, P, P, P, P, P, P, P]),
    "rs_tune": (i32, [P, f32, P, i32, P, P, i32, i32, P, P, P, P, P, P]),
    "rs_render_fixed_scratch": (i32, [P, P, i32, P, P, P, P]),
    "rs_accel_destroy": (i32, [P]),
    "rs_state_destroy": (i32, [P]),
    "rs_check_device": (i32, [P, P, P]),
    "rs_accel_export": (i32, [P, P, P, P, P, P, P, P, P, P]),
    "rs_debug_rays": (i32, [P, i32, i64, P, P, P, P, P, P]),
    "rs_debug_hits": (i32, [P, i64, P, P, P, f32, f32, P, P]),
    "rs_test_fail_alloc": (i32, [i64]),
    "rs_loss_l2_dssim": (i32, [P, P, P, i32, f32, P, P, P, P]),
    "rs_loss_state_destroy": (i32, [P]),
    "rs_adam_step": (i32, [P, P, P, P, i64, f32, f32, f32, f32, i32, P]),
    "rs_sigmoid": (i32, [P, P, i64, P]),
    "rs_sigmoid_backward": (i32, [P, P, P, i64, P]),
    "rs_build_mesh": (i32, [P, P]),
    "rs_mesh_destroy": (i32, [P]),
    "rs_render_scene": (i32, [P, P, P, P, P, i32, P, P, P, P, P]),
    "rs_render_scene_backward": (i32, [P, P, P, P, P, P]),
    "rs_scene_state_destroy": (i32, [P]),
}

_LIB = None


class RaySplatsError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"raysplats status {status}: {msg}")
        self.status = status


def library_path() -> str:
    return _build.library_path()


def load(build_if_missing: bool = True):
    """Load the CUDA library (building it first when absent).  Raises when it cannot load."""
    global _LIB
    if _LIB is not None:
        return _LIB
    path = library_path()
    if not os.path.exists(path):
        if not build_if_missing:
            raise RaySplatsError(-4, f"{path} is missing; run paper_2501_19196_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    if lib.rs_abi_version() != 1:
        raise RaySplatsError(-4, "ABI version mismatch")
    _LIB = lib
    return lib


def check(status: int):
    if status != RS_OK:
        raise RaySplatsError(status, load().rs_last_error().decode())


def exported_symbols():
    return list(_SIGS)


def default_tune(**overrides) -> RsTuneParams:
    t = RsTuneParams()
    check(load().rs_default_tune(ctypes.byref(t)))
    for k, v in overrides.items():
        setattr(t, k, int(v))
    if "tile_w" in overrides and "tile_h" not in overrides:
        t.tile_h = 32 // t.tile_w
    return t


def cameras_to_ctypes(cams):
    """workloads.Cameras (or any object with the same arrays) -> ctypes array of RsCamera."""
    n = int(cams.pos.shape[0])
    arr = (RsCamera * n)()
    for c in range(n):
        R = cams.R_wc[c].reshape(9)
        arr[c].R_wc[:] = [float(x) for x in R]
        arr[c].pos[:] = [float(x) for x in cams.pos[c]]
        arr[c].fx, arr[c].fy = float(cams.fx[c]), float(cams.fy[c])
        arr[c].cx, arr[c].cy = float(cams.cx[c]), float(cams.cy[c])
        arr[c].width, arr[c].height = int(cams.width[c]), int(cams.height[c])
    return arr
