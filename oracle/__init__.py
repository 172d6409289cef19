"""FP64 CPU oracle for the RaySplats rendering path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import
this package.  The product path (paper_2501_19196_gb300) never imports it and shares no code
with it; the two meet only in the seeded generators of `workloads`.

The arithmetic lives in raysplats_oracle.c (plain C, FP64, brute force over every
ray/Gaussian pair, built with -ffp-contract=off); this module compiles it on demand and
marshals numpy arrays.  Paper passages followed: Prop. 1 / App. A.1 (ray-ellipsoid entry),
Prop. 2 / App. A.2 (maximum response), Eq. 3 (compositing), Sec. 3 (eps1 cut, K_max),
App. A.3-A.6 (gradients).  Morton codes, the stable order and the radix tree are the plain
definitions the device LBVH must reproduce (no paper counterpart).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .build import build_oracle, library_path

_LIB = None

AMB_BOUNDARY, AMB_TIE, AMB_EPS1, AMB_TNEAR, AMB_IMPACT, AMB_EPS2 = 1, 2, 4, 8, 16, 256
AMB_DECISION = AMB_BOUNDARY | AMB_TIE | AMB_EPS1 | AMB_TNEAR | AMB_EPS2
IMP_BOUNDARY, IMP_TIE, IMP_EPS1 = 32, 64, 128


class OrParams(ctypes.Structure):
    _fields_ = [("Q", ctypes.c_double), ("eps1", ctypes.c_double), ("t_near", ctypes.c_double),
                ("bg", ctypes.c_double * 3), ("k_max", ctypes.c_int32), ("sort_key", ctypes.c_int32),
                ("eps2", ctypes.c_double), ("grad_mode", ctypes.c_int32), ("pad", ctypes.c_int32)]


def lib():
    global _LIB
    if _LIB is None:
        build_oracle()
        L = ctypes.CDLL(library_path())
        P = ctypes.c_void_p
        i64, i32 = ctypes.c_int64, ctypes.c_int32
        L.or_render.restype = ctypes.c_int
        L.or_render.argtypes = [i64, P, P, P, P, P, i64, P, P, P, P, P, P, P, P, P, P, P, P, P, P,
                                P, P, P, i32]
        L.or_raygen_f32.restype = None
        L.or_raygen_f32.argtypes = [P, i64, P, P, P, P, P]
        L.or_raygen_f64.restype = None
        L.or_raygen_f64.argtypes = [P, i64, P, P, P, P]
        L.or_ray_gaussian.restype = None
        L.or_ray_gaussian.argtypes = [P, P, P, P, P, ctypes.c_double, ctypes.c_double, P]
        L.or_quat_to_rot.restype = None
        L.or_quat_to_rot.argtypes = [P, P]
        L.or_morton.restype = None
        L.or_morton.argtypes = [i64, P, P, i32, P, P]
        L.or_sort_perm.restype = ctypes.c_int
        L.or_sort_perm.argtypes = [i64, P, P, P]
        L.or_radix_tree.restype = ctypes.c_int
        L.or_radix_tree.argtypes = [i64, P, P, P, P]
        L.or_chi2_3_quantile.restype = ctypes.c_double
        L.or_chi2_3_quantile.argtypes = [ctypes.c_double]
        L.or_render_scene.restype = ctypes.c_int
        L.or_render_scene.argtypes = [i64, P, P, P, P, P, P, i64, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P, P]
        _LIB = L
    return _LIB


def _p(a):
    return None if a is None else a.ctypes.data_as(ctypes.c_void_p)


def _c(a, dtype):
    return np.ascontiguousarray(a, dtype=dtype)


def default_threads() -> int:
    return max(1, os.cpu_count() or 1)


def raygen_f32(cams, ray_cam, px, py):
    """Rays (o, d) float32 (R, 3) by the fixed FP32 operation sequence."""
    rec = np.ascontiguousarray(cams.pack())
    ray_cam, px, py = _c(ray_cam, np.int32), _c(px, np.int32), _c(py, np.int32)
    n = ray_cam.shape[0]
    o = np.empty((n, 3), np.float32)
    d = np.empty((n, 3), np.float32)
    lib().or_raygen_f32(_p(rec), n, _p(ray_cam), _p(px), _p(py), _p(o), _p(d))
    return o, d


def raygen_f64(cams, cam_index, px, py):
    """Rays (o, d) float64 for camera `cam_index` (FP64 arithmetic, for closed-form pins)."""
    c = np.concatenate([cams.R_wc[cam_index].reshape(9), cams.pos[cam_index],
                        [cams.fx[cam_index], cams.fy[cam_index], cams.cx[cam_index],
                         cams.cy[cam_index]]]).astype(np.float64)
    px, py = _c(px, np.int32).ravel(), _c(py, np.int32).ravel()
    n = px.shape[0]
    o = np.empty((n, 3), np.float64)
    d = np.empty((n, 3), np.float64)
    lib().or_raygen_f64(_p(c), n, _p(px), _p(py), _p(o), _p(d))
    return o, d


def ray_gaussian(o, d, mean, quat, scale, Q, t_near=0.0, with_tol=False):
    """(D2, t1, hit, tau) of one ray against one Gaussian (Prop. 1 and 2), FP64; with_tol adds
    the oracle's models of the uncertainty of an FP32 evaluation of t1, of D2 and of t_m (the
    per-hit halves of its TIE and BOUNDARY bands; t_m's for sort key 1)."""
    out = np.zeros(7, np.float64)
    args = [_c(x, np.float64) for x in (o, d, mean, quat, scale)]
    lib().or_ray_gaussian(*[_p(a) for a in args], float(Q), float(t_near), _p(out))
    res = (float(out[0]), float(out[1]), bool(out[2] > 0.5), float(out[3]))
    return res + (float(out[4]), float(out[5]), float(out[6])) if with_tol else res


def quat_to_rot(q):
    R = np.zeros(9, np.float64)
    lib().or_quat_to_rot(_p(_c(q, np.float64)), _p(R))
    return R.reshape(3, 3)


def render_rays(scene, ray_o, ray_d, Q, eps1=1e-4, k_max=2 ** 31 - 1, background=(0, 0, 0),
                t_near=0.0, dl_rgb=None, dl_alpha=None, threads=None, params64=None, sort_key=0,
                dl_depth=None, eps2=None):
    """Render explicit rays.  `scene` fields are converted to float64 exactly (or taken from
    `params64`, a dict of float64 arrays, for finite differences).  sort_key 0 orders hits by
    the entry t1, 1 by the maximum-response parameter t_m.  Returns a dict with rgb (R,3),
    alpha, depth, T, n_hits, mask and, when dl_rgb or dl_depth is given, the float64
    gradients of <dl_rgb, rgb> + <dl_alpha, alpha> + <dl_depth, depth> (with eps2 given: the
    paper's eps2 estimator for the last composited hit of each ray cut by eps1)."""
    src = params64 if params64 is not None else {
        "means": scene.means, "quats": scene.quats, "scales": scene.scales,
        "opacities": scene.opacities, "rgb": scene.rgb}
    means, quats, scales = (_c(src[k], np.float64) for k in ("means", "quats", "scales"))
    opac, rgb = _c(src["opacities"], np.float64), _c(src["rgb"], np.float64)
    n = means.shape[0]
    ray_o, ray_d = _c(ray_o, np.float64), _c(ray_d, np.float64)
    R = ray_o.shape[0]
    prm = OrParams(float(Q), float(eps1), float(t_near), (ctypes.c_double * 3)(*background),
                   int(k_max), int(sort_key), float(eps2 if eps2 is not None else 0.0),
                   1 if eps2 is not None else 0, 0)
    out = {"rgb": np.zeros((R, 3)), "alpha": np.zeros(R), "depth": np.zeros(R),
           "T": np.zeros(R), "n_hits": np.zeros(R, np.int32), "mask": np.zeros(R, np.int32)}
    grads = None
    if dl_rgb is None and dl_depth is not None:
        dl_rgb = np.zeros((R, 3))
    if dl_rgb is not None:
        dl_rgb = _c(dl_rgb, np.float64)
        dl_alpha = None if dl_alpha is None else _c(dl_alpha, np.float64)
        dl_depth = None if dl_depth is None else _c(dl_depth, np.float64)
        grads = {"means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 3)),
                 "opacities": np.zeros(n), "rgb": np.zeros((n, 3))}
    rc = lib().or_render(
        n, _p(means), _p(quats), _p(scales), _p(opac), _p(rgb), R, _p(ray_o), _p(ray_d),
        ctypes.byref(prm), _p(out["rgb"]), _p(out["alpha"]), _p(out["depth"]), _p(out["T"]),
        _p(out["n_hits"]), _p(out["mask"]), _p(dl_rgb), _p(dl_alpha), _p(dl_depth),
        *(_p(grads[k]) if grads else None for k in ("means", "quats", "scales", "opacities", "rgb")),
        int(threads or default_threads()))
    if rc != 0:
        raise MemoryError("oracle render failed")
    if grads is not None:
        out["grads"] = grads
    return out


def render(scene, cams, ray_cam, px, py, Q, eps1=1e-4, k_max=2 ** 31 - 1, background=(0, 0, 0),
           t_near=0.0, dl_rgb=None, dl_alpha=None, threads=None, sort_key=0, dl_depth=None, eps2=None):
    """Render the listed pixels (camera index, x, y) with FP32-defined rays."""
    o, d = raygen_f32(cams, ray_cam, px, py)
    return render_rays(scene, o, d, Q, eps1, k_max, background, t_near, dl_rgb, dl_alpha, threads,
                       sort_key=sort_key, dl_depth=dl_depth, eps2=eps2)


def morton(means, bits, scales=None):
    """Morton codes (bits = 10, 21) or extended codes with a size class (bits = 20, needs scales)."""
    means = _c(means, np.float32)
    n = means.shape[0]
    codes = np.zeros(n, np.uint64)
    lohi = np.zeros(6, np.float32)
    sc = None if scales is None else _c(scales, np.float32)
    if bits == 20 and sc is None:
        raise ValueError("extended codes need the scales")
    lib().or_morton(n, _p(means), _p(sc), int(bits), _p(codes), _p(lohi))
    return codes, lohi


def sort_perm(codes):
    codes = _c(codes, np.uint64)
    n = codes.shape[0]
    perm = np.zeros(n, np.uint32)
    sc = np.zeros(n, np.uint64)
    if lib().or_sort_perm(n, _p(codes), _p(perm), _p(sc)) != 0:
        raise MemoryError
    return perm, sc


def radix_tree(sorted_codes):
    """(first, last, split) int32 arrays for internal nodes 0..n-2 (Karras numbering)."""
    sc = _c(sorted_codes, np.uint64)
    n = sc.shape[0]
    m = max(n - 1, 0)
    f, l, s = (np.full(m, -1, np.int32) for _ in range(3))
    if lib().or_radix_tree(n, _p(sc), _p(f), _p(l), _p(s)) != 0:
        raise MemoryError
    return f, l, s


def chi2_3_quantile(p):
    return float(lib().or_chi2_3_quantile(float(p)))


AMB_SURFACE = 512  # a triangle decision within FP32 rounding (scene renders)


class OrScene(ctypes.Structure):
    _fields_ = [("n_tri", ctypes.c_int64), ("verts", ctypes.c_void_p), ("mat", ctypes.c_void_p),
                ("albedo", ctypes.c_void_p), ("light", ctypes.c_float * 3), ("max_bounces", ctypes.c_int32),
                ("eps_off", ctypes.c_float)]


def render_scene(scene, mesh, ray_o, ray_d, Q, eps1=1e-4, k_max=2 ** 31 - 1, background=(0, 0, 0), t_near=0.0,
                 dl_rgb=None, dl_alpha=None, dl_depth=None, params64=None):
    """Render FP32 rays through Gaussians and a triangle mesh (mirror / diffuse, one point light).
    mesh: dict with verts (T, 3, 3) float32, mat (T,) int32 (0 mirror, 1 diffuse), albedo (T, 3),
    light (3,), max_bounces, eps_off.  Returns rgb, alpha, depth, n_hits, mask and, with dl_rgb,
    the float64 gradients w.r.t. the Gaussian parameters."""
    src = params64 if params64 is not None else {
        "means": scene.means, "quats": scene.quats, "scales": scene.scales,
        "opacities": scene.opacities, "rgb": scene.rgb}
    means, quats, scales = (_c(src[k], np.float64) for k in ("means", "quats", "scales"))
    opac, rgb = _c(src["opacities"], np.float64), _c(src["rgb"], np.float64)
    n = means.shape[0]
    ray_o, ray_d = _c(ray_o, np.float32), _c(ray_d, np.float32)
    R = ray_o.shape[0]
    verts = _c(mesh["verts"], np.float32).reshape(-1, 9)
    mat = _c(mesh["mat"], np.int32)
    alb = _c(mesh["albedo"], np.float32).reshape(-1, 3)
    S = OrScene(verts.shape[0], _p(verts), _p(mat), _p(alb), (ctypes.c_float * 3)(*mesh["light"]),
                int(mesh["max_bounces"]), float(mesh["eps_off"]))
    prm = OrParams(float(Q), float(eps1), float(t_near), (ctypes.c_double * 3)(*background), int(k_max), 0,
                   0.0, 0, 0)
    out = {"rgb": np.zeros((R, 3)), "alpha": np.zeros(R), "depth": np.zeros(R),
           "n_hits": np.zeros(R, np.int32), "mask": np.zeros(R, np.int32)}
    grads = None
    if dl_rgb is not None:
        dl_rgb = _c(dl_rgb, np.float64)
        dl_alpha = None if dl_alpha is None else _c(dl_alpha, np.float64)
        dl_depth = None if dl_depth is None else _c(dl_depth, np.float64)
        grads = {"means": np.zeros((n, 3)), "quats": np.zeros((n, 4)), "scales": np.zeros((n, 3)),
                 "opacities": np.zeros(n), "rgb": np.zeros((n, 3))}
    rc = lib().or_render_scene(
        n, _p(means), _p(quats), _p(scales), _p(opac), _p(rgb), ctypes.byref(S), R, _p(ray_o), _p(ray_d),
        ctypes.byref(prm), _p(out["rgb"]), _p(out["alpha"]), _p(out["depth"]), _p(out["n_hits"]), _p(out["mask"]),
        _p(dl_rgb), _p(dl_alpha), _p(dl_depth),
        *(_p(grads[k]) if grads else None for k in ("means", "quats", "scales", "opacities", "rgb")))
    if rc != 0:
        raise MemoryError("oracle scene render failed")
    if grads is not None:
        out["grads"] = grads
    return out
