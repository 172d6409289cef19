"""Gaussians rendered together with a triangle mesh: mirror bounces and diffuse surfaces lit by a
point light through the Gaussians (rs_build_mesh, rs_render_scene, rs_render_scene_backward).
Argument marshalling only; the rules are stated in include/raysplats.h."""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import native
from .renderer import RenderParams, Renderer, _ptr, _stream_handle


class SceneRenderer:
    """mesh: dict with verts (T, 3, 3), mat (T,) (0 mirror, 1 diffuse), albedo (T, 3), light (3,),
    max_bounces and eps_off (as produced by workloads.scenes.mirror_scene_mesh)."""

    def __init__(self, mesh, tune=None, Q_box=None, list_cap=512, shadow_cap=256):
        self.lib = native.load()
        self.gauss = Renderer(tune=tune, Q_box=Q_box)
        self._verts = np.ascontiguousarray(mesh["verts"], np.float32).reshape(-1)
        self._mat = np.ascontiguousarray(mesh["mat"], np.int32)
        self._alb = np.ascontiguousarray(mesh["albedo"], np.float32).reshape(-1)
        desc = native.RsMeshDesc(len(self._mat), self._verts.ctypes.data_as(ctypes.c_void_p),
                                 self._mat.ctypes.data_as(ctypes.c_void_p), self._alb.ctypes.data_as(ctypes.c_void_p))
        self._mesh = ctypes.c_void_p()
        native.check(self.lib.rs_build_mesh(ctypes.byref(desc), ctypes.byref(self._mesh)))
        self.sp = native.RsSceneParams((ctypes.c_float * 3)(*mesh["light"]), int(mesh["max_bounces"]),
                                       float(mesh["eps_off"]), int(list_cap), int(shadow_cap))
        self._state = ctypes.c_void_p()
        self._cams = None
        self.n_pixels = 0

    def build(self, means, quats, scales, opacities, rgb, stream=None):
        self.gauss.build(means, quats, scales, opacities, rgb, stream=stream)

    def render(self, cams, params: RenderParams | None = None, out=None, stream=None):
        params = params or RenderParams()
        self._cams = native.cameras_to_ctypes(cams)
        self.n_pixels = int(sum(c.width * c.height for c in self._cams))
        dev = self.gauss._keep[0].device
        if out is None:
            out = (torch.empty((self.n_pixels, 3), device=dev), torch.empty(self.n_pixels, device=dev),
                   torch.empty(self.n_pixels, device=dev))
        frame = native.RsFrame(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
        pc = params.to_c()
        native.check(self.lib.rs_render_scene(ctypes.byref(self.gauss._g), self.gauss._accel, self._mesh,
                                              ctypes.byref(self.sp), self._cams, len(self._cams), ctypes.byref(pc),
                                              ctypes.byref(self.gauss.tune), ctypes.byref(frame),
                                              ctypes.byref(self._state), _stream_handle(stream)))
        return out

    def backward(self, d_rgb, d_alpha=None, d_depth=None, grads=None, stream=None):
        means = self.gauss._keep[0]
        n = means.shape[0]
        if grads is None:
            grads = {"means": torch.zeros((n, 3), device=means.device), "quats": torch.zeros((n, 4), device=means.device),
                     "scales": torch.zeros((n, 3), device=means.device), "opacities": torch.zeros(n, device=means.device),
                     "rgb": torch.zeros((n, 3), device=means.device)}
        dl = native.RsFrameGrad(d_rgb.data_ptr(), None if d_alpha is None else d_alpha.data_ptr(),
                                None if d_depth is None else d_depth.data_ptr())
        out = native.RsGaussianGrads(*[grads[k].data_ptr() for k in ("means", "quats", "scales", "opacities", "rgb")])
        native.check(self.lib.rs_render_scene_backward(ctypes.byref(self.gauss._g), self.gauss._accel, self._state,
                                                       ctypes.byref(dl), ctypes.byref(out), _stream_handle(stream)))
        return grads

    def check_device(self, stream=None):
        native.check(self.lib.rs_check_device(self.gauss._accel, None, _stream_handle(stream)))

    def close(self):
        if self._state:
            self.lib.rs_scene_state_destroy(self._state)
            self._state = ctypes.c_void_p()
        if self._mesh:
            self.lib.rs_mesh_destroy(self._mesh)
            self._mesh = ctypes.c_void_p()
        self.gauss.close()
