"""Torch-facing wrapper of the C ABI: device memory and streams come from PyTorch, every step
of the render and its adjoint runs in libraysplats.so.

    r = Renderer()
    r.build(means, quats, scales, opacities, rgb)         # rs_build_accel
    rgb, alpha, depth = r.render(cams, params)            # rs_render
    grads = r.backward(d_rgb, d_alpha)                    # rs_render_backward

`render_gaussians(...)` is the autograd entry point (torch.autograd.Function): its backward
calls rs_render_backward.  Parameters are physical (scales > 0, opacity in [0, 1)); apply
exp / sigmoid activations in torch before calling it.
"""
from __future__ import annotations

import ctypes
import dataclasses

import torch

from . import native

_DEFAULT_Q = 11.344866730144373  # chi^2(3) quantile at 0.99


@dataclasses.dataclass
class RenderParams:
    Q: float = _DEFAULT_Q
    eps1: float = 1e-4
    t_near: float = 0.0
    background: tuple = (0.0, 0.0, 0.0)
    k_max: int = 2 ** 31 - 1
    sort_key: int = 0  # 0: order hits by entry t1; 1: by t_m (maximum response)
    eps2: float | None = None  # set: the adjoint uses the paper's eps2 estimator

    def to_c(self) -> native.RsRenderParams:
        p = native.RsRenderParams()
        p.Q, p.eps1, p.t_near = float(self.Q), float(self.eps1), float(self.t_near)
        p.background[:] = [float(x) for x in self.background]
        p.k_max, p.depth_mode, p.sort_key = int(self.k_max), 0, int(self.sort_key)
        p.grad_mode, p.eps2 = (0, 1.0) if self.eps2 is None else (1, float(self.eps2))
        return p


def _ptr(t):
    return None if t is None else ctypes.c_void_p(t.data_ptr())


def _stream_handle(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


def _check_param(t, name, n, width):
    if not t.is_cuda or t.dtype != torch.float32 or not t.is_contiguous():
        raise ValueError(f"{name}: need a contiguous float32 CUDA tensor")
    if t.numel() != n * width:
        raise ValueError(f"{name}: expected {n * width} elements, got {t.numel()}")


class Renderer:
    """Owns one rs_accel and one rs_fwd_state (reused across calls)."""

    def __init__(self, tune: native.RsTuneParams | None = None, Q_box: float = _DEFAULT_Q):
        self.lib = native.load()
        self.tune = tune if tune is not None else native.default_tune()
        self.Q_box = float(Q_box)
        self._accel = ctypes.c_void_p()
        self._state = ctypes.c_void_p()
        self._g = None
        self._keep = None
        self.n_pixels = 0
        self._cams = None

    # -- scene -------------------------------------------------------------------------------
    def _gaussians(self, means, quats, scales, opacities, rgb):
        n = means.shape[0]
        for t, nm, w in ((means, "means", 3), (quats, "quats", 4), (scales, "scales", 3),
                         (opacities, "opacities", 1), (rgb, "rgb", 3)):
            _check_param(t, nm, n, w)
        g = native.RsGaussians(n, means.data_ptr(), quats.data_ptr(), scales.data_ptr(),
                               opacities.data_ptr(), rgb.data_ptr())
        return g

    def build(self, means, quats, scales, opacities, rgb, stream=None):
        self._g = self._gaussians(means, quats, scales, opacities, rgb)
        self._keep = (means, quats, scales, opacities, rgb)
        native.check(self.lib.rs_build_accel(ctypes.byref(self._g), self.Q_box, ctypes.byref(self.tune),
                                             ctypes.byref(self._accel), _stream_handle(stream)))

    # -- forward -----------------------------------------------------------------------------
    def set_cameras(self, cams):
        self._cams = native.cameras_to_ctypes(cams)
        self.n_pixels = int(sum(c.width * c.height for c in self._cams))

    def render(self, cams=None, params: RenderParams | None = None, out=None, stats=None, stream=None):
        """Render all cameras; returns (rgb (P,3), alpha (P,), depth (P,)) with P = sum W*H."""
        if cams is not None:
            self.set_cameras(cams)
        params = params or RenderParams()
        dev = self._keep[0].device
        if out is None:
            out = (torch.empty((self.n_pixels, 3), device=dev, dtype=torch.float32),
                   torch.empty(self.n_pixels, device=dev, dtype=torch.float32),
                   torch.empty(self.n_pixels, device=dev, dtype=torch.float32))
        rgb, alpha, depth = out
        frame = native.RsFrame(rgb.data_ptr(), alpha.data_ptr(), None if depth is None else depth.data_ptr())
        self._params_c = params.to_c()
        if stats is None:
            st = self.lib.rs_render(ctypes.byref(self._g), self._accel, self._cams, len(self._cams),
                                    ctypes.byref(self._params_c), ctypes.byref(self.tune), ctypes.byref(frame),
                                    ctypes.byref(self._state), _stream_handle(stream))
        else:
            st = self.lib.rs_render_counted(ctypes.byref(self._g), self._accel, self._cams, len(self._cams),
                                            ctypes.byref(self._params_c), ctypes.byref(self.tune),
                                            ctypes.byref(frame), ctypes.byref(self._state), _ptr(stats),
                                            _stream_handle(stream))
        native.check(st)
        return out

    # -- backward ----------------------------------------------------------------------------
    def backward(self, d_rgb, d_alpha=None, grads=None, stream=None, stats=None, d_depth=None):
        """Accumulate dL/d(params) into `grads` (dict of zeroed tensors, created if None) for the
        upstream gradients of rgb (required), alpha and depth (optional)."""
        means = self._keep[0]
        n = means.shape[0]
        if grads is None:
            grads = {"means": torch.zeros((n, 3), device=means.device), "quats": torch.zeros((n, 4), device=means.device),
                     "scales": torch.zeros((n, 3), device=means.device), "opacities": torch.zeros(n, device=means.device),
                     "rgb": torch.zeros((n, 3), device=means.device)}
        if not d_rgb.is_contiguous() or d_rgb.numel() != 3 * self.n_pixels:
            raise ValueError("d_rgb: expected a contiguous (P, 3) tensor")
        if d_alpha is not None and (not d_alpha.is_contiguous() or d_alpha.numel() != self.n_pixels):
            raise ValueError("d_alpha: expected a contiguous (P,) tensor")
        if d_depth is not None and (not d_depth.is_contiguous() or d_depth.numel() != self.n_pixels):
            raise ValueError("d_depth: expected a contiguous (P,) tensor")
        dl = native.RsFrameGrad(d_rgb.data_ptr(), None if d_alpha is None else d_alpha.data_ptr(),
                                None if d_depth is None else d_depth.data_ptr())
        out = native.RsGaussianGrads(*[None if grads.get(k) is None else grads[k].data_ptr()
                                       for k in ("means", "quats", "scales", "opacities", "rgb")])
        if stats is None:
            st = self.lib.rs_render_backward(ctypes.byref(self._g), self._accel, self._state, ctypes.byref(dl),
                                             ctypes.byref(self.tune), ctypes.byref(out), _stream_handle(stream))
        else:
            st = self.lib.rs_render_backward_counted(ctypes.byref(self._g), self._accel, self._state,
                                                     ctypes.byref(dl), ctypes.byref(self.tune), ctypes.byref(out),
                                                     _ptr(stats), _stream_handle(stream))
        native.check(st)
        return grads

    def check_device(self, stream=None):
        native.check(self.lib.rs_check_device(self._accel, self._state, _stream_handle(stream)))

    def export_accel(self):
        """Host copies of the LBVH internals (synchronises)."""
        import numpy as np
        n = ctypes.c_int64()
        native.check(self.lib.rs_accel_export(self._accel, ctypes.byref(n), None, None, None, None, None, None,
                                              None, None))
        n = n.value
        m = max(n - 1, 1)
        out = {"codes": np.zeros(n, np.uint64), "perm": np.zeros(n, np.uint32), "first": np.zeros(m, np.int32),
               "last": np.zeros(m, np.int32), "split": np.zeros(m, np.int32), "boxes": np.zeros((m, 6), np.float32),
               "prim_boxes": np.zeros((n, 6), np.float32), "lo_hi": np.zeros(6, np.float32)}
        P = lambda a: a.ctypes.data_as(ctypes.c_void_p)  # noqa: E731
        native.check(self.lib.rs_accel_export(self._accel, None, P(out["codes"]), P(out["perm"]), P(out["first"]),
                                              P(out["last"]), P(out["split"]), P(out["boxes"]),
                                              P(out["prim_boxes"]), P(out["lo_hi"])))
        return out

    def debug_hits(self, ray_o, ray_d, sorted_j, Q, t_near=0.0, stream=None):
        n = sorted_j.numel()
        out = torch.empty((n, 8), device=ray_o.device, dtype=torch.float32)
        native.check(self.lib.rs_debug_hits(self._accel, n, _ptr(ray_o), _ptr(ray_d), _ptr(sorted_j), float(Q),
                                            float(t_near), _ptr(out), _stream_handle(stream)))
        return out

    def close(self):
        if self._state:
            native.check(self.lib.rs_state_destroy(self._state))
            self._state = ctypes.c_void_p()
        if self._accel:
            native.check(self.lib.rs_accel_destroy(self._accel))
            self._accel = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def debug_rays(cams, cam_idx, px, py, stream=None):
    """Device rays of listed pixels (int32 CUDA tensors) by the renderer's FP32 sequence."""
    lib = native.load()
    arr = native.cameras_to_ctypes(cams)
    n = cam_idx.numel()
    o = torch.empty((n, 3), device=cam_idx.device, dtype=torch.float32)
    d = torch.empty((n, 3), device=cam_idx.device, dtype=torch.float32)
    native.check(lib.rs_debug_rays(arr, len(arr), n, _ptr(cam_idx), _ptr(px), _ptr(py), _ptr(o), _ptr(d),
                                   _stream_handle(stream)))
    return o, d


class _RenderFn(torch.autograd.Function):
    @staticmethod
    def forward(ctx, means, quats, scales, opacities, rgb, renderer, cams, params):
        renderer.build(means, quats, scales, opacities, rgb)
        out_rgb, out_alpha, out_depth = renderer.render(cams, params)
        ctx.renderer = renderer
        return out_rgb, out_alpha, out_depth

    @staticmethod
    def backward(ctx, g_rgb, g_alpha, g_depth):
        r = ctx.renderer
        g_rgb = torch.zeros((r.n_pixels, 3), device=r._keep[0].device) if g_rgb is None else g_rgb.contiguous()
        g_alpha = None if g_alpha is None else g_alpha.contiguous()
        g_depth = None if g_depth is None else g_depth.contiguous()
        grads = r.backward(g_rgb, g_alpha, d_depth=g_depth)
        return grads["means"], grads["quats"], grads["scales"], grads["opacities"], grads["rgb"], None, None, None


def render_gaussians(means, quats, scales, opacities, rgb, cams, params: RenderParams | None = None,
                     renderer: Renderer | None = None):
    """Differentiable render of every camera in `cams`; returns (rgb, alpha, depth) per pixel.
    All three outputs carry gradients (depth through opacities and the hits' sort keys)."""
    renderer = renderer or Renderer()
    return _RenderFn.apply(means.contiguous(), quats.contiguous(), scales.contiguous(), opacities.contiguous(),
                           rgb.contiguous(), renderer, cams, params or RenderParams())
