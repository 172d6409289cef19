"""The training step around the rendering path: sigmoid activations, render, L2 + D-SSIM loss,
adjoint, Adam (Sec. 3 "Loss Function", App. A.7, Sec. 5).  Argument marshalling only: every
step runs in libraysplats.so (rs_sigmoid, rs_build_accel, rs_render, rs_loss_l2_dssim,
rs_render_backward, rs_sigmoid_backward, rs_adam_step).
"""
from __future__ import annotations

import ctypes

import torch

from . import native
from .renderer import RenderParams, Renderer, _ptr, _stream_handle


def sigmoid(x, out=None, stream=None):
    out = torch.empty_like(x) if out is None else out
    native.check(native.load().rs_sigmoid(_ptr(x), _ptr(out), x.numel(), _stream_handle(stream)))
    return out


def sigmoid_backward(y, dy, out=None, stream=None):
    out = torch.empty_like(y) if out is None else out
    native.check(native.load().rs_sigmoid_backward(_ptr(y), _ptr(dy), _ptr(out), y.numel(), _stream_handle(stream)))
    return out


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8, stream=None):
    """In-place Adam update of the contiguous float32 CUDA tensor p (moments m, v)."""
    native.check(native.load().rs_adam_step(_ptr(p), _ptr(g), _ptr(m), _ptr(v), p.numel(), float(lr), float(beta1),
                                            float(beta2), float(eps), int(step), _stream_handle(stream)))


class ImageLoss:
    """L2 + D-SSIM loss of a batch of rendered images (rs_render layout) and its gradient."""

    def __init__(self, lam=0.2):
        self.lam = float(lam)
        self.lib = native.load()
        self._state = ctypes.c_void_p()
        self._cams = None
        self.loss = None
        self.d_rgb = None

    def __call__(self, rgb, target, cams, stream=None):
        """Returns (loss (1,) device tensor, dL/drgb (P, 3)); both buffers are reused."""
        self._cams = native.cameras_to_ctypes(cams) if not isinstance(cams, ctypes.Array) else cams
        if self.loss is None or self.loss.device != rgb.device:
            self.loss = torch.zeros(1, device=rgb.device)
        if self.d_rgb is None or self.d_rgb.shape != rgb.shape:
            self.d_rgb = torch.empty_like(rgb)
        native.check(self.lib.rs_loss_l2_dssim(_ptr(rgb), _ptr(target), self._cams, len(self._cams), self.lam,
                                               _ptr(self.loss), _ptr(self.d_rgb), ctypes.byref(self._state),
                                               _stream_handle(stream)))
        return self.loss, self.d_rgb

    def close(self):
        if self._state:
            self.lib.rs_loss_state_destroy(self._state)
            self._state = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class TrainStep:
    """One optimisation step of the scene parameters against target images.

    Parameters live in one flat float32 buffer [means 3n | quats 4n | scale logits 3n |
    opacity logits n | rgb 3n]; scales and opacities are the sigmoids of their logits (Sec. 5).
    Each group has its own learning rate; Adam moments are kept per element."""

    GROUPS = (("means", 3), ("quats", 4), ("scale_logits", 3), ("opacity_logits", 1), ("rgb", 3))

    def __init__(self, means, quats, scale_logits, opacity_logits, rgb, lr=None, lam=0.2, tune=None,
                 params: RenderParams | None = None, Q_box=None):
        n = means.shape[0]
        dev = means.device
        self.n = n
        self.flat = torch.cat([t.reshape(-1).float() for t in (means, quats, scale_logits, opacity_logits, rgb)])
        self.grad = torch.zeros_like(self.flat)
        self.m = torch.zeros_like(self.flat)
        self.v = torch.zeros_like(self.flat)
        self.views, self.gviews, off = {}, {}, 0
        for name, w in self.GROUPS:
            shape = (n, w) if w > 1 else (n,)
            self.views[name] = self.flat[off:off + n * w].view(shape)
            self.gviews[name] = self.grad[off:off + n * w].view(shape)
            off += n * w
        self.lr = dict(means=1.6e-4, quats=1e-3, scale_logits=5e-3, opacity_logits=5e-2, rgb=2.5e-3)
        if lr:
            self.lr.update(lr)
        self.scales = torch.empty((n, 3), device=dev)
        self.opacities = torch.empty(n, device=dev)
        self.g_act = {"scales": torch.zeros((n, 3), device=dev), "opacities": torch.zeros(n, device=dev)}
        self.params = params or RenderParams()
        self.renderer = Renderer(tune=tune, Q_box=Q_box or self.params.Q)
        self.loss_fn = ImageLoss(lam)
        self.t = 0

    def step(self, target, cams=None, stream=None):
        """Render, evaluate the loss against `target` (P, 3), back-propagate and update.
        Returns the loss as a (1,) device tensor (no host synchronisation)."""
        V = self.views
        sigmoid(V["scale_logits"], self.scales, stream)
        sigmoid(V["opacity_logits"], self.opacities, stream)
        r = self.renderer
        r.build(V["means"], V["quats"], self.scales, self.opacities, V["rgb"])
        if cams is not None:
            r.set_cameras(cams)
        rgb, _, _ = r.render(None, self.params, stream=stream)
        loss, d_rgb = self.loss_fn(rgb, target, r._cams, stream)
        self.grad.zero_()
        for t in self.g_act.values():
            t.zero_()
        grads = {"means": self.gviews["means"], "quats": self.gviews["quats"], "scales": self.g_act["scales"],
                 "opacities": self.g_act["opacities"], "rgb": self.gviews["rgb"]}
        r.backward(d_rgb, grads=grads, stream=stream)
        sigmoid_backward(self.scales, self.g_act["scales"], self.gviews["scale_logits"], stream)
        sigmoid_backward(self.opacities, self.g_act["opacities"], self.gviews["opacity_logits"], stream)
        self.t += 1
        off = 0
        for name, w in self.GROUPS:
            sl = slice(off, off + self.n * w)
            adam_step(self.flat[sl], self.grad[sl], self.m[sl], self.v[sl], self.t, self.lr[name], stream=stream)
            off += self.n * w
        return loss

    def close(self):
        self.renderer.close()
        self.loss_fn.close()
