"""Pins for the oracle's scenes with triangles (mirror bounces, diffuse surfaces lit through the
Gaussians by a point light).  The paper shows such scenes but gives no algorithm (Sec. 1, Fig. 1);
the rules are stated in raysplats_oracle.c.  Checked against: the pinned primary renderer (a
scene without triangles), closed forms for a flat mirror and for a shadow ray through one
Gaussian, FP64 point-in-triangle geometry, and FP64 central differences."""
import math

import numpy as np
import pytest

import oracle
from workloads import scenes

Q99 = scenes.default_Q()


def _quad(z=None, y=None, half=10.0, mat=0, albedo=(0.0, 0.0, 0.0)):
    if z is not None:
        v = np.array([[-half, -half, z], [half, -half, z], [half, half, z], [-half, half, z]], np.float32)
    else:
        v = np.array([[-half, y, -half], [half, y, -half], [half, y, half], [-half, y, half]], np.float32)
    tris = np.stack([v[[0, 1, 2]], v[[0, 2, 3]]])
    return tris, np.full(2, mat, np.int32), np.tile(np.asarray(albedo, np.float32), (2, 1))


def _mesh(parts, light=(0.0, 10.0, 0.0), max_bounces=2, eps_off=1e-3):
    verts = np.concatenate([p[0] for p in parts]) if parts else np.zeros((0, 3, 3), np.float32)
    mat = np.concatenate([p[1] for p in parts]) if parts else np.zeros(0, np.int32)
    alb = np.concatenate([p[2] for p in parts]) if parts else np.zeros((0, 3), np.float32)
    return {"verts": verts, "mat": mat, "albedo": alb, "light": light, "max_bounces": max_bounces, "eps_off": eps_off}


def _iso(means, scale, ops, cols):
    n = len(ops)
    return scenes.Scene(np.asarray(means, np.float32), np.tile(np.array([[1, 0, 0, 0]], np.float32), (n, 1)),
                        np.full((n, 3), scale, np.float32), np.asarray(ops, np.float32), np.asarray(cols, np.float32))


def _unit(v):
    v = np.asarray(v, np.float64)
    return (v / np.linalg.norm(v)).astype(np.float32)


def test_without_triangles_it_is_the_primary_renderer():
    sc = scenes.random_tiny_scene(7, n=40)
    cams = scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 12, 10, 55.0)
    gx, gy = np.meshgrid(np.arange(12), np.arange(10))
    o, d = oracle.raygen_f32(cams, np.zeros(120, np.int32), gx.ravel(), gy.ravel())
    rng = np.random.default_rng(1)
    gc, ga, gd = rng.standard_normal((120, 3)), rng.standard_normal(120), rng.standard_normal(120)
    kw = dict(Q=Q99, eps1=1e-3, background=(0.2, 0.3, 0.4))
    a = oracle.render_rays(sc, o, d, dl_rgb=gc, dl_alpha=ga, dl_depth=gd, **kw)
    b = oracle.render_scene(sc, _mesh([]), o, d, dl_rgb=gc, dl_alpha=ga, dl_depth=gd, **kw)
    for k in ("rgb", "alpha", "depth"):
        np.testing.assert_allclose(b[k], a[k], atol=1e-14)
    for k in a["grads"]:
        np.testing.assert_allclose(b["grads"][k], a["grads"][k], atol=1e-12)


def test_triangle_hits_follow_fp64_geometry():
    """A diffuse plane, no Gaussians: each pixel is the albedo where the ray meets the triangle
    (FP64 point-in-triangle test away from the edges) and the background elsewhere."""
    tris, mat, alb = _quad(z=1.0, half=0.7, mat=1, albedo=(0.5, 0.6, 0.7))
    mesh = _mesh([(tris, mat, alb)], light=(0.0, 0.0, -5.0))
    cams = scenes.look_at_camera((0.0, 0.0, -2.0), (0, 0, 0), 32, 32, 60.0)
    gx, gy = np.meshgrid(np.arange(32), np.arange(32))
    o, d = oracle.raygen_f32(cams, np.zeros(1024, np.int32), gx.ravel(), gy.ravel())
    empty = _iso(np.zeros((0, 3)), 0.1, [], np.zeros((0, 3)))
    out = oracle.render_scene(empty, mesh, o, d, Q99, background=(0.0, 0.0, 0.0))
    t = (1.0 - o[:, 2].astype(np.float64)) / d[:, 2]
    P = o + t[:, None] * d
    inside = (np.abs(P[:, 0]) < 0.7 - 1e-4) & (np.abs(P[:, 1]) < 0.7 - 1e-4)
    outside = (np.abs(P[:, 0]) > 0.7 + 1e-4) | (np.abs(P[:, 1]) > 0.7 + 1e-4)
    assert inside.sum() > 100 and outside.sum() > 100
    np.testing.assert_allclose(out["rgb"][inside], np.tile([0.5, 0.6, 0.7], (inside.sum(), 1)), atol=1e-7)
    np.testing.assert_allclose(out["rgb"][outside], 0.0, atol=0)


def test_flat_mirror_closed_form():
    """Camera ray to the mirror point (1, 0, 0) of the plane z = 0 reflects to (2, 0, -5); a
    Gaussian centred on the reflected ray at (1.4, 0, -2) and far from the incoming one gives
    alpha = opacity and rgb = alpha c + (1 - alpha) background."""
    tris, mat, alb = _quad(z=0.0, mat=0)
    mesh = _mesh([(tris, mat, alb)], max_bounces=2)
    sc = _iso([[1.4, 0.0, -2.0]], 0.05, [0.7], [[0.2, 0.5, 0.9]])
    o = np.array([[0.0, 0.0, -5.0]], np.float32)
    d = _unit([1.0, 0.0, 5.0])[None]
    bg = np.array([0.1, 0.3, 0.2])
    out = oracle.render_scene(sc, mesh, o, d, Q99, background=tuple(bg))
    a = float(np.float32(0.7))
    np.testing.assert_allclose(out["rgb"][0], a * np.float32([0.2, 0.5, 0.9]) + (1 - a) * bg, atol=1e-6)
    assert out["n_hits"][0] == 1 and out["depth"][0] == 0.0  # the hit is on the second segment
    # with no bounce allowed, the mirror returns nothing
    out0 = oracle.render_scene(sc, dict(mesh, max_bounces=0), o, d, Q99, background=tuple(bg))
    np.testing.assert_array_equal(out0["rgb"][0], 0.0)


def test_shadow_ray_through_one_gaussian_closed_form():
    """Ground plane y = 0 (albedo a), light at (0, 10, 0); the camera ray meets the plane at the
    origin; a Gaussian centred at (0, 4, 0) lies on the shadow ray: rgb = a (1 - opacity).  A
    triangle between the plane and the light blocks it: rgb = 0."""
    tris, mat, alb = _quad(y=0.0, mat=1, albedo=(0.5, 0.6, 0.7))
    sc = _iso([[0.0, 4.0, 0.0]], 0.1, [0.6], [[1.0, 0.0, 0.0]])
    o = np.array([[0.0, 5.0, -5.0]], np.float32)
    d = _unit([0.0, -5.0, 5.0])[None]
    out = oracle.render_scene(sc, _mesh([(tris, mat, alb)]), o, d, Q99)
    np.testing.assert_allclose(out["rgb"][0], np.float32([0.5, 0.6, 0.7]) * (1 - float(np.float32(0.6))), atol=1e-6)
    blocker = _quad(y=7.0, half=1.0, mat=1, albedo=(1.0, 1.0, 1.0))
    out2 = oracle.render_scene(sc, _mesh([(tris, mat, alb), blocker]), o, d, Q99)
    np.testing.assert_array_equal(out2["rgb"][0], 0.0)
    # the shadow ray's own eps1 cut: a product of (1 - alpha) below eps1 is opaque
    two = _iso([[0.0, 4.0, 0.0], [0.0, 6.0, 0.0]], 0.1, [0.6, 0.6], [[1.0, 0.0, 0.0], [0.0, 1.0, 0.0]])
    a = float(np.float32(0.6))
    lit = oracle.render_scene(two, _mesh([(tris, mat, alb)]), o, d, Q99, eps1=0.1)
    np.testing.assert_allclose(lit["rgb"][0], np.float32([0.5, 0.6, 0.7]) * (1 - a) ** 2, atol=1e-6)
    cut = oracle.render_scene(two, _mesh([(tris, mat, alb)]), o, d, Q99, eps1=0.2)
    np.testing.assert_array_equal(cut["rgb"][0], 0.0)


@pytest.mark.parametrize("seed", [1, 2])
def test_scene_gradient_matches_central_differences(seed):
    """Mirror bounces, a diffuse plane lit through the Gaussians: the analytic gradient of
    <gc, rgb> + <ga, alpha> + <gd, depth> w.r.t. every Gaussian parameter against FP64 central
    differences (rays with a flagged decision excluded)."""
    rng = np.random.default_rng(seed)
    n = 14
    means = rng.uniform(-0.6, 0.6, (n, 3)) + np.array([0.0, 0.4, 0.0])
    sc = scenes.Scene(means.astype(np.float32), rng.standard_normal((n, 4)).astype(np.float32),
                      np.exp(rng.normal(-1.6, 0.3, (n, 3))).astype(np.float32), rng.uniform(0.1, 0.9, n).astype(np.float32),
                      rng.uniform(0, 1, (n, 3)).astype(np.float32))
    mirror = _quad(z=1.2, half=1.5, mat=0)
    floor = _quad(y=-0.8, half=3.0, mat=1, albedo=(0.6, 0.5, 0.4))
    mesh = _mesh([mirror, floor], light=(0.3, 3.0, -1.0), max_bounces=2)
    cams = scenes.look_at_camera((0.3, 0.6, -2.5), (0, 0, 0.5), 10, 9, 60.0)
    gx, gy = np.meshgrid(np.arange(10), np.arange(9))
    o, d = oracle.raygen_f32(cams, np.zeros(90, np.int32), gx.ravel(), gy.ravel())
    gc, ga, gd = rng.standard_normal((90, 3)), rng.standard_normal(90), rng.standard_normal(90)
    kw = dict(Q=Q99, eps1=1e-3, background=(0.2, 0.3, 0.4))
    base = oracle.render_scene(sc, mesh, o, d, **kw)
    ok = base["mask"] == 0
    assert ok.mean() > 0.8
    gc[~ok], ga[~ok], gd[~ok] = 0.0, 0.0, 0.0
    base = oracle.render_scene(sc, mesh, o, d, dl_rgb=gc, dl_alpha=ga, dl_depth=gd, **kw)
    P = {k: getattr(sc, k).astype(np.float64).copy() for k in ("means", "quats", "scales", "opacities", "rgb")}

    def loss(params):
        out = oracle.render_scene(None, mesh, o, d, params64=params, **kw)
        return float(np.sum(out["rgb"] * gc) + np.sum(out["alpha"] * ga) + np.sum(out["depth"] * gd))

    for key in P:
        fd = np.zeros_like(P[key])
        flat = P[key].reshape(-1)
        for j in range(flat.size):
            x = flat[j]
            h = 1e-6 * max(1.0, abs(x))
            flat[j] = x + h
            lp = loss(P)
            flat[j] = x - h
            lm = loss(P)
            flat[j] = x
            fd.reshape(-1)[j] = (lp - lm) / (2 * h)
        an = base["grads"][key]
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-300)
        assert err < 1e-6, (key, err)
