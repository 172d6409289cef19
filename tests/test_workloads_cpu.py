"""The seeded synthetic inputs against the recipe the design notes state (shapes, sizes and
value distributions of the stand-ins for the paper's datasets): determinism, ranges, the
flattened and background-shell fractions, the camera ring and the mirror scene's mesh."""
import math

import numpy as np
import pytest

from workloads import scenes


def _flat_fraction(sc, ratio=0.02):
    s = sc.scales.astype(np.float64)
    return float(np.mean(s.min(1) / s.max(1) < ratio))


def test_generators_are_deterministic_per_seed():
    a, b, c = scenes.scene_uniform_cube(500, seed=4), scenes.scene_uniform_cube(500, seed=4), \
        scenes.scene_uniform_cube(500, seed=5)
    for k in ("means", "quats", "scales", "opacities", "rgb"):
        np.testing.assert_array_equal(getattr(a, k), getattr(b, k))
        assert not np.array_equal(getattr(a, k), getattr(c, k))


def test_uniform_cube_recipe():
    sc = scenes.scene_uniform_cube(20000, seed=0)
    assert sc.means.shape == (20000, 3) and sc.means.dtype == np.float32
    assert np.all(np.abs(sc.means) <= 1.0)
    np.testing.assert_allclose(np.linalg.norm(sc.quats.astype(np.float64), axis=1), 1.0, atol=1e-6)
    ls = np.log(sc.scales.astype(np.float64))
    assert abs(ls.mean() + 3.0) < 0.02 and abs(ls.std() - 0.5) < 0.02
    assert sc.opacities.min() >= 0.05 - 1e-6 and sc.opacities.max() <= 0.95 + 1e-6
    assert sc.rgb.min() >= 0.0 and sc.rgb.max() <= 1.0


def test_object_shell_recipe():
    sc = scenes.scene_object_shell(100_000, seed=0)
    r = np.linalg.norm(sc.means.astype(np.float64), axis=1)
    assert abs(r.mean() - 0.8) < 0.005 and abs(r.std() - 0.1) < 0.005
    # 20 % flattened by 100x along one axis: most of them show a scale ratio below 1/50, the
    # others (log-scales N(-4.5, 0.6) per axis) almost never do
    assert 0.15 < _flat_fraction(sc) < 0.21
    o = sc.opacities.astype(np.float64)
    assert abs(o.mean() - 0.5) < 0.005  # Beta(2, 2)


def test_unbounded_recipe():
    sc = scenes.scene_unbounded(200_000, seed=0)
    r = np.linalg.norm(sc.means.astype(np.float64), axis=1)
    shell = np.abs(r - 20.0) < 3.0
    assert 0.09 < shell.mean() < 0.115  # 10 % on the background shell (a few cluster points too)
    assert np.all(np.log(sc.scales.astype(np.float64)) <= -1.0 + 1e-6)  # clipped at -1 before flattening
    assert 0.22 < _flat_fraction(sc) < 0.31  # 30 % flattened
    o = sc.opacities.astype(np.float64)
    assert abs(o.mean() - 0.5) < 0.01  # Beta(0.8, 0.8)
    assert o.min() >= np.float32(1e-4) and o.max() <= np.float32(1 - 1e-4)  # clipped to [1e-4, 1 - 1e-4]


def test_ring_cameras():
    cams = scenes.ring_cameras()
    assert cams.count == 16
    sizes = sorted(zip(cams.width.tolist(), cams.height.tolist()))
    assert sizes.count((1280, 832)) == 8 and sizes.count((960, 640)) == 4 and sizes.count((640, 416)) == 4
    assert int(cams.total_rays()) == 12_042_240
    pos = cams.pos.astype(np.float64)
    np.testing.assert_allclose(np.hypot(pos[:, 0], pos[:, 2]), 12.0, rtol=1e-6)
    np.testing.assert_allclose(pos[:, 1], 2.0, rtol=1e-6)
    # the optical axis (third column of camera-to-world) points at the origin
    fwd = cams.R_wc.astype(np.float64).reshape(-1, 3, 3)[:, :, 2]
    to_origin = -pos / np.linalg.norm(pos, axis=1, keepdims=True)
    np.testing.assert_allclose(np.einsum("ij,ij->i", fwd, to_origin), 1.0, atol=1e-6)
    # horizontal field of view of 60 degrees
    np.testing.assert_allclose(cams.fx.astype(np.float64), cams.width / (2 * math.tan(math.radians(30.0))), rtol=1e-6)


def test_mirror_scene_mesh():
    mesh = scenes.mirror_scene_mesh()
    v = mesh["verts"].astype(np.float64)
    assert v.shape == (50_002, 3, 3)
    sphere = mesh["mat"] == 0
    assert sphere.sum() == 50_000 and (~sphere).sum() == 2
    np.testing.assert_allclose(np.linalg.norm(v[sphere], axis=2), 3.0, rtol=1e-6)
    np.testing.assert_allclose(v[~sphere][:, :, 1], -4.0)
    np.testing.assert_allclose(mesh["albedo"][~sphere], 0.8)
    assert mesh["light"] == (10.0, 15.0, -10.0) and mesh["max_bounces"] == 2


@pytest.mark.parametrize("cfg, name, n", [(1, "1k_gaussians_64x64", 1000), (2, "200k_gaussians_shell_800x800", 200_000)])
def test_small_workloads(cfg, name, n):
    wl = scenes.workload(cfg)
    assert wl.name == name and wl.scene.n == n
