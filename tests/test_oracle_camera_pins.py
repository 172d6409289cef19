"""Pins for the oracle's camera rays (or_raygen_f64 / or_raygen_f32) against geometry that does
not depend on how the oracle writes them out.

The paper does not state its camera model; the reading used throughout (the pinhole ray
through the centre of pixel (u, v), unit direction, origin at the camera centre, image x along
the camera's first axis and image y along its second) is checked here by facts that a dropped
+0.5, a flipped image axis, a swapped fx/fy or cx/cy, or a transposed rotation would break:

* projecting a point of the ray back through the pinhole lands on the pixel centre;
* the pixel pair that straddles the principal point is mirror-symmetric about the optical axis;
* the ray through the image's horizontal edge makes half the field of view with the axis;
* moving right in the image turns the ray towards +R_wc column 0, moving down towards column 1;
* the centre pixel of an odd-sized look-at camera points at the look-at target;
* |d| = 1, the origin is the camera centre, and the FP32 ray is within a few ulp of the FP64 one.
"""
import math

import numpy as np

import oracle
from workloads import scenes


def _camera(pos, target, W, H, fov, up=(0.0, 1.0, 0.0), fy_scale=1.0, shift=(0.0, 0.0)):
    c = scenes.look_at_camera(pos, target, W, H, fov, up=up)
    c.fy = (c.fy * np.float32(fy_scale)).astype(np.float32)
    c.cx = (c.cx + np.float32(shift[0])).astype(np.float32)
    c.cy = (c.cy + np.float32(shift[1])).astype(np.float32)
    return c


CAMS = [
    _camera((0.3, -0.2, -4.0), (0.0, 0.0, 0.0), 64, 48, 50.0),
    _camera((12.0, 2.0, 0.0), (0.0, 0.0, 0.0), 1280, 832, 60.0),
    _camera((-3.0, 0.5, 0.7), (0.1, 0.0, 0.0), 37, 23, 45.0, fy_scale=1.3, shift=(2.25, -3.5)),
    _camera((1.0, 5.0, 2.0), (0.0, 0.0, 0.0), 16, 96, 30.0, up=(0.0, 0.0, 1.0)),
]


def _all_pixels(c):
    W, H = int(c.width[0]), int(c.height[0])
    py, px = np.meshgrid(np.arange(H, dtype=np.int32), np.arange(W, dtype=np.int32), indexing="ij")
    return px.ravel(), py.ravel()


def _cam64(c):
    R = c.R_wc[0].astype(np.float64)
    return R, c.pos[0].astype(np.float64), float(c.fx[0]), float(c.fy[0]), float(c.cx[0]), float(c.cy[0])


def test_rays_project_back_onto_the_pixel_centres():
    for c in CAMS:
        px, py = _all_pixels(c)
        o, d = oracle.raygen_f64(c, 0, px, py)
        R, pos, fx, fy, cx, cy = _cam64(c)
        np.testing.assert_array_equal(o, np.broadcast_to(pos, o.shape))
        for t in (0.5, 3.0):
            x = (o + t * d - pos) @ np.linalg.inv(R).T  # world -> camera
            assert np.all(x[:, 2] > 0.0)  # in front of the camera
            u = fx * x[:, 0] / x[:, 2] + cx
            v = fy * x[:, 1] / x[:, 2] + cy
            np.testing.assert_allclose(u, px + 0.5, rtol=0, atol=1e-9 * max(c.width[0], 1))
            np.testing.assert_allclose(v, py + 0.5, rtol=0, atol=1e-9 * max(c.height[0], 1))


def test_unit_directions_and_fp32_close_to_fp64():
    for c in CAMS:
        px, py = _all_pixels(c)
        o64, d64 = oracle.raygen_f64(c, 0, px, py)
        np.testing.assert_allclose(np.linalg.norm(d64, axis=1), 1.0, rtol=0, atol=4e-16)
        o32, d32 = oracle.raygen_f32(c, np.zeros(px.shape, np.int32), px, py)
        np.testing.assert_array_equal(o32, c.pos[0][None].repeat(px.shape[0], 0))
        n32 = np.linalg.norm(d32.astype(np.float64), axis=1)
        assert np.abs(n32 - 1.0).max() <= 3 * 2.0 ** -24
        # a handful of roundings of size ~1: a few ulp of the largest component
        err = np.abs(d32.astype(np.float64) - d64).max(axis=1)
        assert err.max() <= 8 * 2.0 ** -24, err.max()


def test_principal_point_pair_is_mirror_symmetric():
    # cx = W / 2 exactly (even W): pixels W/2 - 1 - i and W/2 + i straddle the axis
    for c in CAMS[:2] + CAMS[3:]:
        W, H = int(c.width[0]), int(c.height[0])
        assert c.cx[0] == W / 2 and c.cy[0] == H / 2
        Ri = np.linalg.inv(c.R_wc[0].astype(np.float64)).T  # d @ Ri: camera-frame direction
        i = np.arange(W // 2, dtype=np.int32)
        row = np.full(i.shape, H // 3, np.int32)
        _, dl = oracle.raygen_f64(c, 0, (W // 2 - 1 - i).astype(np.int32), row)
        _, dr = oracle.raygen_f64(c, 0, (W // 2 + i).astype(np.int32), row)
        # image-plane coordinates x/z, y/z of the camera-frame directions (the FP32 rotation is
        # orthonormal only to FP32 resolution, so the normalisation is compared separately)
        cl, cr = dl @ Ri, dr @ Ri
        cl, cr = cl[:, :2] / cl[:, 2:], cr[:, :2] / cr[:, 2:]
        np.testing.assert_allclose(cl[:, 0], -cr[:, 0], rtol=0, atol=1e-14)
        np.testing.assert_allclose(cl[:, 1], cr[:, 1], rtol=0, atol=1e-14)
        j = np.arange(H // 2, dtype=np.int32)
        col = np.full(j.shape, W // 5, np.int32)
        _, du = oracle.raygen_f64(c, 0, col, (H // 2 - 1 - j).astype(np.int32))
        _, dd = oracle.raygen_f64(c, 0, col, (H // 2 + j).astype(np.int32))
        cu, cd = du @ Ri, dd @ Ri
        cu, cd = cu[:, :2] / cu[:, 2:], cd[:, :2] / cd[:, 2:]
        np.testing.assert_allclose(cu[:, 1], -cd[:, 1], rtol=0, atol=1e-14)
        np.testing.assert_allclose(cu[:, 0], cd[:, 0], rtol=0, atol=1e-14)


def test_edge_rays_make_half_the_field_of_view():
    # the horizontal fov spans the image's full width: the pixel-centre ray of the last column
    # (u + 0.5 = W - 0.5) makes atan((W/2 - 0.5) / (W/2) * tan(fov/2)) with the axis, in the
    # plane of the centre row (odd H: the row through the principal point)
    for W, H, fov in ((64, 33, 50.0), (1280, 833, 60.0), (7, 5, 90.0)):
        c = scenes.look_at_camera((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), W, H, fov)
        axis = np.array([0.0, 0.0, 1.0])
        _, d = oracle.raygen_f64(c, 0, np.array([W - 1, 0], np.int32), np.array([H // 2, H // 2], np.int32))
        want = math.atan((W / 2 - 0.5) / (W / 2) * math.tan(math.radians(fov) / 2))
        for k in range(2):
            ang = math.acos(float(np.clip(d[k] @ axis, -1, 1)))
            assert abs(ang - want) < 1e-6, (W, fov, ang, want)
        # the left and right edge rays are mirror images: together they span the full fov minus
        # the half-pixel insets
        span = math.acos(float(np.clip(d[0] @ d[1], -1, 1)))
        assert abs(span - 2 * want) < 1e-6


def test_image_axes_follow_the_rotation_columns():
    for c in CAMS:
        W, H = int(c.width[0]), int(c.height[0])
        R = c.R_wc[0].astype(np.float64)
        Ri = np.linalg.inv(R).T  # d @ Ri: the direction in camera coordinates (columns of R)
        u = np.arange(W, dtype=np.int32)
        _, d = oracle.raygen_f64(c, 0, u, np.full(u.shape, H // 2, np.int32))
        x = d @ Ri
        assert np.all(np.diff(x[:, 0] / x[:, 2]) > 0)    # right in the image: towards +column 0
        assert np.allclose(np.diff(x[:, 1] / x[:, 2]), 0.0, atol=1e-12)  # along a row: same y
        assert np.all(np.diff(d @ R[:, 0]) > 0)
        v = np.arange(H, dtype=np.int32)
        _, d = oracle.raygen_f64(c, 0, np.full(v.shape, W // 2, np.int32), v)
        x = d @ Ri
        assert np.all(np.diff(x[:, 1] / x[:, 2]) > 0)    # down in the image: towards +column 1
        assert np.allclose(np.diff(x[:, 0] / x[:, 2]), 0.0, atol=1e-12)
        assert np.all(np.diff(d @ R[:, 1]) > 0)
        assert np.all(x[:, 2] > 0)                       # every ray looks forward (+column 2)


def test_centre_pixel_of_an_odd_look_at_camera_points_at_the_target():
    for pos, target in (((0.3, -0.2, -4.0), (0.0, 0.0, 0.0)), ((12.0, 2.0, 0.0), (0.0, 0.5, 0.0)),
                        ((-2.0, 7.0, 3.0), (1.0, -1.0, 0.5))):
        c = scenes.look_at_camera(pos, target, 9, 7, 40.0)
        _, d = oracle.raygen_f64(c, 0, np.array([4], np.int32), np.array([3], np.int32))
        want = np.asarray(target, np.float64) - np.asarray(pos, np.float64)
        want /= np.linalg.norm(want)
        # the camera is stored in FP32, so the axis agrees to FP32 resolution
        assert np.abs(d[0] - want).max() < 1e-6
