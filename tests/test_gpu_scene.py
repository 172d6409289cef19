"""GPU parity of the scene renderer (Gaussians with a mirror mesh and a diffuse floor lit through
the Gaussians by a point light) against the oracle's scene renderer (raysplats_oracle.c), and
its consistency with the plain renderer on a scene without triangles."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_GRAD, TOL_RGB, params, pixel_index, rel_l2, to_dev
from workloads import scenes

pytestmark = pytest.mark.gpu

KEYS = ("means", "quats", "scales", "opacities", "rgb")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _quad(z=None, y=None, half=10.0, mat=0, albedo=(0.0, 0.0, 0.0), cx=0.0):
    if z is not None:
        v = np.array([[cx - half, -half, z], [cx + half, -half, z], [cx + half, half, z], [cx - half, half, z]], np.float32)
    else:
        v = np.array([[-half, y, -half], [half, y, -half], [half, y, half], [-half, y, half]], np.float32)
    return np.stack([v[[0, 1, 2]], v[[0, 2, 3]]]), np.full(2, mat, np.int32), np.tile(np.asarray(albedo, np.float32), (2, 1))


def _mesh(parts, light, max_bounces=2, eps_off=1e-3):
    if not parts:
        return {"verts": np.zeros((0, 3, 3), np.float32), "mat": np.zeros(0, np.int32), "albedo": np.zeros((0, 3), np.float32),
                "light": light, "max_bounces": max_bounces, "eps_off": eps_off}
    return {"verts": np.concatenate([p[0] for p in parts]), "mat": np.concatenate([p[1] for p in parts]),
            "albedo": np.concatenate([p[2] for p in parts]), "light": light, "max_bounces": max_bounces,
            "eps_off": eps_off}


def _case(seed, n=300):
    sc = scenes.random_tiny_scene(seed, n=n, spread=0.7, log_mu=-2.6)
    sc = scenes.Scene(sc.means + np.array([0.0, 0.3, 0.0], np.float32), sc.quats, sc.scales, sc.opacities, sc.rgb)
    mirror = _quad(z=1.2, half=1.5, mat=0)
    floor = _quad(y=-0.8, half=3.0, mat=1, albedo=(0.6, 0.5, 0.4))
    sphere = scenes.uv_sphere(0.35, 16, 8, center=(-0.9, 0.2, 0.6))
    sph = (sphere, np.zeros(len(sphere), np.int32), np.zeros((len(sphere), 3), np.float32))
    mesh = _mesh([mirror, floor, sph], light=(0.3, 3.0, -1.0))
    cams = scenes.concat_cameras([scenes.look_at_camera((0.3, 0.6, -2.5), (0, 0, 0.5), 40, 30, 60.0),
                                  scenes.look_at_camera((-1.5, 1.5, -1.8), (0, 0, 0.5), 24, 24, 55.0)])
    return sc, mesh, cams


def _gpu(sc, mesh, cams, prm, grads_in=None, list_cap=512, tune_kw=None):
    from paper_2501_19196_gb300 import native
    from paper_2501_19196_gb300.scene import SceneRenderer
    sr = SceneRenderer(mesh, tune=native.default_tune(**(tune_kw or {})), Q_box=scenes.default_Q(), list_cap=list_cap)
    sr.build(*to_dev(sc))
    rgb, alpha, depth = sr.render(cams, prm)
    grads = None
    if grads_in is not None:
        g = [None if x is None else torch.from_numpy(np.ascontiguousarray(x, np.float32)).cuda() for x in grads_in]
        grads = sr.backward(*g)
    torch.cuda.synchronize()
    sr.check_device()
    out = {"rgb": rgb.cpu().numpy().astype(np.float64), "alpha": alpha.cpu().numpy().astype(np.float64),
           "depth": depth.cpu().numpy().astype(np.float64)}
    if grads is not None:
        out["grads"] = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    sr.close()
    return out


def _rays(cams):
    """FP32 camera rays of every pixel, and their rows in the rs_render layout."""
    cam, px, py = scenes.pixel_grid(cams)
    o, d = oracle.raygen_f32(cams, cam, px, py)
    return o, d, pixel_index(cams, cam, px, py)


def test_without_triangles_equals_the_plain_renderer():
    from gpu_util import gpu_render
    sc, _, cams = _case(3)
    prm = params(eps1=1e-3, background=(0.2, 0.3, 0.4))
    a = gpu_render(sc, cams, prm)
    b = _gpu(sc, _mesh([], light=(0.0, 5.0, 0.0)), cams, prm)
    for k in ("rgb", "alpha", "depth"):
        np.testing.assert_array_equal(b[k], a[k], err_msg=k)


def test_leaf_size_does_not_change_the_scene_image():
    """The leaf size changes the order in which the packets meet the Gaussians.  Alpha and depth
    come from the sorted camera-ray segments: the same bits.  A shadow ray multiplies its
    (1 - alpha) factors in traversal order, so the lit colours may differ in their last bits
    (measured up to 9e-8)."""
    sc, mesh, cams = _case(2, n=600)
    prm = params(eps1=1e-3, background=(0.2, 0.3, 0.4))
    a = _gpu(sc, mesh, cams, prm)
    for kw in (dict(leaf_size=16), dict(leaf_size=8), dict(leaf_size=1)):
        b = _gpu(sc, mesh, cams, prm, tune_kw=kw)
        for k in ("alpha", "depth"):
            np.testing.assert_array_equal(b[k], a[k], err_msg=f"{k} {kw}")
        np.testing.assert_allclose(b["rgb"], a["rgb"], rtol=0, atol=1e-6, err_msg=f"rgb {kw}")


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_image_matches_the_scene_oracle(seed):
    sc, mesh, cams = _case(seed)
    prm = params(eps1=1e-3, background=(0.2, 0.3, 0.4))
    g = _gpu(sc, mesh, cams, prm)
    o, d, idx = _rays(cams)
    ora = oracle.render_scene(sc, mesh, o, d, prm.Q, eps1=prm.eps1, background=prm.background)
    ok = ora["mask"] == 0
    e_rgb = np.abs(g["rgb"][idx][ok] - ora["rgb"][ok]).max()
    e_a = np.abs(g["alpha"][idx][ok] - ora["alpha"][ok]).max()
    e_d = (np.abs(g["depth"][idx][ok] - ora["depth"][ok]) / np.maximum(1.0, ora["depth"][ok])).max()
    print(f"[parity] scene seed {seed}: rays {len(ok)} masked {1 - ok.mean():.4f} max|d rgb| {e_rgb:.2e} "
          f"max|d alpha| {e_a:.2e} depth rel {e_d:.2e}")
    # the scene oracle masks every ray with an FP32-sensitive decision (surface edges and ties,
    # Gaussian boundaries and ties, eps1), without testing its impact: measured at most 0.11 %
    assert ok.mean() >= 0.997
    assert e_rgb <= TOL_RGB and e_a <= TOL_RGB and e_d <= 1e-3


@pytest.mark.parametrize("seed", [4, 5])
def test_gradients_match_the_scene_oracle(seed):
    sc, mesh, cams = _case(seed, n=120)
    prm = params(eps1=1e-3, background=(0.2, 0.3, 0.4))
    o, d, idx = _rays(cams)
    R = o.shape[0]
    ora0 = oracle.render_scene(sc, mesh, o, d, prm.Q, eps1=prm.eps1, background=prm.background)
    bad = ora0["mask"] != 0
    rng = np.random.default_rng(seed)
    gc, ga, gd = rng.standard_normal((R, 3)), rng.standard_normal(R), rng.standard_normal(R)
    gc[bad], ga[bad], gd[bad] = 0.0, 0.0, 0.0
    ora = oracle.render_scene(sc, mesh, o, d, prm.Q, eps1=prm.eps1, background=prm.background,
                              dl_rgb=gc, dl_alpha=ga, dl_depth=gd)
    P = int(cams.total_rays())
    full = [np.zeros((P, 3)), np.zeros(P), np.zeros(P)]
    full[0][idx], full[1][idx], full[2][idx] = gc, ga, gd
    g = _gpu(sc, mesh, cams, prm, grads_in=full)
    errs = {k: rel_l2(g["grads"][k].reshape(ora["grads"][k].shape), ora["grads"][k]) for k in KEYS}
    print(f"[parity] scene gradients seed {seed}: masked {bad.mean():.4f}", {k: f"{v:.2e}" for k, v in errs.items()})
    assert max(errs.values()) < TOL_GRAD, errs


def test_short_id_lists_are_reported():
    """A list too short for a ray's hits is an error the device check reports (no fault)."""
    from paper_2501_19196_gb300 import native
    sc, mesh, cams = _case(6)
    with pytest.raises(native.RaySplatsError, match="id-list-overflow"):
        _gpu(sc, mesh, cams, params(eps1=1e-3), list_cap=1)


def test_mirror_workload_full_size_sampled():
    """The full mirror / shadow workload (2M Gaussians, 50,002 triangles, one 1280 x 832 camera)
    in the launch configuration the benchmark times: the whole frame and its adjoint run without
    a device error (loop guards, list overflow), and sampled pixels match the oracle in the
    image and, with an upstream gradient on those pixels only, in every gradient array."""
    from paper_2501_19196_gb300 import native
    from paper_2501_19196_gb300.scene import SceneRenderer
    sc, mesh, cams = scenes.workload_mirror()
    prm = params(eps1=1e-4)
    cam, px, py = scenes.pixel_grid(cams, stride=101)
    o, d = oracle.raygen_f32(cams, cam, px, py)
    idx = pixel_index(cams, cam, px, py)
    ora0 = oracle.render_scene(sc, mesh, o, d, prm.Q, eps1=prm.eps1, background=prm.background)
    ok = ora0["mask"] == 0
    rng = np.random.default_rng(9)
    gc, ga = rng.standard_normal((len(cam), 3)), rng.standard_normal(len(cam))
    gc[~ok], ga[~ok] = 0.0, 0.0
    ora = oracle.render_scene(sc, mesh, o, d, prm.Q, eps1=prm.eps1, background=prm.background, dl_rgb=gc, dl_alpha=ga)
    P = int(cams.total_rays())
    full = [np.zeros((P, 3), np.float32), np.zeros(P, np.float32)]
    full[0][idx], full[1][idx] = gc, ga
    sr = SceneRenderer(mesh, tune=native.default_tune(), Q_box=scenes.default_Q(), list_cap=1024, shadow_cap=1024)
    sr.build(*to_dev(sc))
    rgb, alpha, _ = sr.render(cams, prm)
    grads = sr.backward(torch.from_numpy(full[0]).cuda(), torch.from_numpy(full[1]).cuda())
    torch.cuda.synchronize()
    sr.check_device()
    rgb, alpha = rgb.cpu().numpy().astype(np.float64), alpha.cpu().numpy().astype(np.float64)
    grads = {k: v.cpu().numpy().astype(np.float64) for k, v in grads.items()}
    sr.close()
    e_rgb = np.abs(rgb[idx][ok] - ora["rgb"][ok]).max()
    e_a = np.abs(alpha[idx][ok] - ora["alpha"][ok]).max()
    errs = {k: rel_l2(grads[k].reshape(ora["grads"][k].shape), ora["grads"][k]) for k in KEYS}
    print(f"[parity] mirror workload sampled: pixels {len(cam)} masked {1 - ok.mean():.4f} max|d rgb| {e_rgb:.2e} "
          f"max|d alpha| {e_a:.2e}", {k: f"{v:.2e}" for k, v in errs.items()})
    # every flagged decision masks (no impact test); 117 rays, one of them masked (0.85 %)
    assert (~ok).sum() <= 2
    assert e_rgb <= TOL_RGB and e_a <= TOL_RGB
    assert max(errs.values()) < TOL_GRAD, errs
