"""GPU parity of the forward path (LBVH build, traversal, compositing) against the FP64 oracle,
called through the C ABI.  Bit-exact where the work is integer or a fixed FP32 sequence (rays,
Morton codes, sorted order, radix tree); within 2e-4 absolute per RGB/alpha channel on every
pixel whose value is unique at that tolerance (oracle IMPACT flag clear)."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import (TOL_RGB, compare_image, gpu_render, oracle_pixels, params, pixel_index, to_dev)
from workloads import scenes

pytestmark = pytest.mark.gpu

Q = scenes.default_Q()


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2501_19196_gb300 import native
    native.load()


# ------------------------------------------------------------------------------------------
# bit-exact stages
# ------------------------------------------------------------------------------------------
def test_camera_rays_bit_exact():
    from paper_2501_19196_gb300 import debug_rays
    cams = scenes.concat_cameras([scenes.ring_cameras(), scenes.look_at_camera((0.3, -0.2, -4), (0, 0, 0), 37, 23, 50)])
    rng = np.random.default_rng(0)
    cam = rng.integers(0, cams.count, 20000).astype(np.int32)
    px = (rng.random(20000) * cams.width[cam]).astype(np.int32)
    py = (rng.random(20000) * cams.height[cam]).astype(np.int32)
    px[:17], py[:17] = 0, 0
    o_ref, d_ref = oracle.raygen_f32(cams, cam, px, py)
    t = lambda a: torch.from_numpy(a).cuda()  # noqa: E731
    o, d = debug_rays(cams, t(cam), t(px), t(py))
    np.testing.assert_array_equal(o.cpu().numpy().view(np.uint32), o_ref.view(np.uint32))
    np.testing.assert_array_equal(d.cpu().numpy().view(np.uint32), d_ref.view(np.uint32))


def _export(scene, **tune):
    from paper_2501_19196_gb300 import Renderer, native
    r = Renderer(tune=native.default_tune(**tune))
    r.build(*to_dev(scene))
    torch.cuda.synchronize()
    ex = r.export_accel()
    r.check_device()
    r.close()
    return ex


@pytest.mark.parametrize("bits", [10, 20, 21])
@pytest.mark.parametrize("which", ["cube1k", "dups", "clusters"])
def test_morton_codes_and_order_bit_exact(bits, which):
    if which == "cube1k":
        sc = scenes.workload(1).scene
    elif which == "dups":
        sc = scenes.random_tiny_scene(5, n=30000)
        sc.means[::3] = sc.means[1::3][: sc.means[::3].shape[0]]  # many duplicate means
    else:
        sc = scenes.scene_unbounded(200_000, seed=3)
    ex = _export(sc, morton_bits=bits)
    codes, lohi = oracle.morton(sc.means, bits, sc.scales)
    perm, sorted_codes = oracle.sort_perm(codes)
    np.testing.assert_array_equal(ex["lo_hi"], lohi)
    np.testing.assert_array_equal(ex["codes"], sorted_codes)
    np.testing.assert_array_equal(ex["perm"], perm)


@pytest.mark.parametrize("n,bits", [(2, 21), (3, 21), (1000, 21), (40000, 10), (20000, 20)])
def test_radix_tree_matches_definition(n, bits):
    sc = scenes.random_tiny_scene(n, n=n, spread=2.0)
    ex = _export(sc, morton_bits=bits)
    f, l, s = oracle.radix_tree(ex["codes"])
    np.testing.assert_array_equal(ex["first"][: n - 1], f)
    np.testing.assert_array_equal(ex["last"][: n - 1], l)
    np.testing.assert_array_equal(ex["split"][: n - 1], s)


def test_boxes_conservative_and_nested():
    sc = scenes.scene_object_shell(20000, seed=2)
    ex = _export(sc)
    perm = ex["perm"].astype(np.int64)
    pb = ex["prim_boxes"].astype(np.float64)
    # the ellipsoid |M(x-m)|^2 <= Q extends sqrt(Q)*|row_a(R S)| along world axis a (FP64 here)
    from scipy.spatial.transform import Rotation
    q = sc.quats[perm].astype(np.float64)
    R = Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    RS = R * sc.scales[perm].astype(np.float64)[:, None, :]
    ext = np.sqrt(Q) * np.linalg.norm(RS, axis=2)
    m = sc.means[perm].astype(np.float64)
    assert np.all(pb[:, :3] <= m - ext) and np.all(pb[:, 3:] >= m + ext)
    assert np.all(pb[:, :3] >= m - ext * 1.01 - 1e-5) and np.all(pb[:, 3:] <= m + ext * 1.01 + 1e-5)
    # internal boxes contain their children (children from first/last/split)
    n = sc.n
    f, l, s, nb = ex["first"], ex["last"], ex["split"], ex["boxes"]

    def box(child_first, child_last, internal_index):
        if child_first == child_last:
            return pb[child_first]
        return nb[internal_index]

    for i in range(0, n - 1, 97):
        lb = box(f[i], s[i], s[i])
        rb = box(s[i] + 1, l[i], s[i] + 1)
        for cb in (lb, rb):
            assert np.all(nb[i][:3] <= cb[:3]) and np.all(nb[i][3:] >= cb[3:])


# ------------------------------------------------------------------------------------------
# ray / ellipsoid numerics (Prop. 1, Prop. 2)
# ------------------------------------------------------------------------------------------
def test_hit_test_numerics_against_fp64():
    from paper_2501_19196_gb300 import Renderer
    sc = scenes.scene_unbounded(100_000, seed=4)
    r = Renderer()
    r.build(*to_dev(sc))
    ex = r.export_accel()
    perm = ex["perm"].astype(np.int64)
    cams = scenes.ring_cameras()
    rng = np.random.default_rng(1)
    # rays aimed near random Gaussians so that most pairs are hits or near misses
    k = 20000
    j = rng.integers(0, sc.n, k)
    gi = perm[j]
    c = rng.integers(0, cams.count, k)
    o = cams.pos[c].astype(np.float32)
    target = sc.means[gi] + rng.normal(0, 2.5, (k, 3)) * sc.scales[gi].max(1, keepdims=True)
    d = (target - o).astype(np.float64)
    d = (d / np.linalg.norm(d, axis=1, keepdims=True)).astype(np.float32)
    out = r.debug_hits(torch.from_numpy(o).cuda(), torch.from_numpy(d).cuda(),
                       torch.from_numpy(j.astype(np.int32)).cuda(), Q).cpu().numpy().astype(np.float64)
    r.close()
    D2 = np.zeros(k)
    t1 = np.zeros(k)
    tau = np.zeros(k)
    tol = np.zeros(k)
    d2tol = np.zeros(k)
    mtol = np.zeros(k)
    hit = np.zeros(k, bool)
    for t in range(k):
        D2[t], t1[t], hit[t], tau[t], tol[t], d2tol[t], mtol[t] = oracle.ray_gaussian(
            o[t], d[t], sc.means[gi[t]], sc.quats[gi[t]], sc.scales[gi[t]], Q, with_tol=True)
    near = D2 <= Q * (1.0 + 1e-3)  # pairs whose D2 decides a hit
    ratio_d2 = np.abs(out[near, 0] - D2[near]) / d2tol[near]
    clear = np.abs(D2 - Q) >= d2tol   # outside the oracle's boundary band
    assert np.mean(hit) > 0.2
    assert np.all((out[clear, 2] > 0.5) == hit[clear])
    both = clear & hit
    errD = np.abs(out[both, 0] - D2[both]) / np.maximum(1.0, D2[both])
    errt = np.abs(out[both, 1] - t1[both]) / np.maximum(1.0, np.abs(t1[both]))
    # the ordering parameter: t1 plus the key's sub-ulp residual
    ulp = np.ldexp(1.0, np.frexp(out[both, 1])[1] - 24)
    t_key = out[both, 1] + out[both, 4] * ulp
    quantum = ulp * np.ldexp(1.0, -out[both, 5].astype(np.int64))
    err_key = np.abs(t_key - t1[both])
    ratio = err_key / (tol[both] + 0.5 * quantum)
    # the t_m ordering (sort key 1): max(t_m, t1) plus its residual
    ulp_m = np.ldexp(1.0, np.frexp(out[both, 6])[1] - 24)
    tm_key = out[both, 6] + out[both, 7] * ulp_m
    err_m = np.abs(tm_key - np.maximum(-tau[both], t1[both]))
    # where t_m and t1 are within their bands the key is whichever FP32 found larger
    sep = np.abs(-tau[both] - t1[both]) > mtol[both] + tol[both]
    ratio_m = err_m[sep] / (mtol[both][sep] + 0.5 * ulp_m[sep] * np.ldexp(1.0, -out[both, 5][sep].astype(np.int64)))
    print(f"hit numerics: max |dD2|/max(1,D2) = {errD.max():.3e}, max |dt1|/max(1,t1) = {errt.max():.3e}; "
          f"ordering key: max error {np.max(err_key / ulp):.3e} ulp (median {np.median(err_key / ulp):.2e}), "
          f"max error / oracle band {ratio.max():.3f} (99.9% {np.quantile(ratio, 0.999):.3f}); "
          f"t_m key: max error / oracle band {ratio_m.max():.3f} (99.9% {np.quantile(ratio_m, 0.999):.3f}, "
          f"{sep.sum()} hits); "
          f"D2: max error / oracle band {ratio_d2.max():.3f} (99.9% {np.quantile(ratio_d2, 0.999):.3f})")
    assert errD.max() < 1e-5
    assert errt.max() < 2.5e-7
    # the oracle's per-hit TIE (t1 and t_m orderings) and BOUNDARY bands cover the errors with a
    # margin of two
    assert sep.sum() > 0.9 * both.sum()
    assert ratio.max() < 0.5
    assert ratio_m.max() < 0.5
    assert ratio_d2.max() < 0.5


# ------------------------------------------------------------------------------------------
# full forward parity
# ------------------------------------------------------------------------------------------
def test_forward_workload_1k_full_frame():
    wl = scenes.workload(1)
    prm = params(eps1=wl.eps1, background=wl.background)
    g = gpu_render(wl.scene, wl.cams, prm)
    cam, px, py = scenes.pixel_grid(wl.cams)
    ora = oracle_pixels(wl.scene, wl.cams, cam, px, py, prm)
    err, masked = compare_image(g, ora, pixel_index(wl.cams, cam, px, py), label="1k 64x64")
    print(f"1k/64x64: max err {err:.2e}, masked {masked:.4f}")


CASES = [
    dict(eps1=1e-4), dict(eps1=0.0), dict(eps1=0.3), dict(k_max=1), dict(k_max=3), dict(k_max=16),
    dict(Q=4.0), dict(Q=9.0), dict(Q=16.0), dict(background=(0.2, 0.5, 1.0)), dict(t_near=2.9),
    dict(sort_key=1), dict(sort_key=1, eps1=0.3, k_max=5), dict(sort_key=1, t_near=2.9),
]


@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("case", range(len(CASES)))
def test_forward_random_tiny_scenes(seed, case):
    kw = CASES[case]
    sc = scenes.random_tiny_scene(100 + seed, n=64, flat_frac=0.3 if seed % 2 else 0.0)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 19, 13, 55.0),
                                  scenes.look_at_camera((-3.0, 0.5, 0.7), (0.1, 0, 0), 16, 16, 45.0)])
    prm = params(**kw)
    g = gpu_render(sc, cams, prm)
    cam, px, py = scenes.pixel_grid(cams)
    ora = oracle_pixels(sc, cams, cam, px, py, prm)
    # 503 pixels: one masked pixel is 0.2 %; at most two (measured: at most one)
    compare_image(g, ora, pixel_index(cams, cam, px, py), max_masked=0.004, label=f"seed {seed} {kw}")


def test_forward_shell_200k_sampled_and_crop():
    wl = scenes.workload(2)
    prm = params(eps1=wl.eps1, background=wl.background)
    g = gpu_render(wl.scene, wl.cams, prm)
    cam, px, py = scenes.pixel_grid(wl.cams, stride=20)
    ora = oracle_pixels(wl.scene, wl.cams, cam, px, py, prm)
    err, masked = compare_image(g, ora, pixel_index(wl.cams, cam, px, py), label="200k sampled")
    print(f"200k/800x800 sampled: max err {err:.2e}, masked {masked:.4f}, pixels {len(cam)}")
    # a crop: a 48x40 window of the frame as its own camera
    c = wl.cams
    crop = scenes.Cameras(c.R_wc.copy(), c.pos.copy(), c.fx.copy(), c.fy.copy(), c.cx - 380, c.cy - 300,
                          np.array([48], np.int32), np.array([40], np.int32))
    g2 = gpu_render(wl.scene, crop, prm)
    cam, px, py = scenes.pixel_grid(crop)
    ora = oracle_pixels(wl.scene, crop, cam, px, py, prm)
    # the crop looks through both walls of the shell near its centre (about twice the hits of an
    # average ray, spaced about 2e-3 apart): 3 of its 1,920 rays (0.16 %) hold a pair of hits
    # closer than their FP32 uncertainty whose swap changes the colour by more than 1e-4
    compare_image(g2, ora, pixel_index(crop, cam, px, py), max_masked=0.0025, label="200k crop")


def test_forward_unbounded_1m_sampled():
    wl = scenes.workload(3)
    prm = params(eps1=wl.eps1, background=wl.background)
    g = gpu_render(wl.scene, wl.cams, prm)
    cam, px, py = scenes.pixel_grid(wl.cams, stride=33)
    ora = oracle_pixels(wl.scene, wl.cams, cam, px, py, prm)
    # 1,014 pixels: one masked pixel is 0.1 % (measured: one, a D2 within FP32 error of Q)
    err, masked = compare_image(g, ora, pixel_index(wl.cams, cam, px, py), max_masked=0.002, label="1M sampled")
    print(f"1M/1280x832 sampled: max err {err:.2e}, masked {masked:.4f}, pixels {len(cam)}")


# ------------------------------------------------------------------------------------------
# tunables and launch modes never change a result
# ------------------------------------------------------------------------------------------
def test_tunables_and_launch_modes_bit_identical():
    from paper_2501_19196_gb300 import native
    sc = scenes.scene_object_shell(30000, seed=7)
    cams = scenes.concat_cameras([scenes.look_at_camera((0, 0.5, -3.5), (0, 0, 0), 97, 61, 50),
                                  scenes.look_at_camera((3.0, 1.0, 1.0), (0, 0, 0), 64, 64, 40),
                                  scenes.look_at_camera((-2.0, -2.5, 1.5), (0, 0, 0), 33, 70, 60)])
    prm = params(eps1=1e-3, background=(1, 1, 1))
    ref = gpu_render(sc, cams, prm, tune=native.default_tune())
    # the eps2 estimator changes the adjoint only: the image is the same bits
    est = gpu_render(sc, cams, params(eps1=1e-3, background=(1, 1, 1), eps2=0.01), tune=native.default_tune(traversal=3))
    for k in ("rgb", "alpha", "depth"):
        np.testing.assert_array_equal(est[k], ref[k], err_msg="eps2 " + k)
    prm1 = params(eps1=1e-3, background=(1, 1, 1), sort_key=1)
    ref1 = gpu_render(sc, cams, prm1, tune=native.default_tune())
    for kw in (dict(traversal=0), dict(traversal=1), dict(traversal=3), dict(kbuf=8, leaf_size=1),
               dict(persistent=0, tile_w=4)):
        out = gpu_render(sc, cams, prm1, tune=native.default_tune(**kw))
        for k in ("rgb", "alpha", "depth"):
            np.testing.assert_array_equal(out[k], ref1[k], err_msg="sort_key 1 " + str(kw))
    for kw in (dict(kbuf=8), dict(kbuf=32), dict(leaf_size=1), dict(leaf_size=8), dict(leaf_size=16),
               dict(tile_w=4), dict(tile_w=16), dict(tile_w=32), dict(persistent=0), dict(morton_bits=10),
               dict(morton_bits=20), dict(traversal=0), dict(traversal=0, leaf_size=1, kbuf=8),
               dict(traversal=2), dict(traversal=2, leaf_size=1, kbuf=8), dict(traversal=2, persistent=0),
               dict(smem_nodes=0), dict(smem_nodes=512), dict(smem_nodes=1, traversal=2),
               dict(smem_nodes=3, traversal=0), dict(traversal=3), dict(traversal=3, leaf_size=1, kbuf=8),
               dict(traversal=3, leaf_size=16, kbuf=16), dict(traversal=3, persistent=0),
               dict(block_warps=1), dict(block_warps=2), dict(hit_list=0), dict(hit_list=1),
               dict(hit_list=4096, traversal=1)):
        out = gpu_render(sc, cams, prm, tune=native.default_tune(**kw))
        for k in ("rgb", "alpha", "depth"):
            np.testing.assert_array_equal(out[k], ref[k], err_msg=str(kw))


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------
def _single(mean, scale, op=0.7, col=(0.2, 0.5, 0.9), quat=(1, 0, 0, 0)):
    return scenes.Scene(np.array([mean], np.float32), np.array([quat], np.float32),
                        np.array([scale], np.float32), np.array([op], np.float32), np.array([col], np.float32))


def test_single_gaussian_alpha_equals_opacity_at_centre():
    sc = _single((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))
    cam = scenes.look_at_camera((0, 0, -4), (0, 0, 0), 9, 9, 30)  # odd size: the centre pixel hits the mean
    prm = params(background=(0.3, 0.6, 0.1))
    g = gpu_render(sc, cam, prm)
    c = 4 * 9 + 4
    op = np.float32(0.7)
    assert abs(g["alpha"][c] - op) < 1e-6
    np.testing.assert_allclose(g["rgb"][c], op * sc.rgb[0] + (1 - op) * np.array([0.3, 0.6, 0.1]), atol=1e-6)


def test_misses_give_background_and_inside_camera_misses():
    sc = _single((0.0, 0.0, 10.0), (0.2, 0.2, 0.2))     # behind the camera below
    cam = scenes.look_at_camera((0, 0, 0), (0, 0, -1), 16, 8, 60)
    prm = params(background=(0.25, 0.5, 0.75))
    g = gpu_render(sc, cam, prm)
    np.testing.assert_array_equal(g["alpha"], 0.0)
    np.testing.assert_allclose(g["rgb"], np.tile([0.25, 0.5, 0.75], (128, 1)), atol=0)
    # camera inside the ellipsoid: t1 < 0 -> miss (Sec. 3)
    sc = _single((0.0, 0.0, 0.05), (1.0, 1.0, 1.0))
    g = gpu_render(sc, scenes.look_at_camera((0, 0, 0), (0, 0, 1), 8, 8, 60), prm)
    np.testing.assert_array_equal(g["alpha"], 0.0)


def test_single_gaussian_scene_in_every_traversal_mode():
    sc = _single((0.0, 0.0, 0.0), (0.5, 0.5, 0.5))
    cam = scenes.look_at_camera((0, 0, -4), (0, 0, 0), 9, 9, 30)
    from paper_2501_19196_gb300 import native
    ref = gpu_render(sc, cam, params(), tune=native.default_tune(traversal=0))
    for tr in (1, 2, 3):
        out = gpu_render(sc, cam, params(), tune=native.default_tune(traversal=tr))
        for k in ("rgb", "alpha", "depth"):
            np.testing.assert_array_equal(out[k], ref[k])


def test_invalid_render_arguments_are_rejected():
    from paper_2501_19196_gb300 import Renderer, native
    sc = scenes.random_tiny_scene(1, n=10)
    r = Renderer(Q_box=9.0)
    r.build(*to_dev(sc))
    cam = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 8, 8, 50)
    with pytest.raises(native.RaySplatsError):
        r.render(cam, params(Q=11.0))        # Q above the accel's Q_box
    with pytest.raises(native.RaySplatsError):
        r.render(cam, params(Q=4.0, k_max=0))
    r.render(cam, params(Q=4.0))
    r.check_device()
    r.close()


# ------------------------------------------------------------------------------------------
# rays that start among many overlapping boxes (best-first queue overflow)
# ------------------------------------------------------------------------------------------
def dense_overlap_case(seed=11, n=3000):
    """A camera inside a cloud of large, faint Gaussians: every ray starts inside most of the
    tree's boxes, so the best-first queue (128 entries) overflows with nodes whose entry lies at
    the pass's start, and a ray needs hundreds of hits (many passes of K)."""
    rng = np.random.default_rng(seed)
    sc = scenes.Scene(rng.uniform(-1, 1, (n, 3)).astype(np.float32), rng.standard_normal((n, 4)).astype(np.float32),
                      np.exp(rng.normal(np.log(0.35), 0.2, (n, 3))).astype(np.float32),
                      rng.uniform(0.01, 0.05, n).astype(np.float32), rng.uniform(0, 1, (n, 3)).astype(np.float32))
    cams = scenes.look_at_camera((0.05, 0.02, -0.1), (0.0, 0.0, 1.0), 24, 16, 70.0)
    return sc, cams


def test_rays_starting_inside_many_overlapping_boxes():
    from paper_2501_19196_gb300 import native
    sc, cams = dense_overlap_case()
    prm = params(eps1=1e-4)
    cam, px, py = scenes.pixel_grid(cams)
    ora = oracle_pixels(sc, cams, cam, px, py, prm)
    assert np.median(ora["n_hits"]) > 200  # several passes of K = 32 per ray
    # Large Gaussians (scale about 0.35) next to the camera: the FP32 error of a hit's t grows
    # with the Gaussian's size (1.3e-6 at the 99.9th percentile here, 6e-6 at grazing incidence,
    # against spacings of about 1e-2 between the ~200 hits of a ray), so 1.3 % of these rays (5
    # of 384) hold a pair of hits whose order FP32 cannot decide and whose swap changes the
    # colour by more than 1e-4 (the oracle's per-hit TIE band).
    for tune in (dict(), dict(traversal=1), dict(kbuf=8)):
        g = gpu_render(sc, cams, prm, tune=native.default_tune(**tune))  # raises on a loop-guard error
        compare_image(g, ora, pixel_index(cams, cam, px, py), max_masked=0.016, label=f"dense overlap {tune}")


# ------------------------------------------------------------------------------------------
# ordering below an FP32 ulp (the hit keys' residual)
# ------------------------------------------------------------------------------------------
def test_hits_closer_than_an_ulp_are_ordered_by_their_accurate_entry():
    """Pairs of small spheres on one pixel ray each, 0.3 to 0.45 ulp of t apart in depth: their
    FP32 entries often round to the same float, so only the keys' sub-ulp residual orders them.
    The farther sphere of each pair comes first in the caller's order and both share a Morton
    code (a distant third sphere sets the bounds), so an id tie-break would composite it first.
    The spacing exceeds the oracle's TIE band, so every pixel has one correct value."""
    cam = scenes.look_at_camera((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 7, 7, 40.0)
    cidx, px, py = scenes.pixel_grid(cam)
    o, d = oracle.raygen_f32(cam, cidx, px, py)
    rng = np.random.default_rng(8)
    s = 0.004
    means, rgb = [], []
    for r in range(len(px)):
        t0 = 4.0 + rng.uniform(-0.05, 0.05)
        ulp = np.spacing(np.float32(t0 - np.sqrt(Q) * s))
        sep = rng.uniform(0.3, 0.45) * float(ulp)
        near = o[r].astype(np.float64) + t0 * d[r].astype(np.float64)
        far = o[r].astype(np.float64) + (t0 + sep) * d[r].astype(np.float64)
        means += [far, near]           # the farther one first in the caller's order
        rgb += [(1.0, 0.0, 0.0), (0.0, 0.0, 1.0)]
    means.append((50.0, 50.0, 50.0))   # far away: sets the Morton bounds, hit by no ray
    rgb.append((0.5, 0.5, 0.5))
    n = len(means)
    sc = scenes.Scene(np.asarray(means, np.float32), np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                      np.full((n, 3), s, np.float32), np.full(n, 0.8, np.float32), np.asarray(rgb, np.float32))
    prm = params()
    g = gpu_render(sc, cam, prm)
    ora = oracle_pixels(sc, cam, cidx, px, py, prm)
    assert np.all(ora["n_hits"] == 2)
    assert np.all(ora["mask"] == 0), "the oracle flags a pair: the spacing is inside its TIE band"
    # the nearer (blue) sphere first: blue 0.8, red 0.2 * 0.8
    np.testing.assert_allclose(ora["rgb"][:, 2], 0.8, atol=1e-6)
    compare_image(g, ora, pixel_index(cam, cidx, px, py), max_masked=0.0, label="sub-ulp ordering")
