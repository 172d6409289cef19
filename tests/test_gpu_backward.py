"""GPU parity of the adjoint (reverse replay, gradient scatter by bulk reductions or float4
atomics, finalize) against the oracle's FP64 gradient, through the C ABI and through the
torch.autograd.Function.  Tolerance: 1e-3
relative L2 per gradient array.  Rays where FP32 and FP64 may take a different discrete
decision (any oracle decision flag) get a zero upstream gradient on both sides."""
import numpy as np
import pytest
import torch

import oracle
from gpu_util import TOL_GRAD, gpu_render, oracle_pixels, params, pixel_index, rel_l2, to_dev
from workloads import scenes

pytestmark = pytest.mark.gpu

KEYS = ("means", "quats", "scales", "opacities", "rgb")


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _grad_case(sc, cams, prm, tune=None, stride=1, seed=1, with_alpha=True, with_depth=False):
    from paper_2501_19196_gb300 import native
    cam, px, py = scenes.pixel_grid(cams, stride=stride)
    idx = pixel_index(cams, cam, px, py)
    P = int(cams.n_pixels().sum())
    rng = np.random.default_rng(seed)
    gc_s = rng.standard_normal((len(cam), 3))
    ga_s = rng.standard_normal(len(cam)) if with_alpha else np.zeros(len(cam))
    gd_s = rng.standard_normal(len(cam)) if with_depth else np.zeros(len(cam))
    ora0 = oracle_pixels(sc, cams, cam, px, py, prm)
    bad = (ora0["mask"] & oracle.AMB_DECISION) != 0
    gc_s[bad] = 0.0
    ga_s[bad] = 0.0
    gd_s[bad] = 0.0
    ora = oracle_pixels(sc, cams, cam, px, py, prm, dl_rgb=gc_s, dl_alpha=ga_s,
                        dl_depth=gd_s if with_depth else None)
    # full-frame upstream gradient: zero except at the listed pixels
    gc = np.zeros((P, 3), np.float32)
    ga = np.zeros(P, np.float32)
    gd = np.zeros(P, np.float32)
    gc[idx] = gc_s
    ga[idx] = ga_s
    gd[idx] = gd_s
    out, r, dev = gpu_render(sc, cams, prm, tune=tune or native.default_tune(), keep=True)
    grads = r.backward(torch.from_numpy(gc).cuda(), torch.from_numpy(ga).cuda(),
                       d_depth=torch.from_numpy(gd).cuda() if with_depth else None)
    torch.cuda.synchronize()
    r.check_device()
    r.close()
    errs = {k: rel_l2(grads[k].cpu().numpy().astype(np.float64).reshape(ora["grads"][k].shape), ora["grads"][k])
            for k in KEYS}
    return errs, bad.mean()


@pytest.mark.parametrize("seed", range(5))
def test_gradients_tiny_scenes(seed):
    sc = scenes.random_tiny_scene(300 + seed, n=40, flat_frac=0.3 if seed % 2 else 0.0)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 21, 17, 55.0),
                                  scenes.look_at_camera((-3.0, 0.5, 0.7), (0.1, 0, 0), 16, 16, 45.0)])
    for kw in (dict(), dict(eps1=0.2), dict(k_max=2), dict(background=(0.3, 0.2, 1.0))):
        errs, bad = _grad_case(sc, cams, params(**kw), seed=seed)
        assert max(errs.values()) < TOL_GRAD, (kw, errs)


@pytest.mark.parametrize("seed", range(12))
def test_random_scenes_cameras_and_tunables(seed):
    """Random scene sizes, flat fractions, camera placements and frame sizes, one render setting
    per seed, each under four adjoint configurations (hit lists, re-traversal, lists of two,
    4-wide nodes): gradients within 1e-3 relative L2 of the oracle's."""
    from paper_2501_19196_gb300 import native
    rng = np.random.default_rng(1000 + seed)
    sc = scenes.random_tiny_scene(2000 + seed, n=int(rng.integers(20, 250)), flat_frac=float(rng.uniform(0, 0.5)))
    cams = scenes.concat_cameras(
        [scenes.look_at_camera(tuple(rng.uniform(-3.5, 3.5, 3)), tgt, int(rng.integers(8, 40)), int(rng.integers(8, 40)),
                               float(rng.uniform(30, 70))) for tgt in ((0, 0, 0), (0.1, 0, 0))])
    kw = [dict(), dict(eps1=0.05), dict(k_max=3), dict(background=(0.3, 0.2, 1.0)), dict(sort_key=1)][seed % 5]
    for tune in (dict(), dict(hit_list=0), dict(hit_list=2), dict(traversal=3)):
        errs, bad = _grad_case(sc, cams, params(**kw), tune=native.default_tune(**tune), seed=seed)
        assert max(errs.values()) < TOL_GRAD, (kw, tune, errs)


def test_every_ray_scatters_into_the_same_gaussians():
    """3,072 rays all cross one large Gaussian (and most cross the three small ones in front
    of it): every lane of every warp adds into the same few 64 B accumulators at once, through
    the list replay's bulk reductions (hit lists) and the re-traversal's float4 atomics."""
    from paper_2501_19196_gb300 import native
    means = np.array([(0.0, 0.0, 0.0), (0.15, 0.1, -0.9), (-0.2, -0.1, -0.7), (0.05, -0.15, -1.1)], np.float32)
    scales = np.array([(0.9, 0.8, 0.7), (0.3, 0.25, 0.2), (0.35, 0.3, 0.25), (0.2, 0.3, 0.25)], np.float32)
    rng = np.random.default_rng(5)
    q = rng.standard_normal((4, 4)).astype(np.float32)
    sc = scenes.Scene(means, q, scales, np.array([0.6, 0.4, 0.5, 0.3], np.float32),
                      rng.uniform(0, 1, (4, 3)).astype(np.float32))
    cams = scenes.look_at_camera((0.0, 0.0, -4.0), (0, 0, 0), 64, 48, 30.0)
    for tune in (dict(), dict(hit_list=0)):
        errs, bad = _grad_case(sc, cams, params(), tune=native.default_tune(**tune), seed=11)
        print(f"[parity] shared Gaussians {tune}: {({k: f'{v:.2e}' for k, v in errs.items()})} flagged {bad:.4f}")
        assert bad < 0.05
        assert max(errs.values()) < TOL_GRAD, (tune, errs)


@pytest.mark.parametrize("sort_key", [0, 1])
@pytest.mark.parametrize("seed", range(4))
def test_depth_gradients_tiny_scenes(seed, sort_key):
    """Exact gradient of sum_i w_i t_i (with rgb and alpha terms) for both sort keys, through
    the hit-list replay and through every re-traversing adjoint."""
    from paper_2501_19196_gb300 import native
    sc = scenes.random_tiny_scene(320 + seed, n=40, flat_frac=0.3 if seed % 2 else 0.0)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 21, 17, 55.0),
                                  scenes.look_at_camera((-3.0, 0.5, 0.7), (0.1, 0, 0), 16, 16, 45.0)])
    for kw, tune in ((dict(), dict()), (dict(eps1=0.2), dict(hit_list=0)), (dict(k_max=3), dict(hit_list=0, traversal=0)),
                     (dict(background=(0.3, 0.2, 1.0)), dict(hit_list=0, traversal=1))):
        errs, bad = _grad_case(sc, cams, params(sort_key=sort_key, **kw), tune=native.default_tune(**tune), seed=seed,
                               with_depth=True)
        assert max(errs.values()) < TOL_GRAD, (kw, tune, errs)


@pytest.mark.parametrize("seed", range(4))
def test_eps2_estimator_gradients(seed):
    """The paper's eps2 estimator (Sec. 3): rays cut by eps1 (0.05 / 0.2 here, so that many
    are) give their last composited hit dL/dalpha from the phase-2 hits behind it; through the
    hit-list replay and through every re-traversing adjoint, with and without depth."""
    from paper_2501_19196_gb300 import native
    sc = scenes.random_tiny_scene(340 + seed, n=60, flat_frac=0.3 if seed % 2 else 0.0)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 21, 17, 55.0),
                                  scenes.look_at_camera((-3.0, 0.5, 0.7), (0.1, 0, 0), 16, 16, 45.0)])
    for kw, tune, depth in ((dict(eps1=0.05, eps2=0.01), dict(), False),
                            (dict(eps1=0.2, eps2=0.05, background=(0.3, 0.2, 1.0)), dict(hit_list=0), True),
                            (dict(eps1=0.2, eps2=0.001), dict(hit_list=0, traversal=0), False),
                            (dict(eps1=0.05, eps2=0.01, sort_key=1), dict(hit_list=2, traversal=1), True)):
        errs, bad = _grad_case(sc, cams, params(**kw), tune=native.default_tune(**tune), seed=seed, with_depth=depth)
        assert max(errs.values()) < TOL_GRAD, (kw, tune, errs)


def test_gradients_workload_1k_full_frame():
    wl = scenes.workload(1)
    errs, bad = _grad_case(wl.scene, wl.cams, params(eps1=wl.eps1, background=wl.background))
    print("1k/64x64 gradient rel-L2:", {k: f"{v:.2e}" for k, v in errs.items()}, f"decision-flagged {bad:.4f}")
    assert max(errs.values()) < TOL_GRAD, errs


def test_gradients_shell_200k_sampled_pixels():
    wl = scenes.workload(2)
    errs, bad = _grad_case(wl.scene, wl.cams, params(eps1=wl.eps1, background=wl.background), stride=23)
    print("200k sampled gradient rel-L2:", {k: f"{v:.2e}" for k, v in errs.items()}, f"flagged {bad:.4f}")
    assert max(errs.values()) < TOL_GRAD, errs


def test_gradients_invariant_to_tunables():
    from paper_2501_19196_gb300 import native
    sc = scenes.random_tiny_scene(77, n=300, spread=1.0, log_mu=-2.5)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 40, 24, 55.0),
                                  scenes.look_at_camera((2.0, 2.0, -2.0), (0, 0, 0), 16, 40, 50.0)])
    prm = params(eps1=1e-3)
    # the re-traversing adjoint of every traversal order and setting (hit_list = 0) ...
    retrace = [dict(kbuf=8), dict(kbuf=32), dict(leaf_size=1), dict(persistent=0), dict(tile_w=16),
               dict(traversal=0), dict(traversal=0, kbuf=8, leaf_size=1), dict(traversal=1),
               dict(traversal=2, kbuf=8, leaf_size=1), dict(smem_nodes=0), dict(smem_nodes=512, traversal=2),
               dict(traversal=3), dict(traversal=3, kbuf=8, leaf_size=1), dict(block_warps=1), dict(block_warps=3)]
    # ... and hit lists: the default, tiny (most rays re-traverse), mixed, and the largest
    listed = [dict(), dict(hit_list=1), dict(hit_list=3), dict(hit_list=3, traversal=0),
              dict(hit_list=2, traversal=1), dict(hit_list=4, traversal=3), dict(hit_list=4096, persistent=0)]
    for kw in [dict(kw, hit_list=0) for kw in retrace] + listed:
        errs, _ = _grad_case(sc, cams, prm, tune=native.default_tune(**kw))
        assert max(errs.values()) < TOL_GRAD, (kw, errs)


def test_hit_list_split_counters():
    """The adjoint replays a ray from its hit list exactly when the list holds all its hits:
    with the largest list nothing re-traverses, without a list everything does, and in between
    the listed and re-traversed hits add up to the forward's composited hits."""
    from paper_2501_19196_gb300 import Renderer, native
    sc = scenes.random_tiny_scene(78, n=400, spread=1.0, log_mu=-2.3)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 48, 32, 55.0)])
    prm = params(eps1=1e-3)
    rng = np.random.default_rng(3)
    P = int(cams.total_rays())
    d_rgb = torch.from_numpy(rng.standard_normal((P, 3)).astype(np.float32)).cuda()
    seen = {}
    for H in (0, 1, 4, 4096):
        r = Renderer(tune=native.default_tune(hit_list=H))
        r.build(*to_dev(sc))
        sf = torch.zeros(10, dtype=torch.int64, device="cuda")
        sb = torch.zeros(10, dtype=torch.int64, device="cuda")
        r.render(cams, prm, stats=sf)
        r.backward(d_rgb, stats=sb)
        torch.cuda.synchronize()
        r.check_device()
        f = dict(zip(native.STATS_FIELDS, sf.cpu().tolist()))
        b = dict(zip(native.STATS_FIELDS, sb.cpu().tolist()))
        r.close()
        assert b["hits_composited"] == f["hits_composited"] > 0
        assert b["hits_listed"] <= H * (b["rays"] - b["rays_retraced"])
        if H == 0:
            assert b["hits_listed"] == 0 and b["rays_retraced"] == b["rays"]
        if H == 4096:
            assert b["rays_retraced"] == 0 and b["hits_listed"] == f["hits_composited"] and b["nodes_visited"] == 0
        seen[H] = b
    # more list capacity never re-traverses more rays
    assert seen[0]["rays_retraced"] >= seen[1]["rays_retraced"] >= seen[4]["rays_retraced"] >= 0
    assert 0 < seen[4]["hits_listed"] < seen[4096]["hits_listed"]


def test_autograd_function_matches_direct_backward():
    from paper_2501_19196_gb300 import Renderer, render_gaussians
    sc = scenes.random_tiny_scene(9, n=80, flat_frac=0.2)
    cams = scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 24, 20, 55.0)
    prm = params(background=(0.1, 0.2, 0.3))
    leaves = [t.clone().requires_grad_(True) for t in to_dev(sc)]
    rgb, alpha, depth = render_gaussians(*leaves, cams, prm)
    rng = np.random.default_rng(0)
    w = torch.from_numpy(rng.standard_normal((rgb.shape[0], 3)).astype(np.float32)).cuda()
    wa = torch.from_numpy(rng.standard_normal(rgb.shape[0]).astype(np.float32)).cuda()
    wd = torch.from_numpy(rng.standard_normal(rgb.shape[0]).astype(np.float32)).cuda()
    loss = (rgb * w).sum() + (alpha * wa).sum() + (depth * wd).sum()
    loss.backward()
    r = Renderer()
    r.build(*to_dev(sc))
    r.render(cams, prm)
    ref = r.backward(w.contiguous(), wa.contiguous(), d_depth=wd.contiguous())
    torch.cuda.synchronize()
    # float atomics accumulate in a different order on each call: compare in relative L2
    for leaf, k in zip(leaves, KEYS):
        a = leaf.grad.cpu().numpy().astype(np.float64).reshape(-1)
        b = ref[k].cpu().numpy().astype(np.float64).reshape(-1)
        assert rel_l2(a, b) < 1e-5, (k, rel_l2(a, b))
    r.close()


def test_gradient_through_log_scale_and_logit_activations():
    """The ABI is physical; activations (exp for log-scales, sigmoid for opacity logits) are
    chained by torch autograd on top."""
    from paper_2501_19196_gb300 import render_gaussians
    sc = scenes.random_tiny_scene(11, n=50)
    cams = scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 16, 16, 55.0)
    m, q, s, o, c = to_dev(sc)
    log_s = torch.log(s).requires_grad_(True)
    logit = torch.logit(o).requires_grad_(True)
    rgb, alpha, _ = render_gaussians(m, q, torch.exp(log_s), torch.sigmoid(logit), c, cams, params())
    (rgb.sum() + alpha.sum()).backward()
    assert torch.isfinite(log_s.grad).all() and torch.isfinite(logit.grad).all()
    assert log_s.grad.abs().sum() > 0 and logit.grad.abs().sum() > 0


def test_gradients_rays_starting_inside_many_overlapping_boxes():
    """The dense-overlap case of the forward tests: the re-traversing adjoint's queue overflows
    too (hit_list 0), and hit lists shorter than the rays mix replay and re-traversal."""
    from paper_2501_19196_gb300 import native
    from test_gpu_forward import dense_overlap_case
    sc, cams = dense_overlap_case()
    for tune in (dict(), dict(hit_list=0), dict(hit_list=64)):
        errs, bad = _grad_case(sc, cams, params(eps1=1e-4), tune=native.default_tune(**tune))
        assert max(errs.values()) < TOL_GRAD, (tune, errs)


def test_ring_16_cameras_full_size_sampled():
    """The benchmark's workload at full size (1M Gaussians, 16 ring cameras of mixed resolution,
    12.04M rays) in the batched persistent launch with hit lists: sampled pixels of every camera
    against the oracle, the image and, with an upstream gradient on those pixels only, every
    gradient array."""
    wl = scenes.workload(4)
    prm = params(eps1=wl.eps1, background=wl.background)
    cam, px, py = scenes.pixel_grid(wl.cams, stride=173)
    g = gpu_render(wl.scene, wl.cams, prm)
    ora = oracle_pixels(wl.scene, wl.cams, cam, px, py, prm)
    from gpu_util import compare_image
    err, masked = compare_image(g, ora, pixel_index(wl.cams, cam, px, py), label="16 cameras sampled")
    errs, bad = _grad_case(wl.scene, wl.cams, prm, stride=173)
    print(f"16 cameras sampled: pixels {len(cam)}, image err {err:.2e}, gradient rel-L2",
          {k: f"{v:.2e}" for k, v in errs.items()}, f"flagged {bad:.4f}")
    assert max(errs.values()) < TOL_GRAD, errs
