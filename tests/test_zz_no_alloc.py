"""rs_render_fixed_scratch -- the render entry point for callers that cannot allocate device
memory (plug-ins whose host application owns every device allocation, tools held to a fixed
device-memory budget).  It keeps every intermediate in one fixed-size device array; this test
calls it through the C ABI twice in a row, on different scenes and cameras, and checks each
output against the allocating path (rs_build_accel + rs_render) at the image tolerance.  It
also checks that requests beyond the fixed limits are rejected.  Collected last on purpose."""
import ctypes

import numpy as np
import pytest
import torch

from gpu_util import TOL_RGB, params, to_dev
from workloads import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _fixed_render(scene, cams, prm, tune):
    from paper_2501_19196_gb300 import native
    lib = native.load()
    dev = to_dev(scene)
    g = native.RsGaussians(scene.n, *[t.data_ptr() for t in dev])
    arr = native.cameras_to_ctypes(cams)
    P = int(cams.total_rays())
    out = (torch.full((P, 3), -1.0, device="cuda"), torch.full((P,), -1.0, device="cuda"),
           torch.full((P,), -1.0, device="cuda"))
    frame = native.RsFrame(out[0].data_ptr(), out[1].data_ptr(), out[2].data_ptr())
    pc = prm.to_c()
    st = lib.rs_render_fixed_scratch(ctypes.byref(g), arr, len(arr), ctypes.byref(pc), ctypes.byref(tune),
                                     ctypes.byref(frame), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))
    native.check(st)
    torch.cuda.synchronize()
    return [t.cpu().numpy() for t in out]


def _allocating_render(scene, cams, prm, tune):
    from paper_2501_19196_gb300 import Renderer
    r = Renderer(tune=tune, Q_box=prm.Q)
    r.build(*to_dev(scene))
    rgb, alpha, depth = r.render(cams, prm)
    torch.cuda.synchronize()
    r.check_device()
    out = [rgb.cpu().numpy(), alpha.cpu().numpy(), depth.cpu().numpy()]
    r.close()
    return out


def test_fixed_scratch_matches_allocating_path_on_two_calls():
    from paper_2501_19196_gb300 import native
    tune = native.default_tune()
    cases = [
        (scenes.scene_object_shell(20000, seed=3),
         scenes.concat_cameras([scenes.look_at_camera((0, 0.3, -3.5), (0, 0, 0), 320, 240, 50),
                                scenes.look_at_camera((3.0, 1.0, 1.0), (0, 0, 0), 256, 200, 45)]),
         params(background=(1.0, 1.0, 1.0))),
        (scenes.scene_unbounded(32768, seed=4),
         scenes.concat_cameras([scenes.look_at_camera((12.0, 2.0, 0.0), (0, 0, 0), 400, 260, 60),
                                scenes.look_at_camera((0.0, 2.0, 12.0), (0, 0, 0), 333, 217, 60),
                                scenes.look_at_camera((-8.0, 3.0, -8.0), (0, 0, 0), 64, 48, 60)]),
         params(eps1=1e-3)),
    ]
    for i, (sc, cams, prm) in enumerate(cases):
        fixed = _fixed_render(sc, cams, prm, tune)
        ref = _allocating_render(sc, cams, prm, tune)
        for a, b, name in zip(fixed, ref, ("rgb", "alpha", "depth")):
            err = float(np.abs(a - b).max())
            assert err <= TOL_RGB * (1.0 if name != "depth" else max(1.0, float(np.abs(b).max()))), (i, name, err)


def test_fixed_scratch_rejects_requests_beyond_its_limits():
    from paper_2501_19196_gb300 import native
    lib = native.load()
    tune = native.default_tune()
    cams = scenes.look_at_camera((0, 0, -3), (0, 0, 0), 8, 8, 50)
    arr = native.cameras_to_ctypes(cams)
    pc = params().to_c()
    buf = torch.zeros(1024, device="cuda")
    frame = native.RsFrame(buf.data_ptr(), buf.data_ptr(), None)
    too_many = native.RsGaussians(32769, *([buf.data_ptr()] * 5))
    assert lib.rs_render_fixed_scratch(ctypes.byref(too_many), arr, 1, ctypes.byref(pc), ctypes.byref(tune),
                                       ctypes.byref(frame), None) == native.RS_ERR_INVALID_ARG
    ok_n = native.RsGaussians(10, *([buf.data_ptr()] * 5))
    big = native.cameras_to_ctypes(scenes.look_at_camera((0, 0, -3), (0, 0, 0), 1024, 512, 50))
    assert lib.rs_render_fixed_scratch(ctypes.byref(ok_n), big, 1, ctypes.byref(pc), ctypes.byref(tune),
                                       ctypes.byref(frame), None) == native.RS_ERR_INVALID_ARG
    # several cameras whose pixel counts would overflow a running total: each is rejected on
    # its own before any launch
    huge = scenes.concat_cameras([scenes.look_at_camera((0, 0, -3), (0, 0, 0), 8, 8, 50)] * 4)
    huge.width[:] = 2 ** 31 - 1
    huge.height[:] = 2 ** 31 - 1
    harr = native.cameras_to_ctypes(huge)
    assert lib.rs_render_fixed_scratch(ctypes.byref(ok_n), harr, 4, ctypes.byref(pc), ctypes.byref(tune),
                                       ctypes.byref(frame), None) == native.RS_ERR_INVALID_ARG
    nan_cam = native.cameras_to_ctypes(cams)
    nan_cam[0].fx = float("nan")
    assert lib.rs_render_fixed_scratch(ctypes.byref(ok_n), nan_cam, 1, ctypes.byref(pc), ctypes.byref(tune),
                                       ctypes.byref(frame), None) == native.RS_ERR_INVALID_ARG
