"""Out-of-memory paths of the C ABI, driven by rs_test_fail_alloc.  Each device allocation that a
build, a forward render or a backward pass makes is failed in turn.  Every such call must
return RS_ERR_OOM and leave its handle valid but unusable: later renders and backward passes
reject it instead of reading freed buffers.  No device memory may leak, and the call that
finally succeeds must give the undisturbed result (bit-identical images, gradients equal up to
the order of the atomic additions)."""
import ctypes

import pytest
import torch

from gpu_util import params, to_dev
from workloads import scenes

pytestmark = pytest.mark.gpu

MAX_ALLOCS = 64  # more device allocations than any single call makes


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


class _Case:
    def __init__(self, n=200000, seed=5):
        from paper_2501_19196_gb300 import native
        self.native = native
        self.lib = native.load()
        sc = scenes.scene_object_shell(n, seed=seed)
        self.dev = to_dev(sc)
        self.g = native.RsGaussians(sc.n, *[t.data_ptr() for t in self.dev])
        self.g_small = native.RsGaussians(sc.n // 4, *[t.data_ptr() for t in self.dev])
        cams = scenes.concat_cameras([scenes.look_at_camera((0, 0.3, -3.5), (0, 0, 0), 96, 64, 50),
                                      scenes.look_at_camera((3.0, 1.0, 1.0), (0, 0, 0), 64, 48, 45)])
        self.cams = native.cameras_to_ctypes(cams)
        P = int(cams.total_rays())
        self.rgb, self.alpha, self.depth = (torch.zeros((P, 3), device="cuda"), torch.zeros(P, device="cuda"),
                                            torch.zeros(P, device="cuda"))
        self.frame = native.RsFrame(self.rgb.data_ptr(), self.alpha.data_ptr(), self.depth.data_ptr())
        gen = torch.Generator(device="cpu").manual_seed(seed)
        self.d_rgb = torch.randn((P, 3), generator=gen).cuda()
        self.d_alpha = torch.randn(P, generator=gen).cuda()
        self.dl = native.RsFrameGrad(self.d_rgb.data_ptr(), self.d_alpha.data_ptr())
        self.grads = [torch.zeros(s, device="cuda") for s in ((n, 3), (n, 4), (n, 3), (n,), (n, 3))]
        self.gout = native.RsGaussianGrads(*[t.data_ptr() for t in self.grads])
        self.prm = params().to_c()
        self.tune = native.default_tune()
        self.stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)

    def build(self, acc, g=None):
        return self.lib.rs_build_accel(ctypes.byref(g or self.g), ctypes.c_float(scenes.default_Q()),
                                       ctypes.byref(self.tune), ctypes.byref(acc), self.stream)

    def render(self, acc, state, g=None):
        return self.lib.rs_render(ctypes.byref(g or self.g), acc, self.cams, len(self.cams), ctypes.byref(self.prm),
                                  ctypes.byref(self.tune), ctypes.byref(self.frame), ctypes.byref(state),
                                  self.stream)

    def backward(self, acc, state):
        for t in self.grads:
            t.zero_()
        return self.lib.rs_render_backward(ctypes.byref(self.g), acc, state, ctypes.byref(self.dl),
                                           ctypes.byref(self.tune), ctypes.byref(self.gout), self.stream)

    def outputs(self):
        torch.cuda.synchronize()
        return [t.clone() for t in (self.rgb, self.alpha, self.depth)], [t.clone() for t in self.grads]

    def full_step(self):
        """An undisturbed build + render + backward on fresh handles."""
        acc, state = ctypes.c_void_p(), ctypes.c_void_p()
        self.native.check(self.build(acc))
        self.native.check(self.render(acc, state))
        self.native.check(self.backward(acc, state))
        imgs, grads = self.outputs()
        self.native.check(self.lib.rs_check_device(acc, state, self.stream))
        self.lib.rs_state_destroy(state)
        self.lib.rs_accel_destroy(acc)
        return imgs, grads

    def oom(self, st):
        assert st == self.native.RS_ERR_OOM, (st, self.lib.rs_last_error())
        assert b"injected allocation failure" in self.lib.rs_last_error()


def _same(imgs, grads, ref_imgs, ref_grads):
    for a, b in zip(imgs, ref_imgs):
        assert torch.equal(a, b)
    for a, b in zip(grads, ref_grads):
        assert float(torch.linalg.norm(a - b)) <= 1e-5 * max(float(torch.linalg.norm(b)), 1e-30)


def _free_bytes():
    torch.cuda.synchronize()
    torch.cuda.empty_cache()  # only the library's own allocations should move the figure
    return torch.cuda.mem_get_info()[0]


def test_every_allocation_failure_is_reported_and_recoverable():
    c = _Case()
    lib, native = c.lib, c.native
    ref_imgs, ref_grads = c.full_step()
    c.full_step()  # every kernel is loaded before the memory is measured
    big = native.cameras_to_ctypes(scenes.concat_cameras(
        [scenes.look_at_camera((0, 0.3, -3.5), (0, 0, 0), 200, 160, 50)] * 2))
    P_big = 2 * 200 * 160
    big_out = (torch.zeros((P_big, 3), device="cuda"), torch.zeros(P_big, device="cuda"),
               torch.zeros(P_big, device="cuda"))
    free0 = _free_bytes()

    # 1. builds on a fresh handle: fail allocation k of the call, k = 1, 2, ... until one succeeds
    fails = 0
    for k in range(1, MAX_ALLOCS + 1):
        acc = ctypes.c_void_p()
        assert lib.rs_test_fail_alloc(k) == native.RS_OK
        st = c.build(acc)
        lib.rs_test_fail_alloc(0)
        if st == native.RS_OK:
            break
        c.oom(st)
        fails += 1
        if acc:  # a handle that exists after a failed build holds no build
            state = ctypes.c_void_p()
            assert c.render(acc, state) == native.RS_ERR_INVALID_ARG
            assert not state
            assert lib.rs_accel_destroy(acc) == native.RS_OK
    else:
        pytest.fail("the build never succeeded")
    assert fails >= 10  # the handle and the per-Gaussian buffers were all exercised

    # 2. rebuilds of an existing handle for a larger scene: every reallocation failure
    assert lib.rs_accel_destroy(acc) == native.RS_OK
    acc = ctypes.c_void_p()
    native.check(c.build(acc, c.g_small))
    for k in range(1, MAX_ALLOCS + 1):
        lib.rs_test_fail_alloc(k)
        st = c.build(acc)
        lib.rs_test_fail_alloc(0)
        if st == native.RS_OK:
            break
        c.oom(st)
        state = ctypes.c_void_p()
        assert c.render(acc, state, c.g_small) == native.RS_ERR_INVALID_ARG  # the old build is gone too
        assert c.render(acc, state) == native.RS_ERR_INVALID_ARG
        assert not state
    else:
        pytest.fail("the rebuild never succeeded")

    # 3. forwards: a fresh state for each k
    for k in range(1, MAX_ALLOCS + 1):
        state = ctypes.c_void_p()
        lib.rs_test_fail_alloc(k)
        st = c.render(acc, state)
        lib.rs_test_fail_alloc(0)
        if st == native.RS_OK:
            break
        c.oom(st)
        if state:  # the state exists but holds no render
            assert c.backward(acc, state) == native.RS_ERR_INVALID_ARG
            assert lib.rs_state_destroy(state) == native.RS_OK
    else:
        pytest.fail("the forward never succeeded")

    # 4. backward (gradient scratch, overflow tile list): each allocation fails in turn, then succeeds
    for k in range(1, MAX_ALLOCS + 1):
        lib.rs_test_fail_alloc(k)
        st = c.backward(acc, state)
        lib.rs_test_fail_alloc(0)
        if st == native.RS_OK:
            break
        c.oom(st)
    else:
        pytest.fail("the backward never succeeded")
    assert k >= 3
    imgs, grads = c.outputs()
    native.check(lib.rs_check_device(acc, state, c.stream))
    _same(imgs, grads, ref_imgs, ref_grads)
    del imgs, grads

    # 5. a state whose re-render failed holds no render: backward rejects it, a retry recovers
    saved = c.cams
    c.cams = big  # more pixels than the state holds: its per-ray buffers are reallocated
    frame_saved = c.frame
    c.frame = native.RsFrame(*[t.data_ptr() for t in big_out])
    lib.rs_test_fail_alloc(2)
    c.oom(c.render(acc, state))
    lib.rs_test_fail_alloc(0)
    c.cams, c.frame = saved, frame_saved
    assert c.backward(acc, state) == native.RS_ERR_INVALID_ARG
    native.check(c.render(acc, state))
    native.check(c.backward(acc, state))
    imgs, grads = c.outputs()
    _same(imgs, grads, ref_imgs, ref_grads)
    del imgs, grads
    lib.rs_state_destroy(state)
    lib.rs_accel_destroy(acc)

    # no device memory is left behind by the failed calls
    free1 = _free_bytes()
    assert abs(free0 - free1) <= 4 << 20, (free0, free1)
