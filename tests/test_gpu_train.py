"""GPU parity of the training-step pieces against the FP64 oracle (oracle/train.py): the
L2 + D-SSIM loss and its image gradient (Sec. 3, App. A.7), Adam and the sigmoid activations
(Sec. 5); and a short optimisation that must lower the loss."""
import numpy as np
import pytest
import torch

from oracle import train as otrain
from gpu_util import to_dev
from workloads import scenes

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _cuda():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _images(seed, sizes):
    rng = np.random.default_rng(seed)
    P = sum(w * h for w, h in sizes)
    # smooth-ish images so that SSIM is far from its trivial values
    rgb = rng.uniform(0, 1, (P, 3)).astype(np.float32)
    tgt = np.clip(rgb + rng.normal(0, 0.15, (P, 3)), 0, 1).astype(np.float32)
    return rgb, tgt


@pytest.mark.parametrize("lam", [0.0, 0.2, 1.0])
def test_loss_and_gradient_match_oracle(lam):
    from paper_2501_19196_gb300 import ImageLoss
    sizes = [(37, 23), (16, 40), (5, 3), (64, 33)]
    cams = scenes.concat_cameras([scenes.look_at_camera((0, 0, -3), (0, 0, 0), w, h, 50) for w, h in sizes])
    rgb, tgt = _images(int(lam * 10) + 1, sizes)
    ref_loss, ref_grad = otrain.batch_loss_and_grad(rgb, tgt, sizes, lam)
    fn = ImageLoss(lam)
    loss, grad = fn(torch.from_numpy(rgb).cuda(), torch.from_numpy(tgt).cuda(), cams)
    loss = float(loss.item())
    grad = grad.cpu().numpy().astype(np.float64)
    fn.close()
    assert abs(loss - ref_loss) <= 1e-5 * max(1.0, abs(ref_loss)), (loss, ref_loss)
    err = np.abs(grad - ref_grad).max() / np.abs(ref_grad).max()
    print(f"[parity] loss lambda {lam}: loss {loss:.8f} vs {ref_loss:.8f}, grad max rel err {err:.2e}")
    assert err < 1e-4


def test_loss_is_deterministic():
    from paper_2501_19196_gb300 import ImageLoss
    sizes = [(200, 120), (64, 64)]
    cams = scenes.concat_cameras([scenes.look_at_camera((0, 0, -3), (0, 0, 0), w, h, 50) for w, h in sizes])
    rgb, tgt = (torch.from_numpy(a).cuda() for a in _images(9, sizes))
    fn = ImageLoss(0.2)
    a = [t.clone() for t in fn(rgb, tgt, cams)]
    b = [t.clone() for t in fn(rgb, tgt, cams)]
    fn.close()
    assert torch.equal(a[0], b[0]) and torch.equal(a[1], b[1])


def test_adam_and_sigmoid_match_oracle():
    from paper_2501_19196_gb300 import adam_step, sigmoid, sigmoid_backward
    rng = np.random.default_rng(3)
    n = 1000003  # not a multiple of the block size
    p0 = rng.standard_normal(n).astype(np.float32)
    p, m, v = torch.from_numpy(p0).cuda(), torch.zeros(n, device="cuda"), torch.zeros(n, device="cuda")
    q, mq, vq = p0.astype(np.float64), np.zeros(n), np.zeros(n)
    for step in range(1, 4):
        g = rng.standard_normal(n).astype(np.float32)
        adam_step(p, torch.from_numpy(g).cuda(), m, v, step, 1e-2)
        q, mq, vq = otrain.adam_step(q, g.astype(np.float64), mq, vq, step, 1e-2)
    np.testing.assert_allclose(p.cpu().numpy(), q, rtol=0, atol=2e-6)
    x = torch.linspace(-20, 20, 4001, device="cuda")
    y = sigmoid(x)
    np.testing.assert_allclose(y.cpu().numpy(), otrain.sigmoid(x.cpu().numpy()), rtol=2e-6, atol=1e-7)
    dy = torch.rand_like(x)
    np.testing.assert_allclose(sigmoid_backward(y, dy).cpu().numpy(),
                               otrain.sigmoid_backward(y.cpu().numpy(), dy.cpu().numpy()), rtol=1e-5, atol=1e-8)


def test_training_steps_lower_the_loss():
    """Fit a perturbed copy of a scene to the images of the original: the loss must fall."""
    from paper_2501_19196_gb300 import RenderParams, Renderer, TrainStep, native
    sc = scenes.random_tiny_scene(5, n=300, spread=1.0, log_mu=-2.3)
    cams = scenes.concat_cameras([scenes.look_at_camera((0.4, 0.3, -3.2), (0, 0, 0), 48, 40, 55.0),
                                  scenes.look_at_camera((-3.0, 0.5, 0.7), (0.1, 0, 0), 40, 40, 45.0)])
    prm = RenderParams(background=(0.2, 0.2, 0.2))
    r = Renderer(tune=native.default_tune())
    r.build(*to_dev(sc))
    target = r.render(cams, prm)[0].clone()
    r.close()
    means, quats, scales, ops, rgb = to_dev(sc)
    gen = torch.Generator(device="cpu").manual_seed(0)
    rgb0 = (rgb + 0.3 * torch.randn(rgb.shape, generator=gen).cuda()).clamp(0, 1)
    logit = lambda x: torch.log(x / (1 - x))  # noqa: E731
    ts = TrainStep(means.clone(), quats.clone(), logit(scales.clamp(1e-4, 0.999)), logit(ops.clamp(1e-4, 0.9999)),
                   rgb0, lr=dict(rgb=2e-2), params=prm)
    ts.renderer.set_cameras(cams)
    losses = [float(ts.step(target).item()) for _ in range(25)]
    ts.close()
    print("[train] loss", [f"{x:.5f}" for x in losses[::6]])
    assert losses[-1] < 0.5 * losses[0]
