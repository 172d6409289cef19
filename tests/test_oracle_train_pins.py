"""Pins for the training-step oracle (oracle/train.py): the loss of Sec. 3 / App. A.7, Adam and
the sigmoid activations of Sec. 5, against facts fixed by mathematics and by independent
library routines (scipy's correlation and expit, torch's Adam), not by the oracle itself."""
import numpy as np
import pytest

from oracle import train

ndimage = pytest.importorskip("scipy.ndimage")
special = pytest.importorskip("scipy.special")


def _img(seed, H=9, W=7):
    rng = np.random.default_rng(seed)
    return rng.uniform(0, 1, (H, W, 3)), rng.uniform(0, 1, (H, W, 3))


def test_window_is_normalised_and_separable_gaussian():
    w = train.gaussian_window(5, 1.5)
    assert w.shape == (11, 11)
    assert abs(w.sum() - 1.0) < 1e-15
    g = np.exp(-np.arange(-5, 6) ** 2 / (2 * 1.5 ** 2))
    np.testing.assert_allclose(w, np.outer(g, g) / g.sum() ** 2, rtol=1e-14)


@pytest.mark.parametrize("r", [2, 5])
def test_window_sums_match_scipy_correlation_with_zero_padding(r):
    I, _ = _img(1, 13, 10)
    w = train.gaussian_window(r, 1.5)
    ref = ndimage.correlate(I[..., 0], w, mode="constant", cval=0.0)
    np.testing.assert_allclose(train.window_sum(I[..., 0], w), ref, atol=1e-14)


def test_ssim_of_an_image_with_itself_is_one_and_stationary():
    I, _ = _img(2)
    w = train.gaussian_window()
    for ch in range(3):
        assert abs(train.ssim(I[..., ch], I[..., ch], w) - 1.0) < 1e-14
    assert train.image_loss(I, I, 0.2) < 1e-15
    np.testing.assert_allclose(train.image_loss_grad(I, I, 0.2), 0.0, atol=1e-14)


def test_pure_l2_gradient_closed_form():
    I, J = _img(3)
    H, W, _ = I.shape
    np.testing.assert_allclose(train.image_loss_grad(I, J, 0.0), 2.0 * (I - J) / (H * W) / 3.0, atol=1e-15)


@pytest.mark.parametrize("lam,r", [(0.2, 5), (1.0, 2), (0.5, 5)])
def test_loss_gradient_matches_central_differences(lam, r):
    """App. A.7's E/F/G form against FP64 central differences of the plain loss definition."""
    I, J = _img(4 + r)
    w = train.gaussian_window(r, 1.5)
    an = train.image_loss_grad(I, J, lam, w)
    fd = np.zeros_like(I)
    for idx in np.ndindex(I.shape):
        x = I[idx]
        h = 1e-6
        I[idx] = x + h
        lp = train.image_loss(I, J, lam, w)
        I[idx] = x - h
        lm = train.image_loss(I, J, lam, w)
        I[idx] = x
        fd[idx] = (lp - lm) / (2 * h)
    assert np.abs(an - fd).max() < 1e-9 * max(1.0, np.abs(fd).max())


def test_batch_loss_is_the_mean_of_image_losses():
    (I1, J1), (I2, J2) = _img(5, 6, 4), _img(6, 5, 8)
    rgb = np.concatenate([I1.reshape(-1, 3), I2.reshape(-1, 3)])
    tgt = np.concatenate([J1.reshape(-1, 3), J2.reshape(-1, 3)])
    loss, grad = train.batch_loss_and_grad(rgb, tgt, [(4, 6), (8, 5)], 0.2)
    assert abs(loss - (train.image_loss(I1, J1, 0.2) + train.image_loss(I2, J2, 0.2)) / 2) < 1e-15
    np.testing.assert_allclose(grad[:24], train.image_loss_grad(I1, J1, 0.2).reshape(-1, 3) / 2, atol=1e-16)


def test_adam_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(7)
    p0 = rng.standard_normal(17)
    p = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([p], lr=1e-2, betas=(0.9, 0.999), eps=1e-8)
    q, m, v = p0.copy(), np.zeros(17), np.zeros(17)
    for step in range(1, 6):
        g = rng.standard_normal(17)
        p.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
        q, m, v = train.adam_step(q, g, m, v, step, 1e-2)
    np.testing.assert_allclose(q, p.detach().numpy(), rtol=1e-13, atol=1e-15)


def test_sigmoid_and_its_adjoint():
    x = np.linspace(-20, 20, 81)
    y = train.sigmoid(x)
    np.testing.assert_allclose(y, special.expit(x), rtol=1e-15)
    h = 1e-6
    fd = (train.sigmoid(x + h) - train.sigmoid(x - h)) / (2 * h)
    np.testing.assert_allclose(train.sigmoid_backward(y, np.ones_like(y)), fd, atol=1e-9)
