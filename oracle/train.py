"""FP64 reference of the training-step pieces around the rendering path -- TEST INFRASTRUCTURE ONLY.

Only tests/, __graft_entry__.smoke() and bench.py's cpu_baseline / reference legs may import this
module; the product path never does.  Plain numpy, FP64, written from the paper:

  - the loss of one image, per colour channel (1 - lambda) L2 + lambda (1 - SSIM) / 2, averaged
    over R, G, B ........................................ Sec. 3 "Loss Function", App. A.7
  - SSIM with a normalised Gaussian window of radius r, c1 = 0.01^2, c2 = 0.03^2, pixels
    outside the image taken as 0 ........................ App. A.7 ("Computing dL_SSIM/dI")
  - dL/dI: the L2 term 2 (1 - lambda)(I - I^)/(w h) and the SSIM term from the three window
    sums of E, F and G ................................... App. A.7
  - Adam with bias correction, beta1 0.9, beta2 0.999, eps 1e-8 .................... Sec. 5
  - sigmoid activations of the opacities and scales ................................ Sec. 5

Readings where the paper is silent: the window is 11 x 11 (r = 5) with sigma = 1.5 (the choice
of the 3DGS loss the paper says it follows); a batch of images is averaged image by image.
"""
from __future__ import annotations

import numpy as np

C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(r=5, sigma=1.5):
    """(2r+1)^2 window w[m, n] for m, n in -r..r, separable, summing to 1."""
    x = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-x * x / (2.0 * sigma * sigma))
    g /= g.sum()
    return np.outer(g, g)


def window_sum(X, w):
    """out[k, l] = sum_{m,n} w[m, n] X[k + m, l + n], X taken as 0 outside the image."""
    r = w.shape[0] // 2
    H, W = X.shape
    P = np.zeros((H + 2 * r, W + 2 * r))
    P[r:r + H, r:r + W] = X
    out = np.zeros((H, W))
    for m in range(-r, r + 1):
        for n in range(-r, r + 1):
            out += w[m + r, n + r] * P[r + m:r + m + H, r + n:r + n + W]
    return out


def ssim_terms(I, J, w):
    """The per-pixel quantities of App. A.7 for one channel: mu, sigma^2, sigma_IJ, A, B, C, D."""
    mu1, mu2 = window_sum(I, w), window_sum(J, w)
    s11 = window_sum(I * I, w) - mu1 * mu1
    s22 = window_sum(J * J, w) - mu2 * mu2
    s12 = window_sum(I * J, w) - mu1 * mu2
    A = 2.0 * mu1 * mu2 + C1
    B = 2.0 * s12 + C2
    C = mu1 * mu1 + mu2 * mu2 + C1
    D = s11 + s22 + C2
    return mu1, mu2, A, B, C, D


def ssim(I, J, w):
    _, _, A, B, C, D = ssim_terms(I, J, w)
    return float(np.mean(A * B / (C * D)))


def image_loss(img, target, lam, w=None):
    """Loss of one (H, W, 3) image against its target: mean over channels of
    (1 - lam) mean (I - I^)^2 + lam (1 - SSIM) / 2."""
    w = gaussian_window() if w is None else w
    total = 0.0
    for ch in range(3):
        I, J = img[..., ch].astype(np.float64), target[..., ch].astype(np.float64)
        total += (1.0 - lam) * np.mean((I - J) ** 2) + lam * (1.0 - ssim(I, J, w)) / 2.0
    return total / 3.0


def image_loss_grad(img, target, lam, w=None):
    """dL/dI of image_loss, by App. A.7: dSSIM/dI = ((E*w) + I^ (F*w) - I (G*w)) / (h w)."""
    w = gaussian_window() if w is None else w
    H, W, _ = img.shape
    out = np.zeros(img.shape)
    for ch in range(3):
        I, J = img[..., ch].astype(np.float64), target[..., ch].astype(np.float64)
        mu1, mu2, A, B, C, D = ssim_terms(I, J, w)
        CD2 = (C * D) ** 2
        E = 2.0 / CD2 * (C * D * mu2 * (B - A) - A * B * mu1 * (D - C))
        F = 2.0 / CD2 * A * C * D
        G = 2.0 / CD2 * A * B * C
        # (X * w)_{ij} = sum_{k,l} X_{kl} w_{i-k, j-l}; the window is symmetric
        dssim = (window_sum(E, w) + J * window_sum(F, w) - I * window_sum(G, w)) / (H * W)
        dl2 = 2.0 * (I - J) / (H * W)
        out[..., ch] = ((1.0 - lam) * dl2 - lam / 2.0 * dssim) / 3.0
    return out


def batch_loss_and_grad(rgb, target, sizes, lam, w=None):
    """Images concatenated pixel-major (rs_render layout, (P, 3)); sizes = [(W, H), ...].
    The batch loss is the mean of the image losses; returns (loss, dL/drgb (P, 3))."""
    grad = np.zeros((rgb.shape[0], 3))
    total, base = 0.0, 0
    n = len(sizes)
    for (Wd, Hd) in sizes:
        sl = slice(base, base + Wd * Hd)
        I = rgb[sl].reshape(Hd, Wd, 3).astype(np.float64)
        J = target[sl].reshape(Hd, Wd, 3).astype(np.float64)
        total += image_loss(I, J, lam, w) / n
        grad[sl] = image_loss_grad(I, J, lam, w).reshape(-1, 3) / n
        base += Wd * Hd
    return total, grad


def adam_step(p, g, m, v, step, lr, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba) with bias correction; returns new (p, m, v)."""
    m = beta1 * m + (1.0 - beta1) * g
    v = beta2 * v + (1.0 - beta2) * g * g
    mh = m / (1.0 - beta1 ** step)
    vh = v / (1.0 - beta2 ** step)
    return p - lr * mh / (np.sqrt(vh) + eps), m, v


def sigmoid(x):
    return 1.0 / (1.0 + np.exp(-np.asarray(x, np.float64)))


def sigmoid_backward(y, dy):
    y = np.asarray(y, np.float64)
    return np.asarray(dy, np.float64) * y * (1.0 - y)
