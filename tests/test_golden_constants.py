"""The constants the paper prints (tests/golden/paper_constants.txt) against the oracle's and
the library's: SSIM stabilisers (App. A.7), Adam hyperparameters (Sec. 5) and the definition of
Q as a chi^2(3) quantile (Sec. 3).  Each is checked through behaviour where a closed form
exists: the SSIM of two constant images and the first bias-corrected Adam step."""
import inspect
import os

import numpy as np
import pytest

from oracle import train

HERE = os.path.dirname(os.path.abspath(__file__))


def _golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "paper_constants.txt")) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                k, v = line.split()
                vals[k] = float(v)
    return vals


G = _golden()


def test_ssim_of_constant_images_closed_form():
    """For constant images a and b the windowed variances and covariance vanish away from the
    border, so SSIM = (2ab + c1) / (a^2 + b^2 + c1) with c1 = (k1 L)^2."""
    c1 = (G["ssim_k1"] * G["ssim_L"]) ** 2
    c2 = (G["ssim_k2"] * G["ssim_L"]) ** 2
    assert train.C1 == pytest.approx(c1, rel=1e-15) and train.C2 == pytest.approx(c2, rel=1e-15)
    w = train.gaussian_window()
    a, b = 0.3, 0.05
    I, J = np.full((15, 15), a), np.full((15, 15), b)
    _, _, A, B, C, D = train.ssim_terms(I, J, w)
    centre = (A * B / (C * D))[7, 7]
    assert centre == pytest.approx((2 * a * b + c1) / (a * a + b * b + c1), rel=1e-12)


def test_adam_defaults_and_first_step():
    """Step 1 from zero moments moves every parameter by lr g / (|g| + eps)."""
    for fn in (train.adam_step,):
        sig = inspect.signature(fn).parameters
        assert sig["beta1"].default == G["adam_beta1"]
        assert sig["beta2"].default == G["adam_beta2"]
        assert sig["eps"].default == G["adam_eps"]
    g = np.array([0.5, -2e-3, 1e-9, 0.0])
    p0 = np.array([1.0, 2.0, 3.0, 4.0])
    p1, m, v = train.adam_step(p0, g, np.zeros(4), np.zeros(4), 1, 0.01)
    np.testing.assert_allclose(p1, p0 - 0.01 * g / (np.abs(g) + G["adam_eps"]), rtol=1e-14, atol=1e-18)


def test_product_adam_defaults_match_the_paper():
    """The device Adam's Python entry point carries the same defaults (host logic, no GPU)."""
    from paper_2501_19196_gb300 import train as product_train
    sig = inspect.signature(product_train.adam_step).parameters
    assert (sig["beta1"].default, sig["beta2"].default, sig["eps"].default) == \
        (G["adam_beta1"], G["adam_beta2"], G["adam_eps"])


def test_workload_Q_is_the_chi2_quantile():
    stats = pytest.importorskip("scipy.stats")
    from workloads import scenes
    q = stats.chi2.ppf(G["q_level"], int(G["q_chi2_dof"]))
    assert scenes.default_Q() == pytest.approx(q, rel=1e-12)
