"""Pins for the FP64 oracle against facts fixed by the paper and by mathematics, not by itself.

Each test names the passage of RaySplats (arXiv 2501.19196) whose statement it checks.
References used here are independent of the oracle's code: scipy's quaternion rotation and
chi-square quantile, a long-double quadratic solve of the ellipsoid equation built from the
covariance matrix (Eq. 2), golden-section maximisation of the Gaussian along the ray (Eq. 8),
closed forms for isotropic and flattened Gaussians, explicit products of (1 - alpha), and
FP64 central finite differences.
"""
import math

import numpy as np
import pytest

import oracle
from workloads import scenes

spR = pytest.importorskip("scipy.spatial.transform").Rotation
chi2 = pytest.importorskip("scipy.stats").chi2

Q99 = scenes.default_Q()


def _sigma_inv(q, s, dtype=np.longdouble):
    """Sigma^-1 for Sigma = R S S^T R^T (Eq. 2), R from scipy (scalar-last convention)."""
    R = spR.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    Sig = R @ np.diag(np.asarray(s, np.float64) ** 2) @ R.T
    return np.linalg.inv(Sig).astype(dtype)


def _mahal2_along(o, d, m, A, t):
    x = o + t * d - m
    return x @ A @ x


def _golden_min(f, lo, hi, iters=300):
    g = (math.sqrt(5.0) - 1.0) / 2.0
    a, b = np.longdouble(lo), np.longdouble(hi)
    c, d = b - g * (b - a), a + g * (b - a)
    fc, fd = f(c), f(d)
    for _ in range(iters):
        if fc < fd:
            b, d, fd = d, c, fc
            c = b - g * (b - a)
            fc = f(c)
        else:
            a, c, fc = c, d, fd
            d = a + g * (b - a)
            fd = f(d)
    return min(fc, fd)


def _random_pair(rng):
    m = rng.uniform(-1, 1, 3)
    q = rng.standard_normal(4) * rng.uniform(0.3, 3.0)
    s = np.exp(rng.normal(-1.5, 0.6, 3))
    o = rng.uniform(-1, 1, 3) + np.array([0.0, 0.0, -5.0])
    target = m + rng.normal(0, 2.0 * s.max(), 3)
    d = target - o
    d /= np.linalg.norm(d)
    return o, d, m, q, s


# ----------------------------------------------------------------------------------------
# App. A.6 quaternion -> rotation, against scipy
# ----------------------------------------------------------------------------------------
def test_quaternion_rotation_matches_scipy():
    rng = np.random.default_rng(3)
    for _ in range(200):
        q = rng.standard_normal(4) * rng.uniform(0.1, 10.0)  # unnormalised (App. A.6, s = 2/|q|^2)
        R = oracle.quat_to_rot(q)
        ref = spR.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        np.testing.assert_allclose(R, ref, atol=1e-13)


def test_chi2_quantile_matches_scipy():
    # Sec. 3 "Intersection": Q = F^-1_{chi^2(3)}(alpha)
    for p in (0.5, 0.9, 0.95, 0.99, 0.999):
        assert abs(oracle.chi2_3_quantile(p) - chi2.ppf(p, 3)) < 1e-10
    assert abs(oracle.chi2_3_quantile(0.99) - Q99) < 1e-10


# ----------------------------------------------------------------------------------------
# Prop. 1: ray / confidence ellipsoid entry
# ----------------------------------------------------------------------------------------
def test_prop1_matches_long_double_quadratic():
    rng = np.random.default_rng(1)
    checked = 0
    for _ in range(3000):
        o, d, m, q, s = _random_pair(rng)
        A = _sigma_inv(q, s)
        ol, dl, ml = (np.asarray(x, np.longdouble) for x in (o, d, m))
        a = dl @ A @ dl
        b = dl @ A @ (ol - ml)
        c = (ol - ml) @ A @ (ol - ml) - np.longdouble(Q99)
        disc = b * b - a * c
        D2, t1, hit, _ = oracle.ray_gaussian(o, d, m, q, s, Q99)
        if disc < 0:
            assert not hit and D2 > Q99
            continue
        # well conditioned only: discriminant not tiny relative to b^2
        if disc < 1e-6 * b * b:
            continue
        r1 = (-b - np.sqrt(disc)) / a
        assert D2 <= Q99
        assert abs(t1 - float(r1)) <= 1e-9 * max(1.0, abs(float(r1)))
        assert hit == (float(r1) >= 0.0)
        checked += 1
    assert checked > 500


def test_prop1_isotropic_central_ray_closed_form():
    # Sigma = sigma^2 I, ray through the centre: t1 = |o - m| - sqrt(Q) sigma exactly.
    for sigma in (0.01, 0.1, 0.7):
        for dist in (2.0, 5.0, 30.0):
            o = np.array([0.3, -0.2, 0.1])
            m = o + dist * np.array([0.6, 0.0, 0.8])
            d = (m - o) / dist
            D2, t1, hit, _ = oracle.ray_gaussian(o, d, m, [1, 0, 0, 0], [sigma] * 3, Q99)
            expect = dist - math.sqrt(Q99) * sigma
            assert abs(D2) < 1e-20
            assert abs(t1 - expect) < 1e-12 * dist
            assert hit == (expect >= 0.0)   # camera inside the ellipsoid -> miss


def test_prop1_tangent_and_miss():
    # perpendicular distance rho*sigma from an isotropic Gaussian: D^2 = rho^2, hit iff rho^2 <= Q
    sigma = 0.2
    m = np.zeros(3)
    d = np.array([0.0, 0.0, 1.0])
    for rho in (0.0, 1.0, 2.5, math.sqrt(Q99) * (1 - 1e-9), math.sqrt(Q99) * (1 + 1e-6), 4.0):
        o = np.array([rho * sigma, 0.0, -3.0])
        D2, t1, hit, _ = oracle.ray_gaussian(o, d, m, [0.2, 0.1, -0.4, 0.7], [sigma] * 3, Q99)
        assert abs(D2 - rho * rho) < 1e-12
        assert hit == (rho * rho <= Q99)
        if hit:
            # chord half-length sigma*sqrt(Q - rho^2) before the closest approach at t = 3
            assert abs(t1 - (3.0 - sigma * math.sqrt(Q99 - rho * rho))) < 1e-9


def test_prop1_nearer_root_negative_is_a_miss():
    # Sec. 3: camera inside the ellipsoid (t1 < 0) -> the ray misses the Gaussian
    D2, t1, hit, _ = oracle.ray_gaussian([0.0, 0.0, 0.05], [0, 0, 1.0], [0, 0, 0], [1, 0, 0, 0],
                                         [0.1, 0.1, 0.1], Q99)
    assert D2 <= Q99 and t1 < 0 and not hit
    # Gaussian behind the camera
    D2, t1, hit, _ = oracle.ray_gaussian([0.0, 0.0, 2.0], [0, 0, 1.0], [0, 0, 0], [1, 0, 0, 0],
                                         [0.1, 0.1, 0.1], Q99)
    assert t1 < 0 and not hit


# ----------------------------------------------------------------------------------------
# Prop. 2: maximum response along the ray
# ----------------------------------------------------------------------------------------
def test_prop2_matches_golden_section_maximum():
    rng = np.random.default_rng(2)
    checked = 0
    for _ in range(400):
        o, d, m, q, s = _random_pair(rng)
        D2, t1, hit, _ = oracle.ray_gaussian(o, d, m, q, s, Q99)
        if not hit:
            continue
        A = _sigma_inv(q, s)
        ol, dl, ml = (np.asarray(x, np.longdouble) for x in (o, d, m))
        # for a hit, the unconstrained minimiser t_m lies at t >= t1 >= 0 (chord midpoint),
        # so the paper's max over t >= 0 equals the line maximum
        best = _golden_min(lambda t: _mahal2_along(ol, dl, ml, A, t), 0.0, 50.0)
        assert abs(math.exp(-0.5 * D2) - math.exp(-0.5 * float(best))) < 1e-12
        checked += 1
    assert checked > 50


def test_single_isotropic_gaussian_through_centre_alpha_equals_opacity():
    sc = scenes.Scene(np.array([[0.1, -0.2, 0.3]], np.float32), np.array([[1, 0, 0, 0]], np.float32),
                      np.array([[0.25, 0.25, 0.25]], np.float32), np.array([0.7], np.float32),
                      np.array([[0.2, 0.5, 0.9]], np.float32))
    o = np.array([[0.1, -0.2, -4.0]])
    d = np.array([[0.0, 0.0, 1.0]])
    bg = (0.3, 0.6, 0.1)
    out = oracle.render_rays(sc, o, d, Q99, eps1=1e-4, background=bg)
    op = float(np.float32(0.7))
    c = sc.rgb[0].astype(np.float64)
    np.testing.assert_allclose(out["alpha"], [op], atol=1e-15)
    np.testing.assert_allclose(out["rgb"][0], op * c + (1 - op) * np.array(bg), atol=1e-15)
    assert out["n_hits"][0] == 1
    t1 = (4.0 + float(np.float32(0.3))) - math.sqrt(Q99) * float(np.float32(0.25))
    assert abs(out["depth"][0] - op * t1) < 1e-12


def test_off_centre_alpha_closed_form():
    sigma, op = 0.3, 0.8
    for rho in (0.0, 0.5, 1.7, 3.0, 3.5):
        sc = scenes.Scene(np.zeros((1, 3), np.float32), np.array([[0.3, 0.4, -0.5, 0.2]], np.float32),
                          np.full((1, 3), sigma, np.float32), np.array([op], np.float32),
                          np.ones((1, 3), np.float32))
        s32 = float(np.float32(sigma))
        o = np.array([[rho * s32, 0.0, -5.0]])
        out = oracle.render_rays(sc, o, np.array([[0.0, 0.0, 1.0]]), Q99)
        expect = float(np.float32(op)) * math.exp(-rho * rho / 2) if rho * rho <= Q99 else 0.0
        assert abs(out["alpha"][0] - expect) < 1e-13


# ----------------------------------------------------------------------------------------
# Eq. 3 compositing, the eps1 cut and K_max (Sec. 3, Alg. 1 prose)
# ----------------------------------------------------------------------------------------
def _line_scene(ops, cols, z0=0.0, dz=0.5, sigma=0.05):
    n = len(ops)
    means = np.zeros((n, 3), np.float32)
    means[:, 2] = z0 + dz * np.arange(n)
    perm = np.random.default_rng(7).permutation(n)  # storage order != depth order
    inv = np.argsort(perm)
    return scenes.Scene(means[perm], np.tile(np.array([[1, 0, 0, 0]], np.float32), (n, 1)),
                        np.full((n, 3), sigma, np.float32), np.asarray(ops, np.float32)[perm],
                        np.asarray(cols, np.float32)[perm]), perm, inv


def test_two_and_three_gaussian_closed_forms():
    ops = [0.6, 0.3, 0.9]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1]]
    for n in (2, 3):
        sc, perm, inv = _line_scene(ops[:n], cols[:n])
        out = oracle.render_rays(sc, [[0.0, 0.0, -3.0]], [[0.0, 0.0, 1.0]], Q99, eps1=0.0)
        a = [float(np.float32(x)) for x in ops[:n]]
        C = np.zeros(3)
        T = 1.0
        for i in range(n):
            C += T * a[i] * np.asarray(cols[i], np.float64)
            T *= 1 - a[i]
        np.testing.assert_allclose(out["rgb"][0], C, atol=1e-14)
        assert abs(out["alpha"][0] - (1 - T)) < 1e-14
        assert out["n_hits"][0] == n


def test_transmittance_is_product_of_one_minus_alpha():
    rng = np.random.default_rng(5)
    sc = scenes.random_tiny_scene(11, n=40)
    o, d = oracle.raygen_f64(scenes.look_at_camera((0.2, 0.1, -3.0), (0, 0, 0), 16, 16, 50.0), 0,
                             *np.meshgrid(np.arange(16), np.arange(16)))
    o, d = o.reshape(-1, 3), d.reshape(-1, 3)
    out = oracle.render_rays(sc, o, d, Q99, eps1=0.0)
    # independent product: alpha_i from the Prop. 2 maximum computed here with Sigma^-1
    for r in rng.choice(len(o), 24, replace=False):
        prod = 1.0
        for i in range(sc.n):
            A = _sigma_inv(sc.quats[i], sc.scales[i], np.float64)
            x0 = o[r] - sc.means[i].astype(np.float64)
            a, b, c = d[r] @ A @ d[r], d[r] @ A @ x0, x0 @ A @ x0
            disc = b * b - a * (c - Q99)
            if disc < 0 or (-b - math.sqrt(disc)) / a < 0:
                continue
            prod *= 1 - float(sc.opacities[i]) * math.exp(-0.5 * (c - b * b / a))
        assert abs(out["T"][r] - prod) < 1e-12
        assert abs(out["alpha"][r] - (1 - prod)) < 1e-12


def test_eps1_includes_the_crossing_hit_and_kmax_truncates():
    ops = [0.5, 0.5, 0.5, 0.5, 0.5]
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1]]
    sc, _, _ = _line_scene(ops, cols)
    o, d = [[0.0, 0.0, -3.0]], [[0.0, 0.0, 1.0]]
    # T after hits: 0.5, 0.25, 0.125 ... eps1 = 0.2 -> stop after the 3rd hit (T = 0.125)
    out = oracle.render_rays(sc, o, d, Q99, eps1=0.2)
    assert out["n_hits"][0] == 3 and abs(out["T"][0] - 0.125) < 1e-15
    np.testing.assert_allclose(out["rgb"][0], [0.5, 0.25, 0.125], atol=1e-15)
    # K_max = 1: the nearest hit only
    out = oracle.render_rays(sc, o, d, Q99, eps1=0.0, k_max=1)
    assert out["n_hits"][0] == 1
    np.testing.assert_allclose(out["rgb"][0], [0.5, 0, 0], atol=1e-15)
    # eps1 = 0 and unbounded K_max: full compositing
    out = oracle.render_rays(sc, o, d, Q99, eps1=0.0)
    assert out["n_hits"][0] == 5 and abs(out["T"][0] - 0.5 ** 5) < 1e-15


# ----------------------------------------------------------------------------------------
# Invariances
# ----------------------------------------------------------------------------------------
def _tiny_rays(n=12, seed=0):
    cams = scenes.look_at_camera((0.3, 0.4, -3.0), (0, 0, 0), n, n, 55.0)
    gx, gy = np.meshgrid(np.arange(n), np.arange(n))
    o, d = oracle.raygen_f64(cams, 0, gx.ravel(), gy.ravel())
    return o, d


def test_rigid_motion_invariance():
    sc = scenes.random_tiny_scene(21, n=48)
    o, d = _tiny_rays()
    base = oracle.render_rays(sc, o, d, Q99)
    rng = np.random.default_rng(9)
    Rg = spR.from_quat(rng.standard_normal(4))
    tg = rng.uniform(-2, 2, 3)
    M = Rg.as_matrix()
    q_xyzw = (Rg * spR.from_quat(sc.quats[:, [1, 2, 3, 0]].astype(np.float64))).as_quat()
    moved = {"means": sc.means.astype(np.float64) @ M.T + tg,
             "quats": q_xyzw[:, [3, 0, 1, 2]], "scales": sc.scales, "opacities": sc.opacities,
             "rgb": sc.rgb}
    out = oracle.render_rays(None, o @ M.T + tg, d @ M.T, Q99, params64=moved)
    ok = (base["mask"] == 0) & (out["mask"] == 0)
    assert ok.mean() > 0.95
    np.testing.assert_allclose(out["rgb"][ok], base["rgb"][ok], atol=1e-12)
    np.testing.assert_allclose(out["alpha"][ok], base["alpha"][ok], atol=1e-12)
    np.testing.assert_allclose(out["depth"][ok], base["depth"][ok], atol=1e-11)


def test_permutation_invariance_and_direction_scale():
    sc = scenes.random_tiny_scene(22, n=48)
    o, d = _tiny_rays()
    base = oracle.render_rays(sc, o, d, Q99)
    perm = np.random.default_rng(1).permutation(sc.n)
    out = oracle.render_rays(sc.subset(perm), o, d, Q99)
    ok = base["mask"] == 0
    np.testing.assert_allclose(out["rgb"][ok], base["rgb"][ok], atol=1e-13)
    # alpha (and so the colour) does not depend on the length of d; t1 scales as 1/|d|
    out2 = oracle.render_rays(sc, o, 2.5 * d, Q99)
    np.testing.assert_allclose(out2["rgb"][ok], base["rgb"][ok], atol=1e-13)
    np.testing.assert_allclose(out2["depth"][ok] * 2.5, base["depth"][ok], atol=1e-12)


# ----------------------------------------------------------------------------------------
# Flattened (near-2D) Gaussians reach their limit continuously
# ----------------------------------------------------------------------------------------
def test_flattened_limit_is_continuous():
    rng = np.random.default_rng(4)
    for _ in range(20):
        q = rng.standard_normal(4)
        R = spR.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
        sx, sy = rng.uniform(0.2, 0.5, 2)
        m = rng.uniform(-0.2, 0.2, 3)
        # a ray crossing the Gaussian's plane (local z = 0) at in-plane point (x0, y0)
        x0, y0 = rng.uniform(-0.5, 0.5) * sx, rng.uniform(-0.5, 0.5) * sy
        p_cross = m + R @ np.array([x0, y0, 0.0])
        dl = np.array([rng.uniform(-0.5, 0.5), rng.uniform(-0.5, 0.5), 1.0])
        d = R @ (dl / np.linalg.norm(dl))
        o = p_cross - 4.0 * d
        lim = (x0 / sx) ** 2 + (y0 / sy) ** 2  # in-plane Mahalanobis distance at the crossing
        prev = None
        for k in range(1, 8):
            eps = 10.0 ** (-k)
            D2, t1, hit, _ = oracle.ray_gaussian(o, d, m, q, [sx, sy, eps], Q99)
            assert hit
            assert D2 <= lim + 1e-12                       # approaches from below ...
            if prev is not None:
                assert D2 >= prev - 1e-12                  # ... monotonically
            assert lim - D2 <= 50.0 * eps * eps / min(sx, sy) ** 2 + 1e-12  # O(eps^2)
            prev = D2
        # the workloads' flattening (one axis x 0.01)
        D2, _, _, _ = oracle.ray_gaussian(o, d, m, q, [sx, sy, 0.01 * sx], Q99)
        assert abs(lim - D2) <= 50.0 * (0.01 * sx) ** 2 / min(sx, sy) ** 2


# ----------------------------------------------------------------------------------------
# App. A.4 / A.5: the recurrences equal the division-free back-to-front form
# ----------------------------------------------------------------------------------------
def test_alpha_gradient_recurrences_App_A4_A5():
    rng = np.random.default_rng(8)
    for trial in range(10):
        n = int(rng.integers(2, 9))
        a = rng.uniform(0.05, 0.95, n)
        c = rng.uniform(0, 1, n)
        sc, perm, inv = _line_scene(a, np.stack([c, np.zeros(n), np.zeros(n)], 1))
        a = sc.opacities[inv].astype(np.float64)   # the float32 values actually stored
        c = sc.rgb[inv, 0].astype(np.float64)
        out = oracle.render_rays(sc, [[0.0, 0.0, -3.0]], [[0.0, 0.0, 1.0]], Q99, eps1=0.0,
                                 dl_rgb=[[1.0, 0.0, 0.0]], dl_alpha=[0.0])
        # central ray through isotropic Gaussians: D2 = 0, so dI/dopacity = dI/dalpha
        g = out["grads"]["opacities"][inv]
        T = np.concatenate([[1.0], np.cumprod(1 - a)[:-1]])
        I = float(np.sum(c * a * T))
        # App. A.5, first display: the direct O(N^2) formula
        direct = np.zeros(n)
        for i in range(n):
            s = c[i] * T[i]
            for j in range(i + 1, n):
                s -= c[j] * a[j] * np.prod([1 - a[k] for k in range(j) if k != i])
            direct[i] = s
        # App. A.4 and the App. A.5 recurrence
        rec = np.zeros(n)
        rec[0] = (c[0] - I) / (1 - a[0])
        for i in range(1, n):
            rec[i] = (rec[i - 1] * (1 - a[i - 1]) + (c[i] - c[i - 1]) * T[i]) / (1 - a[i])
        np.testing.assert_allclose(g, direct, atol=1e-13)
        np.testing.assert_allclose(g, rec, atol=1e-11)


# ----------------------------------------------------------------------------------------
# App. A.3-A.6: the oracle's analytic gradient against FP64 central differences
# ----------------------------------------------------------------------------------------
@pytest.mark.parametrize("seed,flat", [(31, 0.0), (32, 0.0), (33, 0.5)])
def test_gradient_matches_central_differences(seed, flat):
    sc = scenes.random_tiny_scene(seed, n=10, spread=0.4, log_mu=-1.5, flat_frac=flat)
    o, d = _tiny_rays(8, seed)
    rng = np.random.default_rng(seed)
    R = o.shape[0]
    gc = rng.standard_normal((R, 3))
    ga = rng.standard_normal(R)
    kw = dict(Q=Q99, eps1=1e-3, background=(0.2, 0.4, 0.6))
    base = oracle.render_rays(sc, o, d, dl_rgb=gc, dl_alpha=ga, **kw)
    ok = base["mask"] == 0
    gc[~ok] = 0.0
    ga[~ok] = 0.0
    base = oracle.render_rays(sc, o, d, dl_rgb=gc, dl_alpha=ga, **kw)
    P = {k: getattr(sc, k).astype(np.float64).copy() for k in ("means", "quats", "scales", "opacities", "rgb")}

    def loss(params):
        out = oracle.render_rays(None, o, d, params64=params, **kw)
        return float(np.sum(out["rgb"] * gc) + np.sum(out["alpha"] * ga))

    for key in P:
        fd = np.zeros_like(P[key])
        flat_view = P[key].reshape(-1)
        for j in range(flat_view.size):
            x = flat_view[j]
            h = 1e-6 * max(1.0, abs(x))
            flat_view[j] = x + h
            lp = loss(P)
            flat_view[j] = x - h
            lm = loss(P)
            flat_view[j] = x
            fd.reshape(-1)[j] = (lp - lm) / (2 * h)
        an = base["grads"][key]
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-300)
        assert err < 1e-6, (key, err)


@pytest.mark.parametrize("sort_key", [0, 1])
@pytest.mark.parametrize("seed,flat", [(41, 0.0), (42, 0.5)])
def test_depth_gradient_matches_central_differences(seed, flat, sort_key):
    """Depth = sum w_i t_key_i: its gradient (colour-like through alpha, plus dt_key/dparams)
    against FP64 central differences, for both sort keys, together with rgb and alpha terms."""
    sc = scenes.random_tiny_scene(seed, n=10, spread=0.4, log_mu=-1.5, flat_frac=flat)
    o, d = _tiny_rays(8, seed)
    rng = np.random.default_rng(seed)
    R = o.shape[0]
    gc = rng.standard_normal((R, 3))
    ga = rng.standard_normal(R)
    gd = rng.standard_normal(R)
    kw = dict(Q=Q99, eps1=1e-3, background=(0.2, 0.4, 0.6), sort_key=sort_key)
    base = oracle.render_rays(sc, o, d, **kw)
    ok = base["mask"] == 0
    gc[~ok], ga[~ok], gd[~ok] = 0.0, 0.0, 0.0
    base = oracle.render_rays(sc, o, d, dl_rgb=gc, dl_alpha=ga, dl_depth=gd, **kw)
    P = {k: getattr(sc, k).astype(np.float64).copy() for k in ("means", "quats", "scales", "opacities", "rgb")}

    def loss(params):
        out = oracle.render_rays(None, o, d, params64=params, **kw)
        return float(np.sum(out["rgb"] * gc) + np.sum(out["alpha"] * ga) + np.sum(out["depth"] * gd))

    for key in P:
        fd = np.zeros_like(P[key])
        flat_view = P[key].reshape(-1)
        for j in range(flat_view.size):
            x = flat_view[j]
            h = 1e-6 * max(1.0, abs(x))
            flat_view[j] = x + h
            lp = loss(P)
            flat_view[j] = x - h
            lm = loss(P)
            flat_view[j] = x
            fd.reshape(-1)[j] = (lp - lm) / (2 * h)
        an = base["grads"][key]
        err = np.linalg.norm(an - fd) / max(np.linalg.norm(fd), 1e-300)
        assert err < 1e-6, (key, err)


def test_sort_key_tm_closed_forms():
    """Isotropic Gaussians (Eq. 8, Prop. 1): t_m is the parameter of the closest approach to
    the mean, <m - o, d>, and t1 = t_m - s sqrt(Q - rho^2/s^2); the depth follows the key."""
    sigma, op = 0.3, 0.8
    for rho in (0.0, 0.5, 1.7):
        s32 = float(np.float32(sigma))
        sc = scenes.Scene(np.array([[0.0, 0.0, 0.25]], np.float32), np.array([[0.3, 0.4, -0.5, 0.2]], np.float32),
                          np.full((1, 3), sigma, np.float32), np.array([op], np.float32),
                          np.ones((1, 3), np.float32))
        o = np.array([[rho * s32, 0.0, -5.0]])
        d = np.array([[0.0, 0.0, 1.0]])
        a = float(np.float32(op)) * math.exp(-rho * rho / 2)
        tm = 5.25
        t1 = tm - s32 * math.sqrt(Q99 - rho * rho)
        out0 = oracle.render_rays(sc, o, d, Q99, sort_key=0)
        out1 = oracle.render_rays(sc, o, d, Q99, sort_key=1)
        assert abs(out0["depth"][0] - a * t1) < 1e-12
        assert abs(out1["depth"][0] - a * tm) < 1e-12
        np.testing.assert_allclose(out0["rgb"], out1["rgb"], atol=0)


def test_sort_key_changes_the_compositing_order():
    """A large Gaussian whose entry comes first but whose centre lies behind a small one:
    ordered by t1 it is composited first, by t_m second (Eq. 3 with the two orders)."""
    means = np.array([[0.0, 0.0, 1.0], [0.0, 0.0, 0.6]], np.float32)   # big (behind), small
    scales = np.array([[0.4, 0.4, 0.4], [0.02, 0.02, 0.02]], np.float32)
    ops = np.array([0.5, 0.7], np.float32)
    cols = np.array([[1, 0, 0], [0, 0, 1]], np.float32)
    sc = scenes.Scene(means, np.tile(np.array([[1, 0, 0, 0]], np.float32), (2, 1)), scales, ops, cols)
    o, d = np.array([[0.0, 0.0, -3.0]]), np.array([[0.0, 0.0, 1.0]])
    a = [float(x) for x in ops]
    big_first = a[0] * cols[0] + (1 - a[0]) * a[1] * cols[1]
    small_first = a[1] * cols[1] + (1 - a[1]) * a[0] * cols[0]
    np.testing.assert_allclose(oracle.render_rays(sc, o, d, Q99, sort_key=0)["rgb"][0], big_first, atol=1e-14)
    np.testing.assert_allclose(oracle.render_rays(sc, o, d, Q99, sort_key=1)["rgb"][0], small_first, atol=1e-14)


def test_eps2_estimator_closed_forms():
    """Sec. 3's second threshold: after the eps1 cut at hit 1, hits behind are collected until
    the product of their (1 - alpha) drops below eps2; dL/dalpha_1 then sees their colour
    instead of the background.  Three Gaussians on the ray through their centres (alpha =
    opacity): with eps2 = 0.01, hit 2 (alpha 0.5) is collected and so is hit 3; with alpha_2 =
    0.995 the product falls below eps2 at hit 2 and hit 3 is not seen."""
    bg = np.array([0.1, 0.2, 0.3])
    c = np.array([[1.0, 0.0, 0.0], [0.0, 1.0, 0.0], [0.0, 0.0, 1.0]])
    for a2, collect3 in ((0.5, True), (0.995, False)):
        ops = [0.99995, a2, 0.7]
        sc, perm, inv = _line_scene(ops, c)
        o, d = [[0.0, 0.0, -3.0]], [[0.0, 0.0, 1.0]]
        a = [float(np.float32(x)) for x in ops]
        kw = dict(Q=Q99, eps1=1e-4, background=tuple(bg))
        gc = np.array([[1.0, 1.0, 1.0]])
        exact = oracle.render_rays(sc, o, d, dl_rgb=gc, **kw)
        est = oracle.render_rays(sc, o, d, dl_rgb=gc, eps2=0.01, **kw)
        np.testing.assert_array_equal(exact["rgb"], est["rgb"])   # the image is unchanged
        assert exact["n_hits"][0] == 1
        S = a[1] * c[1] + (1 - a[1]) * (a[2] * c[2] + (1 - a[2]) * bg) if collect3 else a[1] * c[1] + (1 - a[1]) * bg
        g1 = inv[0]  # storage index of the first Gaussian along the ray
        np.testing.assert_allclose(exact["grads"]["opacities"][g1], np.sum(c[0] - bg), atol=1e-12)
        np.testing.assert_allclose(est["grads"]["opacities"][g1], np.sum(c[0] - S), atol=1e-12)
        # the collected Gaussians are not composited: they receive no gradient
        np.testing.assert_array_equal(est["grads"]["opacities"][inv[1]], 0.0)
        np.testing.assert_array_equal(est["grads"]["rgb"][inv[2]], 0.0)


# ----------------------------------------------------------------------------------------
# Acceleration-structure references (plain definitions)
# ----------------------------------------------------------------------------------------
def test_morton_brute_force_interleave():
    rng = np.random.default_rng(6)
    means = rng.uniform(-3, 5, (300, 3)).astype(np.float32)
    means[5] = means[7]  # duplicates
    for bits in (10, 21):
        codes, lohi = oracle.morton(means, bits)
        lo, hi = means.min(0), means.max(0)
        ext = hi - lo
        u = (means - lo) / ext            # numpy float32: one rounded sub, one rounded div
        cell = np.clip(np.floor(u * np.float32(2 ** bits)), 0, 2 ** bits - 1).astype(np.int64)
        for i in range(0, 300, 7):
            ref = 0
            for b in range(bits - 1, -1, -1):
                for k in range(3):
                    ref = (ref << 1) | int((cell[i, k] >> b) & 1)
            assert int(codes[i]) == ref
        np.testing.assert_array_equal(lohi, np.concatenate([lo, hi]))


def test_extended_morton_size_class():
    rng = np.random.default_rng(16)
    means = rng.uniform(-3, 5, (400, 3)).astype(np.float32)
    scales = np.exp(rng.normal(-4, 1.5, (400, 3))).astype(np.float32)
    codes, _ = oracle.morton(means, 20, scales)
    lo, hi = means.min(0), means.max(0)
    ext = hi - lo
    cell = np.clip(np.floor((means - lo) / ext * np.float32(2 ** 20)), 0, 2 ** 20 - 1).astype(np.int64)
    _, e_ext = np.frexp(np.float32(ext.max()))
    for i in range(0, 400, 3):
        _, e_s = np.frexp(np.float32(scales[i].max()))           # frexp exponent = E - 126
        cls = int(np.clip(e_s - e_ext + 11, 0, 7))
        ref = 0
        for b in range(19, 15, -1):
            for k in range(3):
                ref = (ref << 1) | int((cell[i, k] >> b) & 1)
        ref = (ref << 3) | cls
        for b in range(15, -1, -1):
            for k in range(3):
                ref = (ref << 1) | int((cell[i, k] >> b) & 1)
        assert int(codes[i]) == ref
    assert int(codes.max()) < 2 ** 63


def test_sort_is_stable_by_code_then_index():
    rng = np.random.default_rng(7)
    codes = rng.integers(0, 50, 1000).astype(np.uint64)
    perm, sc = oracle.sort_perm(codes)
    np.testing.assert_array_equal(perm, np.lexsort((np.arange(1000), codes)))
    np.testing.assert_array_equal(sc, codes[perm])


def _tree_brute(keys, f, l, out, node):
    if f == l:
        return
    x = [keys[f], keys[l]]
    bit = (x[0] ^ x[1]).bit_length() - 1
    s = max(i for i in range(f, l + 1) if not (keys[i] >> bit) & 1)
    out[node] = (f, l, s)
    _tree_brute(keys, f, s, out, s)
    _tree_brute(keys, s + 1, l, out, s + 1)


@pytest.mark.parametrize("n,vals", [(2, 4), (9, 3), (64, 1000), (257, 40)])
def test_radix_tree_matches_recursive_definition(n, vals):
    rng = np.random.default_rng(n)
    codes = np.sort(rng.integers(0, vals, n).astype(np.uint64))
    f, l, s = oracle.radix_tree(codes)
    keys = [(int(c) << 32) | i for i, c in enumerate(codes)]
    ref = {}
    _tree_brute(keys, 0, n - 1, ref, 0)
    assert len(ref) == n - 1
    for node, (ff, ll, ss) in ref.items():
        assert (f[node], l[node], s[node]) == (ff, ll, ss)
    # every leaf appears exactly once as a child
    leaves = []
    for node in range(n - 1):
        if s[node] == f[node]:
            leaves.append(f[node])
        if s[node] + 1 == l[node]:
            leaves.append(l[node])
    assert sorted(leaves) == list(range(n))


def test_default_workload_ambiguity_fraction_small():
    wl = scenes.workload(1)
    cam, px, py = scenes.pixel_grid(wl.cams)
    out = oracle.render(wl.scene, wl.cams, cam, px, py, wl.Q, wl.eps1, wl.k_max, wl.background)
    assert (out["mask"] != 0).mean() < 0.01
    assert out["n_hits"].max() > 3
