"""Pins for the oracle's ambiguity flags on constructed scenes whose decisions are known exactly.

A pixel is excluded from image parity only when FP32 could take a discrete decision differently
from FP64 and the other choice changes the pixel by more than 1e-4 (IMPACT).  Each case places
Gaussians on the centre ray of a 9x9 camera at (0, 0, -4) looking at the origin (the ray is
exactly the +z axis in FP32) so that the decision is a tie, a boundary or an eps1 crossing by
construction, or clearly not one:

* TIE: two equal spheres offset sideways by the same distance have the same entry t1 (Prop. 1)
  -> TIE, and IMPACT when their colours differ; the same spheres 0.05 apart in depth -> no TIE.
* BOUNDARY: a sphere whose Mahalanobis distance to the ray is sqrt(Q (1 - 5e-7)) is a hit by a
  hair -> BOUNDARY and IMPACT (toggling it changes the colour by about opacity * e^{-Q/2});
  at Q (1 - 1e-4) it is a clear hit -> no flag (the per-Gaussian FP32 band of a sphere is about
  1e-6 Q).
* EPS1: a central hit with opacity 1 - 1e-4 leaves T = eps1 when eps1 is set to 1 minus that
  (FP32) opacity -> EPS1; opacity 0.5 -> none.
"""
import numpy as np

import oracle
from workloads import scenes

Q = scenes.default_Q()
CAM = scenes.look_at_camera((0.0, 0.0, -4.0), (0.0, 0.0, 0.0), 9, 9, 40.0)
CENTRE = (np.array([0], np.int32), np.array([4], np.int32), np.array([4], np.int32))


def _scene(means, scales, opac, rgb):
    n = len(means)
    return scenes.Scene(np.asarray(means, np.float32), np.tile(np.array([1, 0, 0, 0], np.float32), (n, 1)),
                        np.asarray(scales, np.float32), np.asarray(opac, np.float32), np.asarray(rgb, np.float32))


def _mask(sc, eps1=1e-4):
    cam, px, py = CENTRE
    out = oracle.render(sc, CAM, cam, px, py, Q, eps1, 2 ** 31 - 1, (0.0, 0.0, 0.0))
    return int(out["mask"][0]), out


def test_centre_ray_is_the_z_axis():
    o, d = oracle.raygen_f32(CAM, *CENTRE)
    np.testing.assert_array_equal(o[0], [0.0, 0.0, -4.0])
    np.testing.assert_array_equal(d[0], [0.0, 0.0, 1.0])


def test_equal_entries_are_a_tie_with_impact_only_when_colours_differ():
    s = 0.25
    sc = _scene([(0.1, 0.0, 0.0), (-0.1, 0.0, 0.0)], [(s, s, s)] * 2, [0.5, 0.5], [(1, 0, 0), (0, 0, 1)])
    m, out = _mask(sc)
    assert out["n_hits"][0] == 2
    assert m & oracle.AMB_TIE and m & oracle.AMB_IMPACT and m & oracle.IMP_TIE
    same = _scene([(0.1, 0.0, 0.0), (-0.1, 0.0, 0.0)], [(s, s, s)] * 2, [0.5, 0.5], [(0.3, 0.6, 0.9)] * 2)
    m, _ = _mask(same)
    assert m & oracle.AMB_TIE and not m & oracle.AMB_IMPACT


def test_entries_apart_in_depth_are_no_tie():
    s = 0.25
    sc = _scene([(0.1, 0.0, 0.0), (-0.1, 0.0, 0.05)], [(s, s, s)] * 2, [0.5, 0.5], [(1, 0, 0), (0, 0, 1)])
    m, out = _mask(sc)
    assert out["n_hits"][0] == 2
    assert m == 0


def test_boundary_band_flags_a_hair_but_not_a_clear_hit():
    s = 0.25
    for frac, flagged in ((5e-7, True), (1e-4, False)):
        rho = np.float32(s * np.sqrt(Q * (1.0 - frac)))
        sc = _scene([(rho, 0.0, 0.0)], [(s, s, s)], [0.9], [(1.0, 1.0, 1.0)])
        D2 = (float(rho) / s) ** 2
        assert D2 < Q  # a hit in FP64
        m, out = _mask(sc)
        assert out["n_hits"][0] == 1
        if flagged:
            assert m & oracle.AMB_BOUNDARY and m & oracle.AMB_IMPACT and m & oracle.IMP_BOUNDARY, (frac, m)
        else:
            assert m == 0, (frac, m)


def test_eps1_crossing_is_flagged():
    s = 0.25
    op = np.float32(1.0 - 1e-4)
    eps1 = 1.0 - float(op)  # T after the central hit equals eps1 exactly
    m, out = _mask(_scene([(0.0, 0.0, 0.0)], [(s, s, s)], [op], [(1.0, 0.5, 0.0)]), eps1=eps1)
    assert m & oracle.AMB_EPS1, m
    m, out = _mask(_scene([(0.0, 0.0, 0.0)], [(s, s, s)], [0.5], [(1.0, 0.5, 0.0)]), eps1=eps1)
    assert m == 0
