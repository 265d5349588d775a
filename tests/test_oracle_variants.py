"""Pins of the oracle's decision variants (render_variants).

Where an FP64 decision of the blend lies within the FP32 guard band of its threshold,
the oracle renders the ray both ways.  Each pin builds a ray whose near decision is
known by construction and checks the flipped variant against a closed form built from
single-Gaussian alphas (themselves pinned in closed form) or against a structural
identity: a render of a changed scene (a Gaussian removed, two input slots swapped,
the tile predicate dropped) that must give the same result.
"""
import numpy as np
import pytest

import oracle
from tests.helpers import front_camera, one_gaussian, small_lidar, stack

CAM = dict(width=32, height=32, f=40.0)
K_PIX = 16 * 32 + 16                 # pixel (col 16, row 16), centre (16.5, 16.5)


def _on_pixel(z, scale, opacity, feature, u=16.5, v=16.5):
    """A Gaussian whose mean projects onto the pixel centre (u, v) of the 32 x 32 camera."""
    cam = front_camera(**CAM)
    wy = -(u - cam.cx) * z / cam.fx       # camera x = -world y
    wz = -(v - cam.cy) * z / cam.fy       # camera y = -world z
    return one_gaussian((z, wy, wz), scale, opacity=opacity, feature=feature)


def _alpha(g, s, k):
    return 1.0 - oracle.render(g, s)["T"][k]


def _layers_to_stop(offset, z3=6.0):
    """Three layers, then a fourth tuned so that T after it is 1e-4 (1 + offset), then a
    fifth behind.  Returns the scene, the layer alphas and features."""
    cam = front_camera(**CAM)
    base = [(4.0, 0.8, 1.0), (5.0, 0.85, -2.0), (z3, 0.9, 0.5)]
    layers = [_on_pixel(z, (0.05, 0.2, 0.2), o, (f,)) for z, o, f in base]
    a = [_alpha(l, cam, K_PIX) for l in layers]
    T3 = np.prod([1 - x for x in a])
    assert 1e-3 < T3 < 0.1
    probe = _on_pixel(7.0, (0.05, 0.2, 0.2), 0.5, (3.0,))
    c = _alpha(probe, cam, K_PIX) / 0.5
    a4 = 1.0 - 1e-4 * (1 + offset) / T3
    fourth = _on_pixel(7.0, (0.05, 0.2, 0.2), a4 / c, (3.0,))
    fifth = _on_pixel(8.0, (0.05, 0.2, 0.2), 0.6, (7.0,))
    layers += [fourth, fifth]
    a = [_alpha(l, cam, K_PIX) for l in layers]
    return stack(*layers), a, [1.0, -2.0, 0.5, 3.0, 7.0]


def _blend(a, f, upto):
    T, F = 1.0, 0.0
    for i in range(upto):
        F += f[i] * a[i] * T
        T *= 1 - a[i]
    return F, T


def test_variant_zero_is_the_fp64_render():
    g, a, f = _layers_to_stop(1e-3)
    cam = front_camera(**CAM)
    r = oracle.render(g, cam)
    v = oracle.render_variants(g, cam)
    np.testing.assert_array_equal(v["F"][:, 0], r["F"])
    np.testing.assert_array_equal(v["T"][:, 0], r["T"])
    np.testing.assert_array_equal(v["marginal_bits"], r["marginal_bits"])


def test_stop_decision_above_the_threshold_flips_to_an_earlier_stop():
    g, a, f = _layers_to_stop(1e-3)       # T after the fourth layer: 1.001e-4, kept
    cam = front_camera(**CAM)
    v = oracle.render_variants(g, cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_STOP and v["n_var"][0] == 2
    F4, T4 = _blend(a, f, 4)              # FP64: four layers blended, the fifth stops the ray
    F3, T3 = _blend(a, f, 3)              # the other way: the ray stops before the fourth
    assert T4 == pytest.approx(1.001e-4, rel=1e-6)
    assert v["F"][0, 0, 0] == pytest.approx(F4, rel=1e-12) and v["T"][0, 0] == pytest.approx(T4, rel=1e-12)
    assert v["F"][0, 1, 0] == pytest.approx(F3, rel=1e-12) and v["T"][0, 1] == pytest.approx(T3, rel=1e-12)


def test_stop_decision_below_the_threshold_flips_to_one_more_gaussian():
    g, a, f = _layers_to_stop(-1e-3)      # T after the fourth layer would be 0.999e-4: stop before it
    cam = front_camera(**CAM)
    v = oracle.render_variants(g, cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_STOP and v["n_var"][0] == 2
    F3, T3 = _blend(a, f, 3)
    F4, T4 = _blend(a, f, 4)
    assert v["F"][0, 0, 0] == pytest.approx(F3, rel=1e-12) and v["T"][0, 0] == pytest.approx(T3, rel=1e-12)
    # the flipped ray blends the fourth layer; the fifth then takes T below 1e-4: stop
    assert v["F"][0, 1, 0] == pytest.approx(F4, rel=1e-12) and v["T"][0, 1] == pytest.approx(T4, rel=1e-12)


def test_alpha_threshold_decision_flips_to_blending_the_gaussian():
    """alpha at the ray just below 1/255, the Gaussian itself well visible (o' >> 1/255)."""
    cam = front_camera(**CAM)
    c = _alpha(_on_pixel(5.0, (0.1, 0.3, 0.3), 0.5, (1.0,), u=22.5), cam, K_PIX) / 0.5
    a = (1.0 / 255.0) * (1 - 2e-5)
    g = _on_pixel(5.0, (0.1, 0.3, 0.3), a / c, (2.5,), u=22.5)
    assert oracle.project(g, cam)["rec"][0, 5] > 5.0 / 255.0
    v = oracle.render_variants(g, cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_ALPHA_MIN and v["n_var"][0] == 2
    assert v["F"][0, 0, 0] == 0.0 and v["T"][0, 0] == 1.0
    assert v["F"][0, 1, 0] == pytest.approx(2.5 * a, rel=1e-6) and v["T"][0, 1] == pytest.approx(1 - a, rel=1e-9)


def test_cull_and_alpha_decisions_near_one_over_255_flip_together():
    """o' just below 1/255 (culled in FP64) and the ray at the mean: an FP32 run may keep
    the Gaussian and blend it, which takes both decisions the other way."""
    cam = front_camera(**CAM)
    c = _alpha(_on_pixel(5.0, (0.1, 0.3, 0.3), 0.5, (1.0,)), cam, K_PIX) / 0.5
    a = (1.0 / 255.0) * (1 - 2e-5)
    g = _on_pixel(5.0, (0.1, 0.3, 0.3), a / c, (2.5,))
    v = oracle.render_variants(g, cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_TILE | oracle.NEAR_ALPHA_MIN and v["n_var"][0] == 4
    assert v["F"][0, 0, 0] == 0.0 and v["T"][0, 0] == 1.0
    got = sorted(v["F"][0, :4, 0])
    assert got[:3] == [0.0, 0.0, 0.0]     # one flip alone still leaves it out
    assert got[3] == pytest.approx(2.5 * a, rel=1e-6)


def test_median_crossing_decision_flips_to_the_neighbouring_gaussian():
    lid = small_lidar()
    k = 7 * 256 + 0
    probe = one_gaussian((6.0, 0.0, 0.0), (0.3, 0.5, 0.5), opacity=0.5, feature=(1.0,))
    c = _alpha(probe, lid, k) / 0.5
    first = one_gaussian((6.0, 0.0, 0.0), (0.3, 0.5, 0.5), opacity=(1 - 0.5 * (1 + 5e-4)) / c, feature=(1.0,))
    second = one_gaussian((9.0, 0.0, 0.0), (0.3, 0.6, 0.6), opacity=0.4, feature=(1.0,))
    g = stack(second, first)
    a1, a2 = _alpha(first, lid, k), _alpha(second, lid, k)
    assert (1 - a1) == pytest.approx(0.5 * (1 + 5e-4), rel=1e-6) and (1 - a1) * (1 - a2) < 0.49
    v = oracle.render_variants(g, lid, sel=[k])
    assert v["marginal_bits"][0] == oracle.NEAR_MEDIAN and v["n_var"][0] == 2
    assert v["range_med"][0, 0] == pytest.approx(9.0, rel=1e-12)    # T first below 1/2 after the second
    assert v["range_med"][0, 1] == pytest.approx(6.0, rel=1e-12)    # taken at the first
    np.testing.assert_array_equal(v["F"][0, 1], v["F"][0, 0])        # nothing else changes
    assert v["range_exp"][0, 1] == v["range_exp"][0, 0]


def test_depth_tie_flip_equals_the_render_with_the_two_slots_swapped():
    cam = front_camera(**CAM)
    a = _on_pixel(6.0, (0.05, 0.3, 0.3), 0.7, (1.0, 0.0), u=16.2)
    b = _on_pixel(6.0, (0.05, 0.25, 0.4), 0.6, (0.0, 1.0), u=16.8)
    v = oracle.render_variants(stack(a, b), cam, sel=[K_PIX])
    swapped = oracle.render(stack(b, a), cam, sel=[K_PIX])   # equal depth: the lower slot blends first
    plain = oracle.render(stack(a, b), cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_TIE and v["n_var"][0] == 2
    assert abs(plain["F"][0, 0] - swapped["F"][0, 0]) > 1e-3      # the order matters at this ray
    np.testing.assert_allclose(v["F"][0, 0], plain["F"][0], rtol=0, atol=1e-15)
    np.testing.assert_allclose(v["F"][0, 1], swapped["F"][0], rtol=0, atol=1e-15)
    assert v["T"][0, 1] == pytest.approx(swapped["T"][0], rel=1e-14)


def _edge_gaussian(edge_u):
    """A large Gaussian (sigma about 8 px) whose 3-sigma box ends at image column edge_u."""
    cam = front_camera(**CAM)
    z = 5.0
    g = _on_pixel(z, (0.05, 1.0, 1.0), 0.95, (1.0,), u=0.0)
    ex = oracle.project(g, cam)["rec"][0, 14]
    for _ in range(4):           # place the mean so that mean + extent = edge_u
        g = _on_pixel(z, (0.05, 1.0, 1.0), 0.95, (1.0,), u=edge_u - ex)
        rec = oracle.project(g, cam)["rec"][0]
        ex = rec[14]
    assert abs(rec[0] + rec[14] - edge_u) < 1e-9
    return g


@pytest.mark.parametrize("edge_u, member", [(16.3, True), (15.7, False)])
def test_tile_membership_flip_equals_the_render_with_or_without_the_gaussian(edge_u, member):
    """Guard band of 0.5 px: the box edge lies 0.3 px from the tile edge at column 16."""
    cam = front_camera(**CAM)
    g = _edge_gaussian(edge_u)
    k = 8 * 32 + 16              # pixel (16, 8), tile column 1: beyond the box edge by 0.2 / 0.8 px
    v = oracle.render_variants(g, cam, sel=[k], guard=0.5)
    assert v["marginal_bits"][0] == oracle.NEAR_TILE and v["n_var"][0] == 2
    every = oracle.render(g, cam, sel=[k], every_gaussian=True)        # blended: the per-pixel definition
    assert every["F"][0, 0] > 1.0 / 255.0
    inside, outside = (0, 1) if member else (1, 0)
    np.testing.assert_allclose(v["F"][0, inside], every["F"][0], rtol=1e-14, atol=0)
    assert v["F"][0, outside, 0] == 0.0 and v["T"][0, outside] == 1.0   # as if the Gaussian were absent


def test_line_of_sight_cut_flip_moves_one_alpha_across_the_cut():
    lid = small_lidar()
    k = 7 * 256 + 0
    near = one_gaussian((6.0, 0.0, 0.0), (0.3, 0.5, 0.5), opacity=0.4, feature=(1.0,))
    far = one_gaussian((10.0, 0.0, 0.0), (0.3, 0.5, 0.5), opacity=0.3, feature=(1.0,))
    a1, a2 = _alpha(near, lid, k), _alpha(far, lid, k)
    rp = np.array([10.8 * (1 + 2e-6)])     # r_p - eps = 10.0 + 2.16e-5: the far Gaussian just inside the cut
    v = oracle.render_variants(stack(near, far), lid, sel=[k], los_range=rp, los_eps=0.8)
    assert v["marginal_bits"][0] == oracle.NEAR_LOS and v["n_var"][0] == 2
    assert v["los"][0, 0] == pytest.approx(a1 + a2, rel=1e-12)
    assert v["los"][0, 1] == pytest.approx(a1, rel=1e-12)


def test_two_near_decisions_give_four_variants_and_too_many_are_unresolved():
    """The second and third layers at equal depth (a tie, which leaves T unchanged) and
    the stop decision after the fourth: two near decisions, four renders."""
    g, a, f = _layers_to_stop(1e-3, z3=5.0)
    cam = front_camera(**CAM)
    v = oracle.render_variants(g, cam, sel=[K_PIX])
    assert v["marginal_bits"][0] == oracle.NEAR_TIE | oracle.NEAR_STOP
    assert v["n_near"][0] == 2 and v["n_var"][0] == 4 and not v["unresolved"][0]
    order = [0, 2, 1, 3, 4]                       # the tie taken the other way
    aa, ff = [a[i] for i in order], [f[i] for i in order]
    want = sorted([_blend(a, f, 4)[0], _blend(a, f, 3)[0], _blend(aa, ff, 4)[0], _blend(aa, ff, 3)[0]])
    np.testing.assert_allclose(sorted(v["F"][0, :4, 0]), want, rtol=1e-12, atol=0)
    assert len({round(x, 12) for x in want}) == 4
    v1 = oracle.render_variants(g, cam, sel=[K_PIX], max_dec=1)
    assert v1["unresolved"][0] and v1["n_var"][0] == 1
    np.testing.assert_array_equal(v1["F"][0, 0], v["F"][0, 0])
