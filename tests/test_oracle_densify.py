"""Pins of the densification oracle (Sec. 3.2, Eq. 3-6): the contributor
scores against closed forms, the blend's stop rule and additivity; the
actions against their rules; clone and split against their definitions
with an independent rotation (scipy)."""
import math

import numpy as np
import pytest

import synth
from oracle import densify, render


def rec(mx, my, a, b, c, o, rgb, z):
    t = 2.0 * math.log(255.0 * o)
    return [mx, my, a, b, c, o, rgb[0], rgb[1], rgb[2], z, t, 1.0]


def test_single_gaussian_score_counts_masked_pixels_inside_the_level_set():
    var, o = 6.0, 0.7
    r = np.array([rec(12.3, 10.8, 1 / var, 0.0, 1 / var, o, (1, 1, 1), 2.0)])
    rng = np.random.default_rng(0)
    mask = rng.uniform(size=(24, 26)) > 0.5
    s = render.contrib_score(r, (0, 0, 26, 24), mask.astype(float))
    i, j = np.meshgrid(np.arange(26) + 0.5, np.arange(24) + 0.5)
    inside = o * np.exp(-0.5 * ((i - 12.3) ** 2 + (j - 10.8) ** 2) / var) >= 1 / 255
    assert s[0] == float((mask & inside).sum()) > 0


def test_stopped_splat_scores_nothing_at_the_stopping_pixel():
    # four alpha = 0.95 splats at one pixel: three blend, the fourth stops
    rows = [rec(4.5, 4.5, 1.0, 0.0, 1.0, 0.95, (1, 1, 1), 1.0 + k) for k in range(4)]
    w = np.zeros((9, 9))
    w[4, 4] = 1.0
    s = render.contrib_score(np.array(rows), (0, 0, 9, 9), w)
    np.testing.assert_array_equal(s, [1.0, 1.0, 1.0, 0.0])


def test_scores_are_additive_in_the_weights():
    scene = synth.scene_tiny(6, seed=32, sh_degree=1, width=20, height=16)
    cam = synth.camera_tiny(20, 16)
    from oracle import preprocess

    r = preprocess.pack_for_render(preprocess.project(preprocess.params_from_scene(scene), cam, 1))
    rng = np.random.default_rng(1)
    w1, w2 = rng.uniform(size=(16, 20)), rng.uniform(size=(16, 20))
    a = render.contrib_score(r, (0, 0, 20, 16), w1)
    b = render.contrib_score(r, (0, 0, 20, 16), w2)
    c = render.contrib_score(r, (0, 0, 20, 16), w1 + w2)
    np.testing.assert_allclose(a + b, c, rtol=1e-12)
    assert (a > 0).sum() >= 3


def test_error_mask_normalises_by_the_view_maximum():
    rgb = np.zeros((3, 2, 2))
    tgt = np.zeros((3, 2, 2))
    tgt[:, 0, 0] = [0.5, 0.5, 0.5]  # E = 1.5 (the maximum)
    tgt[0, 1, 1] = 0.6  # E = 0.6 -> 0.4
    tgt[1, 0, 1] = 0.9  # E = 0.9 -> 0.6
    m = densify.error_mask(rgb, tgt, 0.5)
    np.testing.assert_array_equal(m, [[True, True], [False, False]])
    assert not densify.error_mask(rgb, rgb, 0.1).any()


def test_actions_follow_the_rules():
    sc = synth.Scene(np.zeros((5, 3), np.float32), np.log(np.array([[0.01] * 3, [0.01] * 3, [0.2] * 3,
                                                                    [0.01] * 3, [0.2] * 3], np.float32)),
                     np.tile(np.array([[1, 0, 0, 0]], np.float32), (5, 1)),
                     np.array([2.0, 2.0, 2.0, -9.0, 2.0], np.float32), np.zeros((5, 1, 3), np.float32), 0)
    s_plus = np.array([30.0, 1.0, 30.0, 30.0, 30.0]) * 2  # summed over K = 2 views
    r_minus = np.array([0.0, 0.0, 0.0, 0.0, 10.0])
    act = densify.actions(sc, s_plus, r_minus, K=2, tau_plus=5.0, tau_minus=0.9, min_opacity=0.005,
                          percent_dense=0.01, extent=4.0)
    # small + high score: clone; low score: keep; large: split; transparent:
    # prune; the most pruning-scored: prune (wins over split)
    np.testing.assert_array_equal(act, [densify.CLONE, densify.KEEP, densify.SPLIT, densify.PRUNE,
                                        densify.PRUNE])


def test_apply_clone_split_prune_against_definitions():
    Rot = pytest.importorskip("scipy.spatial.transform").Rotation
    rng = np.random.default_rng(3)
    N = 4
    q = rng.standard_normal((N, 4))
    arrays = {"means": rng.standard_normal((N, 3)), "log_scales": rng.normal(-2, 0.3, (N, 3)),
              "quats": q, "opacity_logits": rng.standard_normal(N), "sh": rng.standard_normal((N, 4, 3))}
    m = {k: rng.standard_normal(np.shape(a)) for k, a in arrays.items()}
    v = {k: rng.uniform(size=np.shape(a)) for k, a in arrays.items()}
    act = np.array([densify.KEEP, densify.SPLIT, densify.PRUNE, densify.CLONE], np.int32)
    normals = rng.standard_normal((N, 2, 3))
    out, om, ov = densify.apply(arrays, m, v, act, normals)
    assert out["means"].shape[0] == 1 + 2 + 0 + 2
    # kept row: unchanged with its moments
    for k in arrays:
        np.testing.assert_array_equal(out[k][0], arrays[k][0])
        np.testing.assert_array_equal(om[k][0], m[k][0])
    # split rows: mean + R diag(s) z with R from scipy (w, x, y, z -> scipy's x, y, z, w)
    R = Rot.from_quat(np.roll(q[1] / np.linalg.norm(q[1]), -1)).as_matrix()
    s = np.exp(arrays["log_scales"][1])
    for c in range(2):
        np.testing.assert_allclose(out["means"][1 + c], arrays["means"][1] + R @ (s * normals[1, c]), rtol=1e-12)
        np.testing.assert_allclose(np.exp(out["log_scales"][1 + c]), s / 1.6, rtol=1e-12)
        np.testing.assert_array_equal(out["sh"][1 + c], arrays["sh"][1])
        assert not om["means"][1 + c].any() and not ov["sh"][1 + c].any()
    # clone: the original with its moments, then a copy with zero moments
    for k in arrays:
        np.testing.assert_array_equal(out[k][3], arrays[k][3])
        np.testing.assert_array_equal(out[k][4], arrays[k][3])
        np.testing.assert_array_equal(ov[k][3], v[k][3])
        assert not np.any(ov[k][4])
