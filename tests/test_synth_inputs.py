"""The seeded input generators: the same seed gives the same arrays, and the
recipes have the stated shapes and distributions (these inputs feed both the
CUDA path and the oracle, so their properties are checked on their own)."""
import numpy as np

import synth


def test_generators_are_deterministic_per_seed():
    a, b = synth.scene_clustered(2000, seed=5), synth.scene_clustered(2000, seed=5)
    for x, y in zip(a.arrays(), b.arrays()):
        np.testing.assert_array_equal(x, y)
    c = synth.scene_clustered(2000, seed=6)
    assert not np.array_equal(a.means, c.means)


def test_clustered_scene_recipe():
    sc = synth.scene_clustered(20000, seed=1, sh_degree=3)
    assert sc.means.shape == (20000, 3) and sc.sh.shape == (20000, 16, 3)
    assert sc.means.dtype == np.float32
    # log-scales N(-4, 0.7); unit quaternions; logits N(0, 1)
    assert abs(float(sc.log_scales.mean()) + 4.0) < 0.05 and abs(float(sc.log_scales.std()) - 0.7) < 0.05
    np.testing.assert_allclose(np.linalg.norm(sc.quats, axis=1), 1.0, atol=1e-5)
    assert abs(float(sc.opacity_logits.mean())) < 0.05 and abs(float(sc.opacity_logits.std()) - 1.0) < 0.05


def test_ring_cameras_look_at_the_origin():
    for cam in synth.ring_cameras(16, 1920, 1080):
        R, t = cam.R, cam.t
        np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
        centre = -R.T @ t
        assert abs(np.linalg.norm(centre) - 4.0) < 1e-9
        # the origin projects to the principal point
        pc = R @ np.zeros(3) + t
        assert pc[2] > 0 and abs(cam.fx * pc[0] / pc[2]) < 1e-6 and abs(cam.fy * pc[1] / pc[2]) < 1e-6


def test_camera_pose_error_has_the_stated_size_and_acts_on_the_camera_side():
    R, t = synth.camera_pose_error(0.03, 0.12, seed=7)
    np.testing.assert_allclose(R @ R.T, np.eye(3), atol=1e-12)
    angle = np.arccos(np.clip((np.trace(R) - 1.0) / 2.0, -1.0, 1.0))
    assert abs(angle - 0.03) < 1e-12 and abs(np.linalg.norm(t) - 0.12) < 1e-12
    cams = synth.ring_cameras(4, 64, 48)
    bad = synth.with_pose_error(cams, R, t)
    p = np.array([0.3, -0.2, 0.5])
    for c0, c1 in zip(cams, bad):
        np.testing.assert_allclose(c1.R @ p + c1.t, R @ (c0.R @ p + c0.t) + t, atol=1e-12)
    R2, t2 = synth.camera_pose_error(0.03, 0.12, seed=7)
    np.testing.assert_array_equal(R, R2)
    np.testing.assert_array_equal(t, t2)


def test_time_to_psnr_interpolates_the_curve():
    from paper_2601_19489_gb300.recon import time_to_psnr

    curve = [(0.0, 15.0), (5.0, 20.0), (10.0, 24.0), (15.0, 25.0)]
    assert time_to_psnr(curve, 22.0) == 7.5
    assert time_to_psnr(curve, 15.0) == 0.0
    assert time_to_psnr(curve, 25.0) == 15.0
    assert time_to_psnr(curve, 26.0) is None
