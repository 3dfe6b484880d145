"""Pins of the oracle's per-Gaussian preprocess (Sec. 2.1) against things
other than itself: scipy's spherical harmonics and rotations, numerical
Jacobians of the pinhole map, camera geometry and finite differences."""
import numpy as np
import pytest
import torch

import synth
from oracle import preprocess

scipy_special = pytest.importorskip("scipy.special")
scipy_rot = pytest.importorskip("scipy.spatial.transform")


def _real_sh_scipy(l, m, d):
    x, y, z = d.T
    theta = np.arccos(np.clip(z, -1, 1))
    phi = np.arctan2(y, x)
    Y = scipy_special.sph_harm_y(l, abs(m), theta, phi)
    if m == 0:
        return Y.real
    return np.sqrt(2.0) * (Y.real if m > 0 else Y.imag)


def test_sh_basis_matches_scipy_complex_harmonics():
    rng = np.random.default_rng(3)
    d = rng.standard_normal((200, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    got = preprocess.sh_basis(3, torch.as_tensor(d)).numpy()
    for l in range(4):
        for m in range(-l, l + 1):
            k = l * l + l + m
            np.testing.assert_allclose(got[:, k], _real_sh_scipy(l, m, d), rtol=1e-12, atol=1e-12,
                                       err_msg=f"l={l} m={m}")


def test_sh_basis_is_orthonormal_on_the_sphere():
    # Monte Carlo over the sphere: E[Y_i Y_j] * 4 pi = delta_ij.
    rng = np.random.default_rng(4)
    d = rng.standard_normal((400000, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    Y = preprocess.sh_basis(3, torch.as_tensor(d)).numpy()
    gram = Y.T @ Y * (4.0 * np.pi / d.shape[0])
    np.testing.assert_allclose(gram, np.eye(16), atol=0.02)


def test_quaternion_rotation_matches_scipy():
    rng = np.random.default_rng(5)
    q = rng.standard_normal((100, 4)) * 3.0  # unnormalised on purpose
    got = preprocess.quat_to_rotmat(torch.as_tensor(q)).numpy()
    ref = scipy_rot.Rotation.from_quat(q[:, [1, 2, 3, 0]]).as_matrix()
    np.testing.assert_allclose(got, ref, atol=1e-12)


def _pinhole(cam, pc):
    # the intrinsics as the GPU receives them: rounded to float32
    fx, fy, cx, cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    return np.array([fx * pc[0] / pc[2] + cx, fy * pc[1] / pc[2] + cy])


def _num_jac(cam, pc, h=1e-6):
    J = np.zeros((2, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        J[:, k] = (_pinhole(cam, pc + e) - _pinhole(cam, pc - e)) / (2 * h)
    return J


def test_jacobian_and_covariance_against_numerical_projection():
    cams = synth.ring_cameras(4, 320, 200)
    scene = synth.scene_clustered(300, seed=2, sh_degree=0, log_scale_mean=-2.5)
    rng = np.random.default_rng(0)
    for cam in cams:
        p = preprocess.params_from_scene(scene)
        pr = preprocess.project(p, cam, 0)
        R = cam.w2c()[:, :3].astype(np.float64)
        t = cam.w2c()[:, 3].astype(np.float64)
        for i in rng.choice(scene.n, 20, replace=False):
            pc = R @ scene.means[i].astype(np.float64) + t
            if pc[2] <= 0.2:
                continue
            limx = 1.3 * cam.width / (2 * float(np.float32(cam.fx)))
            limy = 1.3 * cam.height / (2 * float(np.float32(cam.fy)))
            pcl = pc.copy()
            pcl[0] = np.clip(pc[0] / pc[2], -limx, limx) * pc[2]
            pcl[1] = np.clip(pc[1] / pc[2], -limy, limy) * pc[2]
            Jn = _num_jac(cam, pcl)
            np.testing.assert_allclose(pr["J"][i].numpy(), Jn, rtol=1e-6, atol=1e-6)
            Rg = scipy_rot.Rotation.from_quat(scene.quats[i, [1, 2, 3, 0]].astype(np.float64)).as_matrix()
            S = np.diag(np.exp(2.0 * scene.log_scales[i].astype(np.float64)))
            cov = Jn @ R @ Rg @ S @ Rg.T @ R.T @ Jn.T + 0.3 * np.eye(2)
            got = pr["cov2d"][i].numpy()
            np.testing.assert_allclose(got, [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-5)
            conic = pr["conic"][i].numpy()
            Cm = np.array([[conic[0], conic[1]], [conic[1], conic[2]]])
            Sm = np.array([[got[0], got[1]], [got[1], got[2]]])
            np.testing.assert_allclose(Cm @ Sm, np.eye(2), atol=1e-10)
            np.testing.assert_allclose(pr["mean2d"][i].numpy(), _pinhole(cam, pc), rtol=1e-12)


def test_frustum_clamp_uses_the_clamped_point():
    cam = synth.camera_tiny(64, 64)
    scene = synth.scene_tiny(2, seed=1, sh_degree=0)
    scene.means[0] = [3.0, -2.5, 2.0]  # x/z = 1.5 > 1.3 * 0.5
    p = preprocess.params_from_scene(scene)
    pr = preprocess.project(p, cam, 0)
    z = float(scene.means[0, 2])
    lim = 1.3 * 0.5
    Jn = _num_jac(cam, np.array([lim * z, -lim * z, z]))
    np.testing.assert_allclose(pr["J"][0].numpy(), Jn, rtol=1e-6)


def test_ring_camera_geometry():
    cam = synth.ring_cameras(16, 1920, 1080)[5]
    p = preprocess.params_from_scene(synth.Scene(
        np.zeros((2, 3), np.float32), np.zeros((2, 3), np.float32),
        np.tile(np.float32([1, 0, 0, 0]), (2, 1)), np.zeros(2, np.float32),
        np.zeros((2, 1, 3), np.float32), 0))
    # the ring centre projects to the principal point at depth = radius
    pr = preprocess.project(p, cam, 0)
    np.testing.assert_allclose(pr["mean2d"][0].numpy(), [cam.cx, cam.cy], atol=1e-4)
    np.testing.assert_allclose(pr["depth"][0].item(), 4.0, rtol=1e-6)
    # a point offset by delta along the camera's +x axis lands fx*delta/4 to the right
    delta = 0.1
    xaxis = cam.R[0]
    p["means"][1] = torch.as_tensor(xaxis * delta)
    pr = preprocess.project(p, cam, 0)
    np.testing.assert_allclose(pr["mean2d"][1, 0].item() - cam.cx, cam.fx * delta / 4.0, rtol=1e-5)


def test_single_isotropic_gaussian_closed_form():
    f, z, sw = 300.0, 3.0, 0.02
    cam = synth.Camera(f, f, 32.0, 32.0, np.eye(3), np.zeros(3), 64, 64)
    sc = synth.Scene(np.float32([[0, 0, z]]), np.full((1, 3), np.log(sw), np.float32),
                     np.float32([[0.3, -0.2, 0.9, 0.1]]), np.float32([0.4]),
                     np.zeros((1, 1, 3), np.float32), 0)
    pr = preprocess.project(preprocess.params_from_scene(sc), cam, 0)
    sw32 = float(np.exp(np.float64(np.float32(np.log(sw)))))
    var = (f * sw32 / z) ** 2 + 0.3
    np.testing.assert_allclose(pr["cov2d"][0].numpy(), [var, 0.0, var], rtol=1e-9, atol=1e-9)
    np.testing.assert_allclose(pr["conic"][0].numpy(), [1 / var, 0.0, 1 / var], rtol=1e-9, atol=1e-12)
    o = 1.0 / (1.0 + np.exp(-np.float64(np.float32(0.4))))
    np.testing.assert_allclose(pr["opacity"][0].item(), o, rtol=1e-12)
    np.testing.assert_allclose(pr["level"][0].item(), 2 * np.log(255 * o), rtol=1e-12)
    np.testing.assert_allclose(pr["rgb"][0].numpy(), [0.5, 0.5, 0.5], atol=1e-12)


def test_rgb_clamp_and_direction_dependence():
    cam = synth.camera_tiny(16, 16)
    sc = synth.scene_tiny(3, seed=7, sh_degree=1)
    sc.sh[0, 0] = -5.0  # force the clamp on Gaussian 0
    pr = preprocess.project(preprocess.params_from_scene(sc), cam, 1)
    assert bool(pr["rgb_clamped"][0].all())
    assert float(pr["rgb"][0].abs().max()) == 0.0
    # degree-1 colour equals DC + the l = 1 terms along the viewing direction
    m = sc.means[1].astype(np.float64)
    d = m / np.linalg.norm(m)
    Y = [_real_sh_scipy(0, 0, d[None])[0]] + [_real_sh_scipy(1, mm, d[None])[0] for mm in (-1, 0, 1)]
    want = np.maximum(0.0, np.einsum("k,kc->c", Y, sc.sh[1].astype(np.float64)) + 0.5)
    np.testing.assert_allclose(pr["rgb"][1].numpy(), want, rtol=1e-10)


def test_preprocess_backward_matches_finite_differences():
    cam = synth.camera_tiny(16, 16)
    sc = synth.scene_tiny(4, seed=11, sh_degree=2)
    rng = np.random.default_rng(1)
    g2d = rng.standard_normal((sc.n, 10))
    got = preprocess.preprocess_backward(sc, cam, g2d)

    def F(scene):
        pr = preprocess.project(preprocess.params_from_scene(scene), cam, scene.sh_degree)
        vals = torch.cat([pr["mean2d"], pr["conic"], pr["opacity"][:, None], pr["rgb"],
                          (1.0 / pr["depth"])[:, None]], 1).numpy()
        return float((vals * g2d).sum())

    base = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()), sh_degree=sc.sh_degree)
    for name in ("means", "log_scales", "quats", "opacity_logits", "sh"):
        arr = getattr(base, name)
        fd = np.zeros_like(arr)
        for idx in np.ndindex(arr.shape):
            h = 1e-6
            old = arr[idx]
            arr[idx] = old + h
            fp = F(base)
            arr[idx] = old - h
            fm = F(base)
            arr[idx] = old
            fd[idx] = (fp - fm) / (2 * h)
        np.testing.assert_allclose(got[name], fd, rtol=1e-5, atol=1e-6, err_msg=name)
