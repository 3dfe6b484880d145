"""Pins of the pose-refinement oracle (Sec. 2.5) against things other than
itself: scipy's rotation vectors, finite differences of the rendered image
under a perturbed camera, two rigid-motion identities that tie the camera
gradient to the Gaussians' own gradients, and the recovery of a known pose
error by the update rule."""
import math

import numpy as np
import pytest

import synth
from oracle import pose, preprocess, render, step
from synth.scenes import _look_at

scipy_rot = pytest.importorskip("scipy.spatial.transform")

W16 = 16


def _off_axis_camera(width=W16, height=W16, f=None):
    f = float(width) if f is None else f
    R, t = _look_at(np.array([0.7, -0.45, 0.1]), np.array([0.05, 0.0, 3.2]))
    return synth.Camera(f, f, 0.5 * width, 0.5 * height, R, t, width, height)


def _corr():
    return pose.so3_exp([0.03, -0.02, 0.05]), np.array([0.02, -0.01, 0.03])


def test_so3_exp_matches_scipy_rotation_vectors():
    rng = np.random.default_rng(3)
    for th in (0.0, 1e-9, 3e-6, 9e-5, 1.1e-4, 0.01, 0.7, 2.0, math.pi - 1e-6):
        axis = rng.standard_normal(3)
        w = th * axis / np.linalg.norm(axis)
        want = scipy_rot.Rotation.from_rotvec(w).as_matrix()
        np.testing.assert_allclose(pose.so3_exp(w), want, atol=2e-16 * 8, rtol=0)
    # one-parameter subgroup: exp(a w) exp(b w) = exp((a + b) w)
    w = np.array([0.2, -0.5, 0.3])
    np.testing.assert_allclose(pose.so3_exp(0.3 * w) @ pose.so3_exp(0.9 * w), pose.so3_exp(1.2 * w), atol=1e-15)


def test_corrected_camera_is_the_camera_side_composition():
    cam = _off_axis_camera()
    Rc, tc = _corr()
    cc = pose.corrected_camera(cam, Rc, tc)
    p = np.array([0.3, -0.2, 3.0])
    w = cam.w2c().astype(np.float64)
    np.testing.assert_allclose(cc.R @ p + cc.t, Rc @ (w[:, :3] @ p + w[:, 3]) + tc, atol=1e-15)


class Camera64(synth.Camera):
    """A camera whose transform reaches the oracle unrounded (the rigid-motion
    identities below need an orthonormal rotation; float32 rounding breaks
    orthonormality at the 1e-8 level)."""

    def w2c(self):
        return np.concatenate([self.R, self.t[:, None]], axis=1)


def _setup(seed, n=6, degree=1, exact=False):
    sc = synth.scene_tiny(n, seed=seed, sh_degree=degree)
    sc = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()), sh_degree=degree)
    base = _off_axis_camera()
    Rc, tc = _corr()
    if exact:  # composed from the unrounded camera: orthonormal to 1e-16
        cam = Camera64(**{k: getattr(base, k) for k in base.__dataclass_fields__})
        return sc, Camera64(**dict(cam.__dict__, R=Rc @ base.R, t=Rc @ base.t + tc))
    return sc, pose.corrected_camera(base, Rc, tc)


def _render_objective(sc, cam, R, t, g, gd, bg, win):
    import torch

    pr = preprocess.project(preprocess.params_from_scene(sc), cam, sc.sh_degree,
                            R=torch.as_tensor(R), t=torch.as_tensor(t))
    f = render.render_fwd(preprocess.pack_for_render(pr), bg, win, amb=None)
    return float((f["rgb"] * g).sum() + (f["disp"] * gd).sum())


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_pose_gradient_matches_finite_differences(seed):
    sc, cam = _setup(seed, n=6, degree=1 + seed % 3)
    win = (0, 0, W16, W16)
    bg = (0.3, 0.1, 0.6)
    g, gd = synth.upstream_grads(seed + 40, W16, W16)
    g, gd = g.astype(np.float64), gd.astype(np.float64)
    rec = preprocess.pack_for_render(preprocess.project(preprocess.params_from_scene(sc), cam, sc.sh_degree))
    assert rec[:, 11].sum() >= 4  # most Gaussians in front of the camera
    amb = render.render_fwd(rec, bg, win, amb=(1e-4, 1e-4, 1e-4, 1e-6))["amb"]
    g[:, amb] = 0.0
    gd[amb] = 0.0
    g2d = render.render_bwd(rec, bg, win, g, gd)
    got, scale = pose.pose_gradient(sc, [cam], [g2d])
    assert np.all(scale > 0)
    w = cam.w2c().astype(np.float64)
    for k in range(6):
        h = 1e-6
        vals = []
        for sgn in (1.0, -1.0):
            xi = np.zeros(6)
            xi[k] = sgn * h
            E = pose.so3_exp(xi[:3])
            vals.append(_render_objective(sc, cam, E @ w[:, :3], E @ w[:, 3] + xi[3:], g, gd, bg, win))
        fd = (vals[0] - vals[1]) / (2 * h)
        assert abs(got[k] - fd) <= 2e-5 * max(1.0, abs(fd)), (k, got[k], fd)


@pytest.mark.parametrize("degree", [0, 2, 3])
def test_camera_translation_equals_moving_every_gaussian(degree):
    """Shifting the camera by tau in its own frame moves every Gaussian by
    W^T tau relative to it (the camera centre moves by -W^T tau), so
    dL/dtau = W sum_i dL/dmean_i for any SH degree."""
    sc, cam = _setup(5, n=7, degree=degree, exact=True)
    g2d = np.random.default_rng(degree).standard_normal((sc.n, 10))
    terms = pose.pose_grad_terms(sc, cam, g2d)
    gm = preprocess.preprocess_backward(sc, cam, g2d)["means"]
    W = cam.w2c().astype(np.float64)[:, :3]
    np.testing.assert_allclose(terms[:, 3:].sum(0), W @ gm.sum(0), rtol=1e-10, atol=1e-12)
    # and Gaussian by Gaussian
    np.testing.assert_allclose(terms[:, 3:], gm @ W.T, rtol=1e-10, atol=1e-12)


def _quat_left_rotation_grad(q, gq):
    """dL/dphi for q <- exp(phi) o q (a world rotation phi applied to the
    Gaussian's orientation): dq = 1/2 (0, dphi) (x) q (Hamilton product)."""
    w, v = q[:, 0], q[:, 1:]
    out = np.zeros((q.shape[0], 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = 1.0
        dq = np.concatenate([(-(v @ e))[:, None], w[:, None] * e + np.cross(e, v)], 1) * 0.5
        out[:, k] = (gq * dq).sum(1)
    return out


def test_camera_rotation_equals_rotating_the_scene_about_the_camera_centre():
    """With view-independent colour (SH degree 0), rotating the camera by
    omega about its centre c equals rotating every Gaussian (position about c
    and orientation) by the world rotation Q = W^T exp([omega]_x) W, whose axis
    is W^T omega: dL/domega = W sum_i [(p_i - c) x dL/dp_i + dL/dphi_i]."""
    sc, cam = _setup(8, n=7, degree=0, exact=True)
    g2d = np.random.default_rng(2).standard_normal((sc.n, 10))
    terms = pose.pose_grad_terms(sc, cam, g2d)
    gr = preprocess.preprocess_backward(sc, cam, g2d)
    w = cam.w2c().astype(np.float64)
    W, t = w[:, :3], w[:, 3]
    c = -W.T @ t
    p = np.asarray(sc.means, dtype=np.float64)
    dphi = np.cross(p - c, gr["means"]) + _quat_left_rotation_grad(np.asarray(sc.quats, dtype=np.float64),
                                                                    gr["quats"])
    np.testing.assert_allclose(terms[:, :3], dphi @ W.T, rtol=1e-9, atol=1e-11)


def test_first_pose_step_moves_each_component_by_its_rate():
    """Adam's first bias-corrected step is lr * g / |g| per component, so the
    increment is xi = -(lr_rot, lr_rot, lr_rot, lr_trans, ...) * sign(g)."""
    st = pose.identity_state()
    R0, t0 = _corr()
    st["R"], st["t"] = R0.copy(), t0.copy()
    g = np.array([3.0, -1e-3, 2e4, -5.0, 7e-6, 1.0])
    new = pose.pose_step(st, g, lr_rot=1e-3, lr_trans=4e-3)
    xi = -np.sign(g) * np.array([1e-3] * 3 + [4e-3] * 3)
    E = scipy_rot.Rotation.from_rotvec(xi[:3]).as_matrix()
    np.testing.assert_allclose(new["R"], E @ R0, atol=1e-14)
    np.testing.assert_allclose(new["t"], E @ t0 + xi[3:], atol=1e-14)
    assert new["step"] == 1
    # the corrected rotation stays orthonormal
    np.testing.assert_allclose(new["R"] @ new["R"].T, np.eye(3), atol=1e-14)


def test_pose_steps_recover_a_known_camera_side_error():
    """Targets rendered through the true cameras; the training cameras carry
    the same camera-side error (rotation 0.029 rad, translation 0.029).  With the
    Gaussians fixed, pose steps on the loss gradient drive the correction
    towards the inverse of the error."""
    sc = synth.scene_tiny(24, seed=4, sh_degree=0, width=32, height=32)
    sc = synth.Scene(*(a.astype(np.float64) for a in sc.arrays()), sh_degree=0)
    base = [_off_axis_camera(32, 32, f=32.0), synth.camera_tiny(32, 32)]
    base[1] = synth.Camera(32.0, 32.0, 16.0, 16.0, pose.so3_exp([0.0, 0.12, 0.0]), np.array([-0.35, 0.0, 0.1]),
                           32, 32)
    targets = [step.forward_backward(sc, c, np.zeros((3, 32, 32)), lam=0.0)[2]["rgb"] for c in base]
    err_R, err_t = pose.so3_exp([0.02, -0.015, 0.015]), np.array([0.02, 0.015, -0.015])
    train = [pose.corrected_camera(c, err_R, err_t) for c in base]

    def reprojection_error(st):
        # mean pixel distance between the Gaussians' centres seen through the
        # true cameras and through the corrected training cameras (a rotation
        # about the camera centre and a sideways shift look alike at one
        # depth, so the observable is the image, not the transform)
        p = np.asarray(sc.means, dtype=np.float64)
        d = []
        for c0, ct in zip(base, train):
            c1 = pose.corrected_camera(ct, st["R"], st["t"])
            uv = []
            for c in (c0, c1):
                w = c.w2c().astype(np.float64)
                pc = p @ w[:, :3].T + w[:, 3]
                uv.append(c.fx * pc[:, :2] / pc[:, 2:3])
            d.append(np.linalg.norm(uv[0] - uv[1], axis=1).mean())
        return float(np.mean(d))

    st = pose.identity_state()
    e0 = reprojection_error(st)
    losses = []
    for it in range(60):
        cams = [pose.corrected_camera(c, st["R"], st["t"]) for c in train]
        g = np.zeros(6)
        tot = 0.0
        for c, tgt in zip(cams, targets):
            L, _, f = step.forward_backward(sc, c, tgt, lam=0.0)
            tot += L
            g += pose.pose_gradient(sc, [c], [f["grad2d"]])[0]
        losses.append(tot)
        lr = 2e-3 * 0.1 ** (it / 60)
        st = pose.pose_step(st, g, lr_rot=lr, lr_trans=lr)
    e1 = reprojection_error(st)
    assert losses[-1] < 0.2 * losses[0], losses[::10]
    assert e1 < 0.2 * e0, (e0, e1)
