"""Oracle for the global pose refinement of Sec. 2.5, float64 on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA path.

Sec. 2.5 keeps one learnable correction {Delta_R, Delta_t} shared by every
camera (training and test views alike), accumulates the gradient of the
rendering loss with respect to it at every iteration and updates the camera
poses with the optimised correction every 300 iterations.  The paper gives no
parameterisation or optimiser; the readings restated here are:

* The correction acts on the camera side: camera (W, t) (world -> camera)
  sees a world point p at  Delta_R (W p + t) + Delta_t,  i.e. its corrected
  world -> camera transform is [Delta_R W | Delta_R t + Delta_t].  (A
  world-side correction would be a rigid motion of the whole scene, which the
  Gaussians' own parameters already cover.)
* The accumulated gradient is that of the loss with respect to a left
  increment xi = (omega, tau) of the correction at xi = 0, the camera then
  seeing  exp([omega]_x) (Delta_R (W p + t) + Delta_t) + tau.  omega is an
  axis-angle rotation in the camera frame (about the camera centre), tau a
  translation in the camera frame.  Summed over every view and step of the
  window.
* Every `every` steps one Adam step (3DGS betas and eps; one rate for omega in
  radians, one for tau in scene units) turns the window's summed gradient
  into an increment xi = -Adam(g), the correction becomes
  exp(xi) o correction  (Delta_R <- exp([omega]_x) Delta_R,
  Delta_t <- exp([omega]_x) Delta_t + tau) and the sum restarts from zero.
"""
from __future__ import annotations

import math
from dataclasses import replace

import numpy as np
import torch

from . import adam, preprocess

_DT = torch.float64


def skew(w) -> np.ndarray:
    """[w]_x, the matrix of the cross product w x ."""
    x, y, z = (float(v) for v in w)
    return np.array([[0.0, -z, y], [z, 0.0, -x], [-y, x, 0.0]])


def so3_exp(omega) -> np.ndarray:
    """Rotation by the angle |omega| about omega / |omega| (Rodrigues):
    I + (sin th / th) K + ((1 - cos th) / th^2) K^2 with K = [omega]_x; below
    th = 1e-4 the two coefficients are their Taylor series to th^4."""
    omega = np.asarray(omega, dtype=np.float64)
    th2 = float(omega @ omega)
    th = math.sqrt(th2)
    K = skew(omega)
    if th < 1e-4:
        a = 1.0 - th2 / 6.0 + th2 * th2 / 120.0
        b = 0.5 - th2 / 24.0 + th2 * th2 / 720.0
    else:
        a = math.sin(th) / th
        b = (1.0 - math.cos(th)) / th2
    return np.eye(3) + a * K + b * (K @ K)


def identity_state() -> dict:
    """Correction (Delta_R, Delta_t) = (I, 0) and zero Adam moments."""
    return {"R": np.eye(3), "t": np.zeros(3), "m": np.zeros(6), "v": np.zeros(6), "step": 0}


def corrected_camera(cam, R_corr, t_corr):
    """The camera with the correction applied on its camera side, from the
    float32 transform the GPU receives (w2c) widened to float64."""
    w = np.asarray(cam.w2c(), dtype=np.float64)
    Rc = np.asarray(R_corr, dtype=np.float64)
    return replace(cam, R=Rc @ w[:, :3], t=Rc @ w[:, 3] + np.asarray(t_corr, dtype=np.float64))


def _projected_objective(pr, g):
    """sum over Gaussians of the projected quantities weighted by their
    loss gradients (the linearisation the preprocess backward chains
    through); culled Gaussians contribute nothing."""
    valid = pr["valid"].to(_DT)
    total = ((pr["mean2d"] * g[:, 0:2]).sum(-1) + (pr["conic"] * g[:, 2:5]).sum(-1) + pr["opacity"] * g[:, 5]
             + (pr["rgb"] * g[:, 6:9]).sum(-1) + (1.0 / pr["depth"]) * g[:, 9])
    return total * valid


def pose_grad_terms(scene, cam, grad2d: np.ndarray) -> np.ndarray:
    """Per-Gaussian terms of dL/d(omega, tau) for one view, (N, 6) float64:
    row i is what Gaussian i's projection contributes, its 2D gradients being
    grad2d[i] = dL/d[mean2d x, y, conic a, b, c, opacity, r, g, b, 1/z].
    Their sum over the Gaussians is the view's pose gradient.

    Autograd through the projection with a separate increment per Gaussian
    (the same function of xi for every row), so one backward pass yields each
    Gaussian's own share."""
    params = preprocess.params_from_scene(scene)
    n = params["means"].shape[0]
    xi = torch.zeros((n, 6), dtype=_DT, requires_grad=True)
    w = torch.as_tensor(np.asarray(cam.w2c(), dtype=np.float64), dtype=_DT)
    zero = torch.zeros(n, dtype=_DT)
    ox, oy, oz = xi[:, 0], xi[:, 1], xi[:, 2]
    K = torch.stack([torch.stack([zero, -oz, oy], -1), torch.stack([oz, zero, -ox], -1),
                     torch.stack([-oy, ox, zero], -1)], -2)
    E = torch.linalg.matrix_exp(K)
    R = E @ w[:, :3]
    t = torch.einsum("nij,j->ni", E, w[:, 3]) + xi[:, 3:6]
    pr = preprocess.project(params, cam, scene.sh_degree, R=R, t=t)
    _projected_objective(pr, torch.as_tensor(grad2d, dtype=_DT)).sum().backward()
    return xi.grad.detach().numpy().copy()


def pose_gradient(scene, cams, grad2ds) -> tuple[np.ndarray, np.ndarray]:
    """dL/d(omega, tau) summed over the views of a step, and the sum of the
    absolute per-Gaussian terms (the scale a float32 sum's rounding error is
    measured against)."""
    g = np.zeros(6)
    a = np.zeros(6)
    for cam, g2d in zip(cams, grad2ds):
        terms = pose_grad_terms(scene, cam, g2d)
        g += terms.sum(0)
        a += np.abs(terms).sum(0)
    return g, a


def pose_step(state: dict, grad, lr_rot: float, lr_trans: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-15) -> dict:
    """One update of the correction from the window's summed gradient."""
    step = state["step"] + 1
    lr = np.array([lr_rot] * 3 + [lr_trans] * 3)
    xi, m, v = adam.adam_step(np.zeros(6), grad, state["m"], state["v"], step, lr, b1, b2, eps)
    E = so3_exp(xi[:3])
    return {"R": E @ state["R"], "t": E @ state["t"] + xi[3:], "m": m, "v": v, "step": step}
