"""Oracle for the per-Gaussian preprocess (EWA projection, SH colour, opacity
level set) and its backward, in float64 PyTorch on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.  It shares no code with the CUDA path.

The forward is the definition written out term by term; the backward is
PyTorch autograd through that definition, so the chain rule (through the
conic inverse, the low-pass dilation, the clamped Jacobian, the world-to-camera
rotation, R S S^T R^T, the quaternion normalisation, exp, sigmoid and the SH
evaluation including its dependence on the mean) is exact by construction.

Paper passages followed: Sec. 2.1 (preprocessCUDA: project each Gaussian with
the local affine approximation, 2D centroid and covariance, Eq. 1 level set
t = 2 ln(255 o) whose ellipse is written with the conic {a, b, c}).  Where the
paper is silent it builds on the original 3DGS conventions, restated here:
near plane z > 0.2; Sigma = R(q/|q|) diag(e^{2s}) R^T; J the Jacobian of
(fx x/z + cx, fy y/z + cy) at the camera-space mean with x/z and y/z clamped to
+-1.3 tan(fov/2); Sigma' = J W Sigma W^T J^T + 0.3 I; conic = Sigma'^{-1};
o = sigmoid(logit); colour = max(0, sum_k sh_k Y_k(d) + 0.5) with d the unit
vector from the camera centre to the mean and Y_k the real spherical harmonics
(Condon-Shortley phase) of degree <= 3.
"""
from __future__ import annotations

import math

import numpy as np
import torch

NEAR_DEFAULT = 0.2
DILATION = 0.3
FRUSTUM_SLACK = 1.3

_DT = torch.float64


def _t(a) -> torch.Tensor:
    return torch.as_tensor(np.asarray(a, dtype=np.float64), dtype=_DT)


def camera_tensors(cam):
    """World->camera rotation/translation widened from float32 (the values
    the GPU receives) to float64."""
    w2c = torch.as_tensor(cam.w2c().astype(np.float64), dtype=_DT)
    return w2c[:, :3], w2c[:, 3]


def intrinsics(cam):
    """fx, fy, cx, cy rounded to float32 (the values the GPU receives) and
    widened to float64."""
    return tuple(float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))


def quat_to_rotmat(q: torch.Tensor) -> torch.Tensor:
    """Rotation matrix of the unit quaternion q / |q|, q = (w, x, y, z)."""
    q = q / torch.linalg.norm(q, dim=-1, keepdim=True)
    w, x, y, z = q.unbind(-1)
    r00 = 1 - 2 * (y * y + z * z)
    r01 = 2 * (x * y - w * z)
    r02 = 2 * (x * z + w * y)
    r10 = 2 * (x * y + w * z)
    r11 = 1 - 2 * (x * x + z * z)
    r12 = 2 * (y * z - w * x)
    r20 = 2 * (x * z - w * y)
    r21 = 2 * (y * z + w * x)
    r22 = 1 - 2 * (x * x + y * y)
    return torch.stack([r00, r01, r02, r10, r11, r12, r20, r21, r22], -1).reshape(q.shape[:-1] + (3, 3))


def sh_basis(degree: int, d: torch.Tensor) -> torch.Tensor:
    """Real spherical harmonics Y_k(d), k = l^2 + l + m, for unit vectors d.

    Real form of the complex harmonics with the Condon-Shortley phase:
    m > 0 -> sqrt(2) Re Y_l^m, m < 0 -> sqrt(2) Im Y_l^|m|, m = 0 -> Y_l^0,
    written as polynomials in (x, y, z) with normalisation constants computed
    from their closed forms.
    """
    x, y, z = d.unbind(-1)
    pi = math.pi
    out = [torch.full_like(x, 0.5 / math.sqrt(pi))]
    if degree >= 1:
        c1 = math.sqrt(3.0 / (4.0 * pi))
        out += [-c1 * y, c1 * z, -c1 * x]
    if degree >= 2:
        c2a = 0.5 * math.sqrt(15.0 / pi)
        c2b = 0.25 * math.sqrt(5.0 / pi)
        c2c = 0.25 * math.sqrt(15.0 / pi)
        out += [c2a * x * y, -c2a * y * z, c2b * (3.0 * z * z - 1.0), -c2a * x * z,
                c2c * (x * x - y * y)]
    if degree >= 3:
        c3a = 0.25 * math.sqrt(35.0 / (2.0 * pi))
        c3b = 0.5 * math.sqrt(105.0 / pi)
        c3c = 0.25 * math.sqrt(21.0 / (2.0 * pi))
        c3d = 0.25 * math.sqrt(7.0 / pi)
        c3e = 0.25 * math.sqrt(105.0 / pi)
        out += [-c3a * y * (3.0 * x * x - y * y), c3b * x * y * z, -c3c * y * (5.0 * z * z - 1.0),
                c3d * z * (5.0 * z * z - 3.0), -c3c * x * (5.0 * z * z - 1.0),
                c3e * z * (x * x - y * y), -c3a * x * (x * x - 3.0 * y * y)]
    return torch.stack(out, -1)


def params_from_scene(scene, requires_grad: bool = False) -> dict:
    p = {
        "means": _t(scene.means),
        "log_scales": _t(scene.log_scales),
        "quats": _t(scene.quats),
        "opacity_logits": _t(scene.opacity_logits),
        "sh": _t(scene.sh),
    }
    if requires_grad:
        for v in p.values():
            v.requires_grad_(True)
    return p


def project(params: dict, cam, sh_degree: int, R: torch.Tensor | None = None,
            t: torch.Tensor | None = None) -> dict:
    """Per-Gaussian projected quantities in float64 (differentiable).

    R, t: the world->camera transform to use instead of the camera's own,
    either one (3, 3) / (3,) for all Gaussians or one per Gaussian (N, 3, 3) /
    (N, 3) (the pose gradient of Sec. 2.5 differentiates through these).

    Returns a dict with mean2d (N, 2), conic (N, 3) = (a, b, c), cov2d (N, 3)
    = (Sxx, Sxy, Syy) after dilation, opacity (N,), rgb (N, 3), depth (N,),
    level t (N,), valid (N,) bool, rgb_clamped (N, 3) bool, J (N, 2, 3)."""
    if R is None:
        R, tr = camera_tensors(cam)
    else:
        tr = t
    means = params["means"]
    if R.dim() == 3:
        pc = torch.einsum("nij,nj->ni", R, means) + tr
    else:
        pc = means @ R.T + tr
    x, y, z = pc.unbind(-1)
    near = getattr(cam, "near", NEAR_DEFAULT)
    valid = z > near
    zs = torch.where(valid, z, torch.ones_like(z))  # keep culled rows finite

    rot = quat_to_rotmat(params["quats"])
    s = torch.exp(params["log_scales"])
    M = rot * s[:, None, :]  # R diag(s)
    sigma = M @ M.transpose(-1, -2)

    fx, fy, cx, cy = intrinsics(cam)
    tan_fovx = cam.width / (2.0 * fx)
    tan_fovy = cam.height / (2.0 * fy)
    limx = FRUSTUM_SLACK * tan_fovx
    limy = FRUSTUM_SLACK * tan_fovy
    txz = torch.clamp(x / zs, -limx, limx) * zs
    tyz = torch.clamp(y / zs, -limy, limy) * zs
    zero = torch.zeros_like(zs)
    J = torch.stack([
        torch.stack([fx / zs, zero, -fx * txz / (zs * zs)], -1),
        torch.stack([zero, fy / zs, -fy * tyz / (zs * zs)], -1),
    ], -2)
    T = J @ R
    cov = T @ sigma @ T.transpose(-1, -2)
    cov = cov + DILATION * torch.eye(2, dtype=_DT)
    sxx, sxy, syy = cov[:, 0, 0], cov[:, 0, 1], cov[:, 1, 1]
    det = sxx * syy - sxy * sxy
    conic = torch.stack([syy / det, -sxy / det, sxx / det], -1)

    mean2d = torch.stack([fx * x / zs + cx, fy * y / zs + cy], -1)
    opacity = torch.sigmoid(params["opacity_logits"])
    level = 2.0 * torch.log(255.0 * opacity)

    if R.dim() == 3:
        cam_centre = -torch.einsum("nji,nj->ni", R, tr)
    else:
        cam_centre = -(R.T @ tr)
    dvec = means - cam_centre
    dirs = dvec / torch.linalg.norm(dvec, dim=-1, keepdim=True)
    basis = sh_basis(sh_degree, dirs)  # (N, K)
    raw = torch.einsum("nk,nkc->nc", basis, params["sh"]) + 0.5
    rgb_clamped = raw < 0.0
    rgb = torch.clamp(raw, min=0.0)
    return {
        "mean2d": mean2d, "conic": conic,
        "cov2d": torch.stack([sxx, sxy, syy], -1), "opacity": opacity, "rgb": rgb,
        "depth": zs, "level": level, "valid": valid & (det > 0), "rgb_clamped": rgb_clamped,
        "J": J, "pc": pc,
    }


def pack_for_render(pr: dict) -> np.ndarray:
    """Rows of the render oracle's record (mx, my, a, b, c, o, r, g, b, z, t,
    valid), float64."""
    n = pr["mean2d"].shape[0]
    out = np.zeros((n, 12), dtype=np.float64)
    d = lambda k: pr[k].detach().numpy()
    out[:, 0:2] = d("mean2d")
    out[:, 2:5] = d("conic")
    out[:, 5] = d("opacity")
    out[:, 6:9] = d("rgb")
    out[:, 9] = d("depth")
    out[:, 10] = d("level")
    out[:, 11] = d("valid").astype(np.float64)
    return out


def preprocess_backward(scene, cam, grad2d: np.ndarray) -> dict:
    """Chain rule from per-Gaussian 2D gradients to the parameters.

    grad2d (N, 10): dL/d[mean2d x, y, conic a, b, c, opacity, r, g, b, 1/z].
    Returns float64 numpy gradients for means, log_scales, quats,
    opacity_logits and sh.  Culled Gaussians receive zero gradient."""
    params = params_from_scene(scene, requires_grad=True)
    pr = project(params, cam, scene.sh_degree)
    g = torch.as_tensor(grad2d, dtype=_DT)
    valid = pr["valid"].to(_DT)
    total = (
        (pr["mean2d"] * g[:, 0:2]).sum(-1)
        + (pr["conic"] * g[:, 2:5]).sum(-1)
        + pr["opacity"] * g[:, 5]
        + (pr["rgb"] * g[:, 6:9]).sum(-1)
        + (1.0 / pr["depth"]) * g[:, 9]
    )
    (total * valid).sum().backward()
    return {k: v.grad.detach().numpy().copy() for k, v in params.items()}


def preprocess_backward_abs(scene, cam, slack2d: np.ndarray) -> dict:
    """Bound on how far the parameter gradients move when each Gaussian's 2D
    gradients (N, 10) move by at most slack2d (elementwise, >= 0): for every
    Gaussian, sum over the ten 2D quantities of |d quantity / d parameter|
    times that quantity's slack.  The Jacobian of a Gaussian's 2D quantities
    depends only on its own parameters, so one autograd pass per quantity
    gives every Gaussian's column at once."""
    slack2d = np.asarray(slack2d, dtype=np.float64)
    out = None
    rows = np.nonzero(np.any(slack2d > 0, axis=1))[0]
    for c in range(slack2d.shape[1]):
        if not np.any(slack2d[:, c] > 0):
            continue
        e = np.zeros_like(slack2d)
        e[rows, c] = 1.0
        jc = preprocess_backward(scene, cam, e)
        if out is None:
            out = {k: np.zeros_like(v) for k, v in jc.items()}
        for k, v in jc.items():
            w = slack2d[:, c].reshape((-1,) + (1,) * (v.ndim - 1))
            out[k] += np.abs(v) * w
    if out is None:
        params = params_from_scene(scene)
        out = {k: np.zeros(tuple(v.shape)) for k, v in params.items()}
    return out
