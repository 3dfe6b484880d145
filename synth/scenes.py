"""Seeded scene, camera and target generators.

Every generator takes an integer seed and draws from numpy's
``Generator(PCG64(seed))``; the same seed gives the same arrays on x86 and on
aarch64.  Arrays are float32 (the precision the CUDA path stores parameters
in); the oracle widens exactly these float32 values to float64, so both sides
start from bit-identical inputs.

Recipes (sizes and distributions of the paper's workloads, Sec. 4):

* ``scene_c1``: 4096 Gaussians, x, y ~ U[-1, 1], z ~ U[2, 6], log-scales
  N(-3, 0.5), quaternions N(0, 1)^4 normalised, opacity logits N(0, 1),
  SH degree 0 whose colour is U(0, 1) per channel, seen by a pinhole camera at
  the origin looking down +z (fx = fy = 256, 256 x 256).
* ``scene_clustered``: N Gaussians in 64 anisotropic clusters with centres
  U[-1.5, 1.5]^3, Dirichlet(0.3) cluster weights (uneven per-tile load),
  cluster covariance R diag(sigma^2) R^T with sigma = exp(N(ln 0.25, 0.5)),
  log-scales N(-4, 0.7), SH degree 3 (DC from a U(0, 1) colour, higher
  coefficients N(0, 0.1)).
* ``ring_cameras``: cameras on a y = 0 ring of radius 4 looking at the origin,
  OpenCV axes (x right, y down, z forward), horizontal field of view 60 deg.
* ``camera_pose_error`` / ``with_pose_error``: one systematic camera-side
  pose error shared by every camera of a capture (the inaccurate poses that
  Sec. 2.5's global correction is for).
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

# The degree-0 real spherical harmonic is the constant 1/(2 sqrt(pi)); a DC
# coefficient f gives the colour f / (2 sqrt(pi)) + 0.5.  The generators draw
# the colour and store the coefficient, so this constant belongs to the input
# recipe ("colour ~ U(0, 1)"), not to the evaluation of the method.
_DC_SCALE = 2.0 * np.sqrt(np.pi)


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(int(seed)))


@dataclass
class Camera:
    """Pinhole camera, OpenCV axes; ``R``/``t`` map world to camera."""

    fx: float
    fy: float
    cx: float
    cy: float
    R: np.ndarray  # (3, 3) float64, world -> camera rotation
    t: np.ndarray  # (3,) float64, world -> camera translation
    width: int
    height: int
    near: float = 0.2

    def w2c(self) -> np.ndarray:
        """Row-major 3x4 [R | t] as float32 (the precision the GPU sees)."""
        m = np.concatenate([self.R, self.t[:, None]], axis=1)
        return m.astype(np.float32)


@dataclass
class Scene:
    means: np.ndarray  # (N, 3) float32
    log_scales: np.ndarray  # (N, 3) float32
    quats: np.ndarray  # (N, 4) float32, (w, x, y, z)
    opacity_logits: np.ndarray  # (N,) float32
    sh: np.ndarray  # (N, K, 3) float32, K = (deg + 1)^2
    sh_degree: int
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    def arrays(self):
        return (self.means, self.log_scales, self.quats, self.opacity_logits, self.sh)

    def copy(self) -> "Scene":
        return Scene(*(a.copy() for a in self.arrays()), sh_degree=self.sh_degree,
                     meta=dict(self.meta))


def _quats(rng, n):
    q = rng.standard_normal((n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    return q.astype(np.float32)


def _sh(rng, n, degree, rest_std):
    k = (degree + 1) ** 2
    sh = np.zeros((n, k, 3), dtype=np.float64)
    rgb = rng.uniform(0.0, 1.0, size=(n, 3))
    sh[:, 0, :] = (rgb - 0.5) * _DC_SCALE
    if k > 1:
        sh[:, 1:, :] = rng.normal(0.0, rest_std, size=(n, k - 1, 3))
    return sh.astype(np.float32)


def scene_c1(seed: int = 0, n: int = 4096) -> Scene:
    rng = _rng(seed)
    means = np.empty((n, 3))
    means[:, 0:2] = rng.uniform(-1.0, 1.0, size=(n, 2))
    means[:, 2] = rng.uniform(2.0, 6.0, size=n)
    log_scales = rng.normal(-3.0, 0.5, size=(n, 3))
    quats = _quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n)
    sh = _sh(rng, n, 0, 0.0)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats,
                 logits.astype(np.float32), sh, 0, meta={"recipe": "c1", "seed": seed})


def camera_c1() -> Camera:
    return Camera(256.0, 256.0, 128.0, 128.0, np.eye(3), np.zeros(3), 256, 256)


def _random_rotation(rng) -> np.ndarray:
    """Uniform random rotation from the QR factorisation of a normal matrix."""
    a = rng.standard_normal((3, 3))
    qm, rm = np.linalg.qr(a)
    qm = qm * np.sign(np.diag(rm))
    if np.linalg.det(qm) < 0:
        qm[:, 0] = -qm[:, 0]
    return qm


def scene_clustered(n: int, seed: int = 0, sh_degree: int = 3, n_clusters: int = 64,
                    log_scale_mean: float = -4.0, log_scale_std: float = 0.7,
                    rest_std: float = 0.1) -> Scene:
    rng = _rng(seed)
    centres = rng.uniform(-1.5, 1.5, size=(n_clusters, 3))
    weights = rng.dirichlet(np.full(n_clusters, 0.3))
    counts = rng.multinomial(n, weights)
    means = np.empty((n, 3))
    at = 0
    for c in range(n_clusters):
        m = int(counts[c])
        if m == 0:
            continue
        rot = _random_rotation(rng)
        sigma = np.exp(rng.normal(np.log(0.25), 0.5, size=3))
        local = rng.standard_normal((m, 3)) * sigma
        means[at:at + m] = centres[c] + local @ rot.T
        at += m
    perm = rng.permutation(n)
    means = means[perm]
    log_scales = rng.normal(log_scale_mean, log_scale_std, size=(n, 3))
    quats = _quats(rng, n)
    logits = rng.normal(0.0, 1.0, size=n)
    sh = _sh(rng, n, sh_degree, rest_std)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats,
                 logits.astype(np.float32), sh, sh_degree,
                 meta={"recipe": "clustered", "seed": seed, "n_clusters": n_clusters})


def _look_at(eye: np.ndarray, target: np.ndarray) -> tuple[np.ndarray, np.ndarray]:
    """World->camera (R, t) for OpenCV axes: +z towards target, +y down."""
    z = target - eye
    z = z / np.linalg.norm(z)
    down = np.array([0.0, 1.0, 0.0])
    x = np.cross(down, z)
    x = x / np.linalg.norm(x)
    y = np.cross(z, x)
    R = np.stack([x, y, z])
    t = -R @ eye
    return R, t


def ring_cameras(n_views: int = 16, width: int = 1920, height: int = 1080,
                 fov_x_deg: float = 60.0, radius: float = 4.0,
                 elevation: float = 0.0, phase: float = 0.0) -> list[Camera]:
    fx = 0.5 * width / np.tan(np.deg2rad(fov_x_deg) * 0.5)
    cams = []
    for v in range(n_views):
        th = phase + 2.0 * np.pi * v / n_views
        eye = np.array([radius * np.sin(th), elevation, radius * np.cos(th)])
        R, t = _look_at(eye, np.zeros(3))
        cams.append(Camera(fx, fx, 0.5 * width, 0.5 * height, R, t, width, height))
    return cams


def mixed_ring_cameras(n_views: int = 8, seed: int = 0) -> list[Camera]:
    """Views of uneven resolution for one batched launch: 3 x 960x540,
    3 x 1280x720, 2 x 1920x1080, at seeded ring angles."""
    rng = _rng(seed)
    sizes = [(960, 540)] * 3 + [(1280, 720)] * 3 + [(1920, 1080)] * 2
    sizes = (sizes * ((n_views + 7) // 8))[:n_views]
    cams = []
    for (w, h) in sizes:
        th = rng.uniform(0.0, 2.0 * np.pi)
        cams.append(ring_cameras(1, w, h, phase=th)[0])
    return cams


def orbit_cameras(n_views: int = 200, width: int = 1600, height: int = 1060, fov_x_deg: float = 60.0,
                  radius: float = 4.0, elev_min: float = -1.2, elev_max: float = 1.8) -> list[Camera]:
    """Views on a ring around the origin whose height swings between
    elev_min and elev_max three times per revolution (ring and elevation
    views of one object-centred capture)."""
    cams = []
    fx = 0.5 * width / np.tan(np.deg2rad(fov_x_deg) * 0.5)
    for v in range(n_views):
        th = 2.0 * np.pi * v / n_views
        y = elev_min + (elev_max - elev_min) * 0.5 * (1.0 - np.cos(3.0 * th))
        eye = np.array([radius * np.sin(th), y, radius * np.cos(th)])
        R, t = _look_at(eye, np.zeros(3))
        cams.append(Camera(fx, fx, 0.5 * width, 0.5 * height, R, t, width, height))
    return cams


def camera_pose_error(rot: float, trans: float, seed: int = 0) -> tuple[np.ndarray, np.ndarray]:
    """One seeded camera-side pose error: a rotation of `rot` radians about a
    uniformly random axis and a translation of length `trans` in a uniformly
    random direction, (R, t) in float64 (scipy builds the rotation)."""
    from scipy.spatial.transform import Rotation

    rng = _rng(seed)
    axis = rng.standard_normal(3)
    d = rng.standard_normal(3)
    R = Rotation.from_rotvec(rot * axis / np.linalg.norm(axis)).as_matrix()
    return R, trans * d / np.linalg.norm(d)


def with_pose_error(cams, R_err: np.ndarray, t_err: np.ndarray) -> list:
    """The cameras as a capture with a systematic pose error reports them:
    every camera's world -> camera transform [R | t] becomes
    [R_err R | R_err t + t_err] (the same error in each camera's own frame)."""
    from dataclasses import replace

    return [replace(c, R=R_err @ c.R, t=R_err @ c.t + t_err) for c in cams]


def recon_init(gt: Scene, n_init: int, seed: int = 0, pos_noise: float = 0.02, rgb_noise: float = 0.05,
               sh_degree: int = 3) -> Scene:
    """Starting point of a reconstruction from a sparse point cloud: n_init
    ground-truth centres with N(0, pos_noise) jitter, their DC colour with
    N(0, rgb_noise) noise, no higher SH, isotropic log-scale from the mean
    distance to the three nearest starting points, opacity 0.1, identity
    rotation (the usual 3DGS initialisation)."""
    from scipy.spatial import cKDTree

    rng = _rng(seed)
    idx = rng.choice(gt.n, size=n_init, replace=False)
    means = gt.means[idx].astype(np.float64) + rng.normal(0.0, pos_noise, size=(n_init, 3))
    dist, _ = cKDTree(means).query(means, k=4)
    d = np.maximum(dist[:, 1:].mean(axis=1), 1e-4)
    log_scales = np.repeat(np.log(d)[:, None], 3, axis=1)
    quats = np.zeros((n_init, 4), dtype=np.float32)
    quats[:, 0] = 1.0
    logits = np.full(n_init, np.log(0.1 / 0.9))
    K = (sh_degree + 1) ** 2
    sh = np.zeros((n_init, K, 3), dtype=np.float32)
    sh[:, 0, :] = gt.sh[idx, 0, :] + rng.normal(0.0, rgb_noise * _DC_SCALE, size=(n_init, 3))
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats, logits.astype(np.float32), sh,
                 sh_degree, meta={"recipe": "recon_init", "seed": seed, "n": n_init})


def scene_tiny(n: int = 6, seed: int = 0, sh_degree: int = 1, width: int = 16,
               height: int = 16) -> Scene:
    """A handful of Gaussians in front of ``camera_tiny`` (finite-difference
    sized scenes).  Scales are chosen so each covers several pixels."""
    rng = _rng(seed)
    means = np.empty((n, 3))
    means[:, 2] = rng.uniform(2.5, 4.0, size=n)
    means[:, 0] = rng.uniform(-0.25, 0.25, size=n) * means[:, 2]
    means[:, 1] = rng.uniform(-0.25, 0.25, size=n) * means[:, 2]
    log_scales = rng.normal(np.log(0.12), 0.3, size=(n, 3))
    quats = _quats(rng, n)
    logits = rng.normal(0.0, 0.8, size=n)
    sh = _sh(rng, n, sh_degree, 0.2)
    return Scene(means.astype(np.float32), log_scales.astype(np.float32), quats,
                 logits.astype(np.float32), sh, sh_degree,
                 meta={"recipe": "tiny", "seed": seed})


def camera_tiny(width: int = 16, height: int = 16) -> Camera:
    f = float(width)
    return Camera(f, f, 0.5 * width, 0.5 * height, np.eye(3), np.zeros(3), width, height)


def target_uniform(seed: int, width: int, height: int, channels: int = 3) -> np.ndarray:
    """Planar (C, H, W) float32 image with entries U(0, 1)."""
    rng = _rng(seed)
    return rng.uniform(0.0, 1.0, size=(channels, height, width)).astype(np.float32)


def upstream_grads(seed: int, width: int, height: int) -> tuple[np.ndarray, np.ndarray]:
    """Seeded upstream gradients (dL/dimage (3, H, W), dL/ddisparity (H, W))."""
    rng = _rng(seed)
    g = rng.normal(0.0, 1.0, size=(3, height, width)).astype(np.float32)
    gd = rng.normal(0.0, 1.0, size=(height, width)).astype(np.float32)
    return g, gd


def ng_anchors(points: np.ndarray, n_anchors: int, seed: int = 0, feat_dim: int = 32, hidden: int = 32,
               k_children: int = 10) -> dict:
    """Seeded neural-Gaussian anchor set: positions subsampled from `points`,
    features N(0, 0.1), offset log-scale log(0.02), child log-scale log(0.01),
    MLP weights N(0, 1 / fan_in), biases 0 except the rotation outputs'
    first component (1: identity rotation) and the opacity outputs (0.5)."""
    rng = _rng(seed)
    idx = rng.choice(points.shape[0], size=n_anchors, replace=False)
    xyz = points[idx].astype(np.float32)
    feat = rng.normal(0.0, 0.1, size=(n_anchors, feat_dim)).astype(np.float32)
    ls = np.empty((n_anchors, 6), dtype=np.float32)
    ls[:, 0:3] = np.log(0.02)
    ls[:, 3:6] = np.log(0.01)
    in_dim = feat_dim + 3
    out_dim = k_children * 14
    w1 = (rng.normal(0.0, 1.0, size=(hidden, in_dim)) / np.sqrt(in_dim)).astype(np.float32)
    b1 = np.zeros(hidden, dtype=np.float32)
    w2 = (rng.normal(0.0, 1.0, size=(out_dim, hidden)) / np.sqrt(hidden)).astype(np.float32)
    b2 = np.zeros(out_dim, dtype=np.float32)
    b2.reshape(k_children, 14)[:, 10] = 1.0
    b2.reshape(k_children, 14)[:, 3] = 0.5
    return {"anchor_xyz": xyz, "feat": feat, "anchor_ls": ls, "w1": w1, "b1": b1, "w2": w2, "b2": b2}
