"""Oracle for the neural-Gaussian (anchor + MLP) decoder and its backward,
float64 PyTorch on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

Paper passage: Sec. 2.3 (the Scaffold-GS representation: anchors with
learnable features and a shallow global MLP that infers the attributes of the
anchors' child Gaussians; gradients reach only the anchor features and the
MLP).  The paper gives no architecture; the reading used here (and by the
CUDA path) is:

  x_a   = [f_a (32), d_a (3)] with d_a = (anchor - camera centre) / |.|
  h_a   = ReLU(W1 x_a + b1)              W1: 32 x 35
  y_a   = W2 h_a + b2                    W2: 140 x 32  (10 children x 14)
  child c of anchor a, with u = y_a[14 c : 14 c + 14]:
    mean      = anchor + tanh(u[0:3]) * exp(s_off)       (s_off: 3 per anchor)
    opacity   = tanh(u[3]); a child with opacity <= 0 is not rendered
    colour    = sigmoid(u[4:7])
    log-scale = s_scale + log(sigmoid(u[7:10]))          (s_scale: 3 per anchor)
    rotation  = u[10:14] (normalised by the preprocess)
  handed to the splatting step as Gaussian parameters: opacity logit
  log(o / (1 - o)) (o clipped below 1 - 1e-6; -30 for o <= 0), SH degree 0
  with DC coefficient (colour - 0.5) * 2 sqrt(pi).

Precision of the method (the tensor-core formulation): the GEMM operands are
bfloat16 and the sums float32.  The oracle rounds to bfloat16 at the same
points, correctly rounded from float64:
  forward:  f_a, d_a, W1, W2 and h_a (after the ReLU) are rounded;
  backward: dL/dy and dL/dh (after the ReLU mask) are rounded before they
            enter dL/dh = W2^T dy, dL/dx = W1^T dh, dW2 = sum dy h^T and
            dW1 = sum dh x^T; the bias gradients use the unrounded values.
With bf16=False every rounding is skipped and the explicit backward must equal
autograd of the forward (pinned in the tests).
"""
from __future__ import annotations

import math

import numpy as np
import torch

_DT = torch.float64
K_CHILD = 10
OUT_PER_CHILD = 14
FEAT = 32
HIDDEN = 32
IN_DIM = FEAT + 3
OUT_DIM = K_CHILD * OUT_PER_CHILD
LOGIT_FLOOR = -30.0
OPACITY_CEIL = 1.0 - 1e-6
DC_SCALE = 2.0 * math.sqrt(math.pi)


def bf16_round(t: torch.Tensor) -> torch.Tensor:
    """Round float64 values to the nearest bfloat16 (ties to even), returned
    as float64.  bfloat16 keeps 8 significant bits."""
    a = t.detach().numpy() if isinstance(t, torch.Tensor) else np.asarray(t, dtype=np.float64)
    m, e = np.frexp(a)  # a = m 2^e, 0.5 <= |m| < 1
    r = np.ldexp(np.rint(m * 256.0) / 256.0, e)
    return torch.as_tensor(r, dtype=_DT)


def _maybe(x, on):
    return bf16_round(x) if on else x


def view_dirs(anchor_xyz: torch.Tensor, campos) -> torch.Tensor:
    d = anchor_xyz - torch.as_tensor(np.asarray(campos, dtype=np.float64))
    return d / torch.linalg.norm(d, dim=-1, keepdim=True)


def decode_forward(anchor_xyz, feat, anchor_ls, w1, b1, w2, b2, campos, bf16: bool = True):
    """Child Gaussian parameters (float64) and the cache for the backward.

    Shapes: anchor_xyz (A, 3), feat (A, 32), anchor_ls (A, 6), w1 (32, 35),
    b1 (32,), w2 (140, 32), b2 (140,).  Returns a dict with means (A*10, 3),
    log_scales, quats (A*10, 4), opacity_logits (A*10,), sh (A*10, 1, 3)."""
    T = lambda a: a.to(_DT) if isinstance(a, torch.Tensor) else torch.as_tensor(np.asarray(a, dtype=np.float64))
    xyz, feat, ls = T(anchor_xyz), T(feat), T(anchor_ls)
    w1, b1, w2, b2 = T(w1), T(b1), T(w2), T(b2)
    A = xyz.shape[0]
    d = view_dirs(xyz, campos)
    x = torch.cat([_maybe(feat, bf16), _maybe(d, bf16)], 1)
    w1r, w2r = _maybe(w1, bf16), _maybe(w2, bf16)
    h_pre = x @ w1r.T + b1
    h_absum = x.abs() @ w1r.abs().T + b1.abs()  # scale of the float32 rounding of h_pre
    h = _maybe(torch.clamp(h_pre, min=0.0), bf16)
    y = h @ w2r.T + b2
    u = y.reshape(A, K_CHILD, OUT_PER_CHILD)
    s_off = torch.exp(ls[:, 0:3])[:, None, :]
    off = torch.tanh(u[..., 0:3]) * s_off
    means = xyz[:, None, :] + off
    o = torch.tanh(u[..., 3])
    oc = torch.clamp(o, max=OPACITY_CEIL)
    logit = torch.where(o > 0, torch.log(oc.clamp(min=1e-300)) - torch.log1p(-oc), torch.full_like(o, LOGIT_FLOOR))
    rgb = torch.sigmoid(u[..., 4:7])
    log_scales = ls[:, None, 3:6] + torch.nn.functional.logsigmoid(u[..., 7:10])
    quats = u[..., 10:14]
    out = {
        "means": means.reshape(-1, 3), "log_scales": log_scales.reshape(-1, 3),
        "quats": quats.reshape(-1, 4), "opacity_logits": logit.reshape(-1),
        "sh": ((rgb - 0.5) * DC_SCALE).reshape(-1, 1, 3),
    }
    cache = {k: v.detach() for k, v in {"x": x, "h_pre": h_pre, "h": h, "y": y, "u": u, "o": o, "rgb": rgb,
                                         "off": off, "s_off": s_off, "w1r": w1r, "w2r": w2r,
                                         "h_absum": h_absum}.items()}
    cache["A"] = A
    return out, cache


def decode_backward(cache, grads: dict, bf16: bool = True) -> dict:
    """Gradients of the anchor features, anchor log-scales and MLP from the
    child parameter gradients (keys as decode_forward's outputs)."""
    T = lambda a: torch.as_tensor(np.asarray(a, dtype=np.float64))
    A = cache["A"]
    u, o, rgb, off, s_off = cache["u"], cache["o"], cache["rgb"], cache["off"], cache["s_off"]
    g_mean = T(grads["means"]).reshape(A, K_CHILD, 3)
    g_ls = T(grads["log_scales"]).reshape(A, K_CHILD, 3)
    g_q = T(grads["quats"]).reshape(A, K_CHILD, 4)
    g_logit = T(grads["opacity_logits"]).reshape(A, K_CHILD)
    g_sh = T(grads["sh"]).reshape(A, K_CHILD, 3)
    du = torch.zeros_like(u)
    th = torch.tanh(u[..., 0:3])
    du[..., 0:3] = g_mean * s_off * (1.0 - th * th)
    d_soff = (g_mean * off).sum(1)  # d/d s_off of tanh * exp(s_off)
    oc = torch.clamp(o, max=OPACITY_CEIL)
    vis = (o > 0) & (o < OPACITY_CEIL)
    du[..., 3] = torch.where(vis, g_logit / (oc * (1.0 - oc)) * (1.0 - o * o), torch.zeros_like(o))
    du[..., 4:7] = g_sh * DC_SCALE * rgb * (1.0 - rgb)
    du[..., 7:10] = g_ls * torch.sigmoid(-u[..., 7:10])
    du[..., 10:14] = g_q
    d_sscale = g_ls.sum(1)
    dy = du.reshape(A, -1)
    dy_r = _maybe(dy, bf16)
    dh = dy_r @ cache["w2r"]
    dh_pre = dh * (cache["h_pre"] > 0).to(_DT)
    dh_r = _maybe(dh_pre, bf16)
    dx = dh_r @ cache["w1r"]
    return {
        "feat": dx[:, :FEAT].numpy().copy(),
        "anchor_ls": torch.cat([d_soff, d_sscale], 1).numpy().copy(),
        "w2": (dy_r.T @ cache["h"]).numpy().copy(),
        "b2": dy.sum(0).numpy().copy(),
        "w1": (dh_r.T @ cache["x"]).numpy().copy(),
        "b1": dh_pre.sum(0).numpy().copy(),
        "_dy": dy.numpy().copy(),
        "_dh_pre": dh_pre.numpy().copy(),
        "_dh_absum": (dy_r.abs() @ cache["w2r"].abs()).numpy().copy(),
    }


def bf16_midpoint_distance(v) -> np.ndarray:
    """Absolute distance of v to the nearest bfloat16 rounding midpoint (a
    float32 evaluation of v that is off by less than this rounds to the same
    bfloat16 value)."""
    a = np.asarray(v, dtype=np.float64)
    m, e = np.frexp(a)
    t = np.abs(m) * 256.0
    frac = t - np.floor(t)
    return np.where(a != 0.0, np.abs(frac - 0.5) * np.ldexp(1.0, e - 8), np.inf)
