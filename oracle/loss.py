"""Oracle for the photometric and disparity losses and their image gradients,
float64 PyTorch on the CPU.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

Paper passages: Eq. 5 (photometric loss (1 - lambda) L1 + lambda (1 - SSIM));
Sec. 3.1 (disparity supervision, weight 0.1 decayed to 0).  Readings where the
paper is silent: lambda = 0.2; SSIM with an 11 x 11 Gaussian window of
sigma = 1.5, C1 = 0.01^2, C2 = 0.03^2, zero-padded "same" windows, averaged
over channels and pixels; L1 is the mean absolute difference over all
channels and pixels; the disparity term is the mean absolute difference
of the blended disparity and the target disparity.  Gradients are autograd
through these definitions.
"""
from __future__ import annotations

import numpy as np
import torch
import torch.nn.functional as F

_DT = torch.float64
WINDOW = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2


def gaussian_window(size: int = WINDOW, sigma: float = SIGMA) -> torch.Tensor:
    """Normalised 2D Gaussian window (outer product of the 1D one)."""
    r = torch.arange(size, dtype=_DT) - (size - 1) / 2.0
    g = torch.exp(-(r * r) / (2.0 * sigma * sigma))
    g = g / g.sum()
    return g[:, None] * g[None, :]


def _win(x: torch.Tensor) -> torch.Tensor:
    """Zero-padded same-size windowed mean of each channel of (C, H, W)."""
    w = gaussian_window()[None, None]
    return F.conv2d(x[:, None], w, padding=WINDOW // 2)[:, 0]


def ssim(img: torch.Tensor, ref: torch.Tensor) -> torch.Tensor:
    """Mean SSIM of two (C, H, W) images."""
    mu_x = _win(img)
    mu_y = _win(ref)
    sxx = _win(img * img) - mu_x * mu_x
    syy = _win(ref * ref) - mu_y * mu_y
    sxy = _win(img * ref) - mu_x * mu_y
    num = (2.0 * mu_x * mu_y + C1) * (2.0 * sxy + C2)
    den = (mu_x * mu_x + mu_y * mu_y + C1) * (sxx + syy + C2)
    return (num / den).mean()


def photometric(img: np.ndarray, ref: np.ndarray, lam: float = 0.2):
    """(1 - lam) L1 + lam (1 - SSIM) and its gradient w.r.t. img."""
    x = torch.as_tensor(np.asarray(img, dtype=np.float64)).requires_grad_(True)
    y = torch.as_tensor(np.asarray(ref, dtype=np.float64))
    l1 = (x - y).abs().mean()
    loss = (1.0 - lam) * l1
    if lam != 0.0:
        loss = loss + lam * (1.0 - ssim(x, y))
    loss.backward()
    return float(loss.detach()), x.grad.numpy().copy()


def disparity_l1(disp: np.ndarray, ref: np.ndarray, weight: float):
    """weight * mean |disp - ref| and its gradient w.r.t. disp."""
    x = torch.as_tensor(np.asarray(disp, dtype=np.float64)).requires_grad_(True)
    y = torch.as_tensor(np.asarray(ref, dtype=np.float64))
    loss = weight * (x - y).abs().mean()
    loss.backward()
    return float(loss.detach()), x.grad.numpy().copy()
