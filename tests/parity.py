"""Helpers shared by the GPU parity tests: running the CUDA path through the
C ABI on seeded inputs, and the comparison rules.

Tolerances (stated by the method's float32 precision target):
  per pixel     |gpu - ref| <= 1e-4 |ref| + 1e-7   on pixels the oracle does
                not flag as threshold-ambiguous or ill-conditioned
  per gradient  |gpu - ref| <= 1e-3 max(|ref|, 1e-3 max|ref|), elementwise
                over each gradient array (the ten per-Gaussian 2D gradients
                and the parameter gradients)
  block_mismatch  the normwise variant per Gaussian block (max over a
                Gaussian's entries of one parameter), used where the same sums
                are compared in two association orders
"""
from __future__ import annotations

import numpy as np
import torch

PIX_RTOL = 1e-4
PIX_ATOL = 1e-7
GRAD_RTOL = 1e-3


def pixel_mismatch(gpu: np.ndarray, ref: np.ndarray, mask: np.ndarray | None = None):
    """Boolean array of pixels outside the per-pixel tolerance (optionally
    restricted to `mask`)."""
    bad = np.abs(gpu - ref) > PIX_RTOL * np.abs(ref) + PIX_ATOL
    if mask is not None:
        bad &= mask
    return bad


def grad_mismatch(gpu: np.ndarray, ref: np.ndarray, rtol: float = GRAD_RTOL):
    scale = max(np.abs(ref).max(), 1e-30)
    tol = rtol * np.maximum(np.abs(ref), 1e-3 * scale)
    return np.abs(gpu - ref) > tol


def block_mismatch(gpu: np.ndarray, ref: np.ndarray, rtol: float = GRAD_RTOL):
    """Rows (one per Gaussian) whose normwise error exceeds the tolerance."""
    g = np.asarray(gpu, dtype=np.float64).reshape(gpu.shape[0], -1)
    r = np.asarray(ref, dtype=np.float64).reshape(ref.shape[0], -1)
    top = max(np.abs(r).max(), 1e-30)
    scale = np.maximum(np.abs(r).max(axis=1), 1e-3 * top)
    return np.abs(g - r).max(axis=1) > rtol * scale


def to_np(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy()


def view_image(flat: torch.Tensor, width: int, height: int, offset: int = 0, channels: int = 3):
    """(C, H, W) numpy image of view at pixel `offset` from a flat planar buffer."""
    n = width * height
    a = to_np(flat)[channels * offset: channels * offset + channels * n]
    return a.reshape(channels, height, width)


def cuda_available() -> bool:
    return torch.cuda.is_available()
