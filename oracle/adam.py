"""Oracle for the Adam update, float64 numpy.

TEST INFRASTRUCTURE: only the test suite, the smoke check and the benchmark's
CPU-baseline leg may import this module.

The paper does not name its optimiser; the 3DGS training it builds on uses
Adam, restated here with bias correction:
  m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2
  p <- p - lr * (m / (1 - b1^t)) / (sqrt(v / (1 - b2^t)) + eps)
"""
from __future__ import annotations

import numpy as np


def adam_step(p, g, m, v, step: int, lr: float, b1: float = 0.9, b2: float = 0.999,
              eps: float = 1e-15):
    p = np.asarray(p, dtype=np.float64)
    g = np.asarray(g, dtype=np.float64)
    m = b1 * np.asarray(m, dtype=np.float64) + (1.0 - b1) * g
    v = b2 * np.asarray(v, dtype=np.float64) + (1.0 - b2) * g * g
    mhat = m / (1.0 - b1 ** step)
    vhat = v / (1.0 - b2 ** step)
    p = p - lr * mhat / (np.sqrt(vhat) + eps)
    return p, m, v


def adam_step_visible(p, g, m, v, step: int, lr, visible, b1: float = 0.9, b2: float = 0.999,
                      eps: float = 1e-15):
    """Sparse (visible-only) Adam of the Taming-3DGS line that the paper
    builds on (Sec. 2.2): the rows (first axis) flagged in `visible` take the
    update above with the global step count; the other rows keep their
    parameters and both moments (their moments do not decay)."""
    p = np.asarray(p, dtype=np.float64).copy()
    m = np.asarray(m, dtype=np.float64).copy()
    v = np.asarray(v, dtype=np.float64).copy()
    vis = np.asarray(visible, dtype=bool)
    lr_rows = lr[vis] if np.ndim(lr) else lr
    p[vis], m[vis], v[vis] = adam_step(p[vis], np.asarray(g, dtype=np.float64)[vis], m[vis], v[vis], step, lr_rows,
                                       b1, b2, eps)
    return p, m, v
