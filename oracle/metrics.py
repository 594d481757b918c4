"""FP64 losses and image metrics (Sec. 3.5.2, Sec. 4.1.3).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

* ``l1_l2``: mean |r| + mean r^2 over all voxels, r = pred - target (the slice
  loss of the plain-fit workload).
* ``smooth_l1``: Eq. E11 averaged over voxels (0.5 r^2 for |r| < 1, else |r| - 0.5).
* ``psnr``: 10 log10(MAX^2 / MSE) with MAX = 1 (intensities in [0, 1]); the
  paper does not define its PSNR, this is the reading.
* ``aniso``: Eq. E13 with the ratio taken on the scales exp(s) (a ratio of
  log-scales has no meaning), mean over Gaussians.

Parity: pinned by closed forms on hand-made inputs in the tests.
"""
from __future__ import annotations

import numpy as np


def l1_l2(pred, target):
    r = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    n = r.size
    loss = np.abs(r).sum() / n + (r * r).sum() / n
    grad = (np.sign(r) + 2.0 * r) / n
    return loss, grad


def smooth_l1(pred, target):
    r = np.asarray(pred, np.float64) - np.asarray(target, np.float64)
    a = np.abs(r)
    v = np.where(a < 1.0, 0.5 * r * r, a - 0.5)
    g = np.where(a < 1.0, r, np.sign(r)) / r.size
    return v.mean(), g


def mse(a, b):
    d = np.asarray(a, np.float64) - np.asarray(b, np.float64)
    return float((d * d).mean())


def psnr(a, b, max_val: float = 1.0):
    m = mse(a, b)
    return float("inf") if m == 0 else 10.0 * np.log10(max_val * max_val / m)


def aniso(scale, lam_r: float = 1.5):
    s = np.asarray(scale, np.float64)
    ratio = s.max(axis=1) / s.min(axis=1)
    return float(np.maximum(0.0, ratio - lam_r).mean())
