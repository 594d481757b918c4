"""FP64 reference of the optimiser step of the fit (Sec. 4.1.4: Adam with one
learning rate per parameter group).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

Adam as defined by Kingma & Ba (2015, Algorithm 1), with epsilon added to the
square root of the bias-corrected second moment; with t the step number
after the increment:

    m_t = b1 m_{t-1} + (1 - b1) g
    v_t = b2 v_{t-1} + (1 - b2) g^2
    m^  = m_t / (1 - b1^t),   v^ = v_t / (1 - b2^t)
    p_t = p_{t-1} - lr m^ / (sqrt(v^) + eps)

followed, for a group with a range, by the clamp of p to [lo, hi] (the alpha
range of Sec. 3.2). A skipped step (the device status predicate) leaves p, m,
v and t unchanged.

Parity: pinned by the tests against torch.optim.Adam in float64 on the CPU
(a library routine of the same definition), and by closed forms: the first
step moves p by -lr g / (|g| + eps); a constant gradient keeps m^ = g and
v^ = g^2 at every step.
"""
from __future__ import annotations

import numpy as np


class Adam:
    def __init__(self, params, lrs, betas=(0.9, 0.999), eps=1e-8, clamps=None):
        self.p = [np.asarray(x, np.float64).copy() for x in params]
        self.lr = [float(x) for x in lrs]
        self.b1, self.b2 = float(betas[0]), float(betas[1])
        self.eps = float(eps)
        self.clamps = list(clamps) if clamps is not None else [None] * len(self.p)
        self.m = [np.zeros_like(x) for x in self.p]
        self.v = [np.zeros_like(x) for x in self.p]
        self.t = 0

    def step(self, grads, skip: bool = False):
        if skip:
            return
        self.t += 1
        t = self.t
        for k, g in enumerate(grads):
            g = np.asarray(g, np.float64)
            self.m[k] = self.b1 * self.m[k] + (1.0 - self.b1) * g
            self.v[k] = self.b2 * self.v[k] + (1.0 - self.b2) * g * g
            m_hat = self.m[k] / (1.0 - self.b1 ** t)
            v_hat = self.v[k] / (1.0 - self.b2 ** t)
            self.p[k] = self.p[k] - self.lr[k] * m_hat / (np.sqrt(v_hat) + self.eps)
            if self.clamps[k] is not None:
                lo, hi = self.clamps[k]
                self.p[k] = np.clip(self.p[k], lo, hi)
