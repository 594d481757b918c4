"""FP64 reference of the fit's parameterisation (Sec. 3.2) and of the
anisotropy regulariser (Eqs. E12, E13).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

mean = centre + half * mean_c; q = q_raw / |q_raw|; scale = exp(ls);
L_aniso = mean_i max(0, max(scale_i) / min(scale_i) - lambda_r) (the ratio of
the scales: E13 writes it on the log-scales). The gradient is taken by
plain PyTorch autograd on CPU in float64 (a library routine as a step) for
L = <g_mean, mean> + <g_quat, q> + <g_scale, scale> + lambda_aniso L_aniso.
Parity: pinned by central finite differences in tests/test_oracle_params.py.
"""
from __future__ import annotations

import numpy as np
import torch


def forward(mean_c, quat_raw, log_scale, centre, half, lambda_r):
    mc = torch.as_tensor(np.asarray(mean_c, np.float64))
    qr = torch.as_tensor(np.asarray(quat_raw, np.float64))
    ls = torch.as_tensor(np.asarray(log_scale, np.float64))
    mean = torch.as_tensor(np.asarray(centre, np.float64)) + half * mc
    q = qr / qr.norm(dim=1, keepdim=True)
    s = torch.exp(ls)
    aniso = torch.clamp(s.max(dim=1).values / s.min(dim=1).values - lambda_r, min=0.0).mean()
    return mean.numpy(), q.numpy(), s.numpy(), float(aniso)


def backward(mean_c, quat_raw, log_scale, centre, half, lambda_r, lambda_aniso, g_mean, g_quat, g_scale):
    mc = torch.tensor(np.asarray(mean_c, np.float64), requires_grad=True)
    qr = torch.tensor(np.asarray(quat_raw, np.float64), requires_grad=True)
    ls = torch.tensor(np.asarray(log_scale, np.float64), requires_grad=True)
    mean = torch.as_tensor(np.asarray(centre, np.float64)) + half * mc
    q = qr / qr.norm(dim=1, keepdim=True)
    s = torch.exp(ls)
    aniso = torch.clamp(s.max(dim=1).values / s.min(dim=1).values - lambda_r, min=0.0).mean()
    L = (mean * torch.as_tensor(np.asarray(g_mean, np.float64))).sum() + \
        (q * torch.as_tensor(np.asarray(g_quat, np.float64))).sum() + \
        (s * torch.as_tensor(np.asarray(g_scale, np.float64))).sum() + lambda_aniso * aniso
    L.backward()
    return mc.grad.numpy(), qr.grad.numpy(), ls.grad.numpy()
