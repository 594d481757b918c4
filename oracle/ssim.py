"""FP64 reference of the reconstruction loss with the SSIM term (Sec. 3.5.2):
L_recon = L_L1 + lambda_SSIM * L_SSIM, L_L1 the smooth-L1 (Huber) mean of
Eq. E11, lambda_SSIM = 0.5 (Sec. 4.1.4).

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``).

The paper does not write L_SSIM out. Reading: L_SSIM = 1 - mean SSIM, the
mean over every pixel of every rendered slice of the structural similarity
of Wang et al. (2004) between the rendered and the acquired slice, each 2-D
slice on its own (the paper notes that the SSIM term needs whole slices).
Per pixel p, with w the 11 x 11 Gaussian window of standard deviation 1.5
pixels (normalised to unit sum, centred on p) and zero padding outside the
slice:

    mu_x = sum_q w x_q,  mu_y = sum_q w y_q,
    s_xx = sum_q w x_q^2 - mu_x^2,  s_yy = sum_q w y_q^2 - mu_y^2,
    s_xy = sum_q w x_q y_q - mu_x mu_y,
    SSIM_p = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)),
    C1 = (0.01 L)^2, C2 = (0.03 L)^2, L = 1 (intensities in [0, 1]).

The gradient with respect to the rendered slice x follows from the chain
rule through the five windowed moments (the window is symmetric, so the
adjoint of the zero-padded windowed sum is the same windowed sum):

    dL/dx_q = sum_p w(p-q) [dS_p/dmu_x + 2 x_q dS_p/dE_xx + y_q dS_p/dE_xy] * dL/dS_p

with E_xx = sum w x^2 and E_xy = sum w x y the raw moments.

Parity: pinned in tests/test_oracle_ssim.py by a per-pixel double loop
over the window (the definition written out, without separable filtering),
SSIM(x, x) = 1, the closed form for constant images away from the border,
the symmetry SSIM(x, y) = SSIM(y, x), and central finite differences of the
loss.
"""
from __future__ import annotations

import numpy as np
from scipy.ndimage import correlate1d

WIN = 11
SIGMA = 1.5
C1 = 0.01 ** 2
C2 = 0.03 ** 2
LAMBDA_SSIM = 0.5


def window_1d(size: int = WIN, sigma: float = SIGMA) -> np.ndarray:
    k = np.arange(size, dtype=np.float64) - (size - 1) / 2.0
    g = np.exp(-k * k / (2.0 * sigma * sigma))
    return g / g.sum()


def _blur(a: np.ndarray) -> np.ndarray:
    """Zero-padded windowed sum over a 2-D image (the 2-D window is the
    outer product of the 1-D one, so two 1-D passes give it exactly)."""
    g = window_1d()
    t = correlate1d(np.asarray(a, np.float64), g, axis=1, mode="constant", cval=0.0)
    return correlate1d(t, g, axis=0, mode="constant", cval=0.0)


def _moments(x, y):
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    return _blur(x), _blur(y), _blur(x * x), _blur(y * y), _blur(x * y)


def ssim_map(x, y) -> np.ndarray:
    mx, my, exx, eyy, exy = _moments(x, y)
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2.0 * mx * my + C1, 2.0 * sxy + C2
    b1, b2 = mx * mx + my * my + C1, sxx + syy + C2
    return (a1 * a2) / (b1 * b2)


def sensitivities(mx, my, exx, eyy, exy):
    """SSIM_p and its partial derivatives with respect to mu_x, E_xx and
    E_xy (the moments of the predicted image), from the window moments.
    SSIM_p = N / D with N = a1 a2, D = b1 b2; by the quotient rule
    (N' D - N D') / D^2. a1 and a2 vanish for anti-correlated windows, while
    b1 >= C1 and b2 >= C2, so only D is divided by."""
    sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
    a1, a2 = 2.0 * mx * my + C1, 2.0 * sxy + C2
    b1, b2 = mx * mx + my * my + C1, sxx + syy + C2
    d = b1 * b2
    s = (a1 * a2) / d
    # N' = (2 my a2 - 2 my a1, 0, 2 a1), D' = (2 mx b2 - 2 mx b1, b1, 0)
    d_mx = 2.0 * (my * (a2 - a1) - s * mx * (b2 - b1)) / d
    d_exx = -s / b2
    d_exy = 2.0 * a1 / d
    return s, d_mx, d_exx, d_exy


def ssim_grad(x, y, dl_ds) -> np.ndarray:
    """dL/dx for a per-pixel upstream gradient dL/dSSIM_p (2-D arrays)."""
    x = np.asarray(x, np.float64)
    y = np.asarray(y, np.float64)
    _, d_mx, d_exx, d_exy = sensitivities(*_moments(x, y))
    u = np.asarray(dl_ds, np.float64)
    return _blur(u * d_mx) + 2.0 * x * _blur(u * d_exx) + y * _blur(u * d_exy)


def recon_loss(pred_slices, target_slices, lam: float = LAMBDA_SSIM):
    """pred_slices, target_slices: lists of 2-D slices (any sizes). Returns
    (L_recon, mean smooth-L1, mean SSIM, dL_recon/dpred as a list)."""
    n = sum(np.asarray(p).size for p in pred_slices)
    l1 = 0.0
    ss = 0.0
    grads = []
    for x, y in zip(pred_slices, target_slices):
        x = np.asarray(x, np.float64)
        y = np.asarray(y, np.float64)
        r = x - y
        a = np.abs(r)
        l1 += float(np.where(a < 1.0, 0.5 * r * r, a - 0.5).sum())
        ss += float(ssim_map(x, y).sum())
        g = np.where(a < 1.0, r, np.sign(r)) / n
        g = g + ssim_grad(x, y, np.full(x.shape, -lam / n))
        grads.append(g)
    l1 /= n
    ss /= n
    return l1 + lam * (1.0 - ss), l1, ss, grads
