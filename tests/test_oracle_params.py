"""Pins of the oracle's parameterisation and regulariser (Sec. 3.2, E12/E13):
closed forms and central finite differences of the scalar it differentiates."""
import numpy as np

from oracle import params


def _case(seed, n=30):
    rng = np.random.default_rng(seed)
    return (rng.normal(size=(n, 3)) * 0.3, rng.normal(size=(n, 4)), rng.normal(size=(n, 3)) * 0.8,
            rng.normal(size=(n, 3)), rng.normal(size=(n, 4)), rng.normal(size=(n, 3)))


def test_forward_closed_forms():
    mc, qr, ls, *_ = _case(0)
    mean, q, s, an = params.forward(mc, qr, ls, (1.0, -2.0, 0.5), 40.0, 1.5)
    np.testing.assert_allclose(mean, np.array([1.0, -2.0, 0.5]) + 40.0 * mc, rtol=1e-15)
    np.testing.assert_allclose(np.linalg.norm(q, axis=1), 1.0, rtol=1e-15)
    np.testing.assert_allclose(s, np.exp(ls), rtol=1e-15)
    ratio = np.exp(ls.max(1) - ls.min(1))
    assert abs(an - np.maximum(ratio - 1.5, 0).mean()) < 1e-13


def test_backward_vs_central_fd():
    mc, qr, ls, gm, gq, gs = _case(1)
    centre, half, lr, la = (0.3, 0.1, -0.2), 25.0, 1.5, 0.7

    def L(mc_, qr_, ls_):
        mean, q, s, an = params.forward(mc_, qr_, ls_, centre, half, lr)
        return (mean * gm).sum() + (q * gq).sum() + (s * gs).sum() + la * an

    g_mc, g_qr, g_ls = params.backward(mc, qr, ls, centre, half, lr, la, gm, gq, gs)
    h = 1e-6
    for arr, g in ((mc, g_mc), (qr, g_qr), (ls, g_ls)):
        for idx in [(0, 0), (3, 1), (7, 2), (12, 0), (29, 1)]:
            p, m = arr.copy(), arr.copy()
            p[idx] += h
            m[idx] -= h
            args_p = [p if a is arr else a for a in (mc, qr, ls)]
            args_m = [m if a is arr else a for a in (mc, qr, ls)]
            fd = (L(*args_p) - L(*args_m)) / (2 * h)
            assert abs(fd - g[idx]) <= 1e-6 * max(1.0, abs(fd)), (idx, fd, g[idx])


def test_forward_known_values():
    """Values fixed by hand: a scaled identity quaternion normalises to the
    identity, an isotropic Gaussian has scale ratio 1 (no penalty above
    lambda_r = 1.5), scales (1, 2, 8) have ratio 8 (penalty 6.5); the mean of
    the two is 3.25."""
    mc = np.array([[0.0, 0.0, 0.0], [1.0, -1.0, 0.5]])
    qr = np.array([[2.0, 0.0, 0.0, 0.0], [0.0, 3.0, 0.0, 4.0]])
    ls = np.log(np.array([[0.5, 0.5, 0.5], [2.0, 8.0, 1.0]]))
    mean, q, s, an = params.forward(mc, qr, ls, (10.0, 20.0, 30.0), 4.0, 1.5)
    np.testing.assert_allclose(mean, [[10.0, 20.0, 30.0], [14.0, 16.0, 32.0]], rtol=1e-15)
    np.testing.assert_allclose(q, [[1.0, 0.0, 0.0, 0.0], [0.0, 0.6, 0.0, 0.8]], atol=1e-15)
    np.testing.assert_allclose(s, [[0.5, 0.5, 0.5], [2.0, 8.0, 1.0]], rtol=1e-14)
    assert abs(an - 3.25) < 1e-12
