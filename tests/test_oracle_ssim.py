"""Pins of the oracle's SSIM reconstruction loss (Sec. 3.5.2)."""
import numpy as np

from oracle import ssim


def _ssim_by_loops(x, y):
    """SSIM of every pixel from the definition: a double loop over the
    11 x 11 window, pixels outside the image counting as zero."""
    H, W = x.shape
    g = ssim.window_1d()
    w2 = np.outer(g, g)
    out = np.zeros((H, W))
    for i in range(H):
        for j in range(W):
            mx = my = exx = eyy = exy = 0.0
            for a in range(-5, 6):
                for b in range(-5, 6):
                    ii, jj = i + a, j + b
                    if 0 <= ii < H and 0 <= jj < W:
                        wt = w2[a + 5, b + 5]
                        mx += wt * x[ii, jj]
                        my += wt * y[ii, jj]
                        exx += wt * x[ii, jj] ** 2
                        eyy += wt * y[ii, jj] ** 2
                        exy += wt * x[ii, jj] * y[ii, jj]
            sxx, syy, sxy = exx - mx * mx, eyy - my * my, exy - mx * my
            out[i, j] = ((2 * mx * my + ssim.C1) * (2 * sxy + ssim.C2)) / \
                ((mx * mx + my * my + ssim.C1) * (sxx + syy + ssim.C2))
    return out


def test_window_is_the_normalised_gaussian():
    g = ssim.window_1d()
    assert g.size == 11 and abs(g.sum() - 1.0) < 1e-15
    assert abs(g[5] / g[6] - np.exp(1.0 / (2 * 1.5 ** 2))) < 1e-12


def test_map_matches_definition_by_loops():
    rng = np.random.default_rng(0)
    x = rng.uniform(0, 1, (9, 13))
    y = np.clip(x + rng.normal(0, 0.1, x.shape), 0, 1)
    np.testing.assert_allclose(ssim.ssim_map(x, y), _ssim_by_loops(x, y), rtol=1e-12, atol=1e-14)


def test_identity_symmetry_and_constant_closed_form():
    rng = np.random.default_rng(1)
    x = rng.uniform(0, 1, (20, 24))
    y = rng.uniform(0, 1, (20, 24))
    np.testing.assert_allclose(ssim.ssim_map(x, x), 1.0, atol=1e-12)
    np.testing.assert_allclose(ssim.ssim_map(x, y), ssim.ssim_map(y, x), rtol=1e-13)
    a, b = 0.3, 0.7
    s = ssim.ssim_map(np.full((30, 30), a), np.full((30, 30), b))
    # away from the border the window is inside: variances vanish, SSIM = (2ab + C1)/(a^2 + b^2 + C1)
    np.testing.assert_allclose(s[5:25, 5:25], (2 * a * b + ssim.C1) / (a * a + b * b + ssim.C1), rtol=1e-12)


def test_gradient_matches_central_differences():
    rng = np.random.default_rng(2)
    xs = [rng.uniform(0, 1, (12, 15)), rng.uniform(0, 1, (7, 9))]
    ys = [np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1) for x in xs]
    xs[0][3, 4] += 1.5   # one residual on the linear branch of the smooth L1
    L, l1, ss, g = ssim.recon_loss(xs, ys)
    assert abs(L - (l1 + 0.5 * (1 - ss))) < 1e-15
    h = 1e-6
    for k, (i, j) in [(0, (0, 0)), (0, (3, 4)), (0, (6, 7)), (0, (11, 14)), (1, (3, 4)), (1, (6, 0))]:
        xp = [x.copy() for x in xs]
        xm = [x.copy() for x in xs]
        xp[k][i, j] += h
        xm[k][i, j] -= h
        fd = (ssim.recon_loss(xp, ys)[0] - ssim.recon_loss(xm, ys)[0]) / (2 * h)
        assert abs(fd - g[k][i, j]) <= 1e-7 * max(1.0, abs(fd)) + 1e-10, (k, i, j, fd, g[k][i, j])


def test_sensitivities_where_the_numerator_factors_vanish():
    """mu_x = mu_y = 0 and E_xy = -C2/2 make a2 = 2 s_xy + C2 exactly zero (and
    a1 = C1): SSIM_p = 0 there, its derivatives are finite and equal central
    finite differences of SSIM_p in (mu_x, E_xx, E_xy)."""
    from oracle.ssim import C2, sensitivities

    pt = dict(mx=0.0, my=0.0, exx=0.01, eyy=0.02, exy=-C2 / 2)
    s, d_mx, d_exx, d_exy = sensitivities(**pt)
    assert s == 0.0 and np.isfinite([d_mx, d_exx, d_exy]).all()
    for key, got in (("mx", d_mx), ("exx", d_exx), ("exy", d_exy)):
        h = 1e-7
        up, dn = dict(pt), dict(pt)
        up[key] += h
        dn[key] -= h
        fd = (sensitivities(**up)[0] - sensitivities(**dn)[0]) / (2 * h)
        assert abs(fd - got) <= 1e-6 * max(1.0, abs(got)), (key, fd, got)
    # and at a generic point
    pt = dict(mx=0.3, my=0.5, exx=0.2, eyy=0.4, exy=0.1)
    s, *ds = sensitivities(**pt)
    for key, got in zip(("mx", "exx", "exy"), ds):
        h = 1e-6
        up, dn = dict(pt), dict(pt)
        up[key] += h
        dn[key] -= h
        fd = (sensitivities(**up)[0] - sensitivities(**dn)[0]) / (2 * h)
        assert abs(fd - got) <= 1e-7 * max(1.0, abs(got)), (key, fd, got)
