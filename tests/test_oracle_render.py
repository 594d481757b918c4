"""Pins of the oracle's slice render against facts fixed by the mathematics.

Each test checks the FP64 oracle against something other than itself:
adaptive quadrature of the profile integral, the paper's point form (Eq. E7)
evaluated through scipy's rotation routine, a textbook 1-D convolution, total
mass, rigid-motion equivariance, and the truncation bound of the binned sum.
"""
import types

import numpy as np
import pytest
from scipy import integrate
from scipy.spatial.transform import Rotation

import mg_synth as ms
import oracle as orc

FWHM2SIG = 1.0 / (2.0 * np.sqrt(2.0 * np.log(2.0)))


def _g64(G):
    """FP64 copy with quaternions renormalised in FP64 (the rotation formula
    assumes a unit quaternion; a float32 one is unit only to ~1e-7)."""
    q = np.asarray(G.quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    return types.SimpleNamespace(mean=np.asarray(G.mean, np.float64), quat=q,
                                 scale=np.asarray(G.scale, np.float64), alpha=np.asarray(G.alpha, np.float64))


def _cov_scipy(q, s):
    """Sigma = R diag(s^2) R^T with R from scipy (scalar-last quaternion order)."""
    R = Rotation.from_quat([q[1], q[2], q[3], q[0]]).as_matrix()
    return R @ np.diag(np.asarray(s, np.float64) ** 2) @ R.T


def _e7(x, mu, q, s, a):
    """Eq. E7 term at point x (Sec. 3.3.2)."""
    Sg = _cov_scipy(q, s)
    y = np.asarray(x) - np.asarray(mu, np.float64)
    return a * np.exp(-0.5 * y @ np.linalg.solve(Sg, y))


def _pixel_world(st, k, i, j):
    xf = np.asarray(st.xform[k], np.float64)
    R = xf[:9].reshape(3, 3)
    u = (i - (st.W - 1) / 2.0) * st.dx
    v = (j - (st.H - 1) / 2.0) * st.dy
    return R @ np.array([u, v, 0.0]) + xf[9:], R[:, 2]


def _oblique_stack(seed, n=3, H=9, W=11, thk=3.0, spacing=2.0):
    rng = np.random.default_rng(seed)
    F = ms.random_rotations(1, rng)[0]
    return ms.make_stack(F, n, H, W, 0.9, 1.1, thk, spacing, centre=rng.uniform(-2, 2, 3))


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_profile_closed_form_vs_quadrature(seed):
    """Slice value = int N(t; 0, sig_s^2) E7(x + t n) dt, by adaptive Gauss-Kronrod."""
    G = ms.random_gaussians(1, 100 + seed, box=(-3, 3), sigma=(0.8, 2.0), aniso=3.0, alpha=(0.3, 1.0))
    st = _oblique_stack(seed)
    S = orc.render(_g64(G), [st], exact=True).reshape(st.n_slices, st.H, st.W)
    sig = st.thickness * FWHM2SIG
    rng = np.random.default_rng(seed)
    for _ in range(6):
        k, i, j = rng.integers(st.n_slices), rng.integers(st.W), rng.integers(st.H)
        x, n = _pixel_world(st, k, i, j)

        def f(t):
            return np.exp(-0.5 * (t / sig) ** 2) / (sig * np.sqrt(2 * np.pi)) * _e7(
                x + t * n, G.mean[0], G.quat[0], G.scale[0], float(G.alpha[0]))

        val, err = integrate.quad(f, -14 * sig, 14 * sig, epsabs=0, epsrel=1e-13, limit=400)
        assert abs(S[k, j, i] - val) <= 1e-11 * max(abs(val), 1e-300) + 1e-15, (S[k, j, i], val)


def test_zero_thickness_is_e7():
    """With no slice profile the render is the paper's point form, Eq. E7."""
    G = ms.random_gaussians(5, 7, box=(-4, 4), sigma=(0.7, 2.0), aniso=4.0, alpha=(-1.0, 1.0))
    st = _oblique_stack(3, thk=0.0)
    S = orc.render(_g64(G), [st], exact=True).reshape(st.n_slices, st.H, st.W)
    for k in range(st.n_slices):
        for j in range(0, st.H, 2):
            for i in range(0, st.W, 3):
                x, _ = _pixel_world(st, k, i, j)
                ref = sum(_e7(x, G.mean[g], G.quat[g], G.scale[g], float(G.alpha[g])) for g in range(G.n))
                assert abs(S[k, j, i] - ref) <= 1e-12 * (1 + abs(ref))


def test_isotropic_textbook_convolution():
    """Sigma = s^2 I, axial slices: alpha s/sqrt(s^2+ss^2) exp(-(du^2+dv^2)/2s^2 - dw^2/2(s^2+ss^2))."""
    s, a = 1.7, 0.8
    G = ms.Gaussians(np.array([[0.3, -0.4, 0.9]]), np.array([[1.0, 0, 0, 0]]), np.full((1, 3), s), np.array([a]))
    st = ms.make_stack(ms.AXIAL, 4, 8, 10, 0.75, 0.6, 2.5, 1.5)
    S = orc.render(G, [st], exact=True).reshape(st.n_slices, st.H, st.W)
    s, a = float(G.scale[0, 0]), float(G.alpha[0])  # the float32 values the oracle sees
    ss2 = (2.5 * FWHM2SIG) ** 2
    mu = G.mean[0].astype(np.float64)
    for k in range(st.n_slices):
        for j in range(st.H):
            for i in range(st.W):
                x, _ = _pixel_world(st, k, i, j)
                d = x - mu
                ref = a * s / np.sqrt(s * s + ss2) * np.exp(-(d[0] ** 2 + d[1] ** 2) / (2 * s * s)
                                                           - d[2] ** 2 / (2 * (s * s + ss2)))
                assert abs(S[k, j, i] - ref) <= 1e-14 + 1e-13 * ref


def _mass(G):
    tot = 0.0
    for g in range(G.n):
        det = np.prod(np.asarray(G.scale[g], np.float64) ** 2)
        tot += float(G.alpha[g]) * (2 * np.pi) ** 1.5 * np.sqrt(det)
    return tot


def test_volume_mass_conservation():
    """h^3 * sum of the sampled volume = sum alpha (2 pi)^(3/2) |Sigma|^(1/2) (spacing <= sigma/2, K = 6)."""
    G = ms.random_gaussians(6, 11, box=(-5, 5), sigma=(1.2, 2.0), aniso=1.5, alpha=(0.2, 1.0))
    h = 0.5
    V = orc.sample_volume(_g64(G), 64, h, K=6.0)
    assert abs(V.sum() * h ** 3 / _mass(G) - 1.0) < 1e-7


def test_slice_mass_conservation():
    """sum over slices of (slice sum * dx * dy * spacing) = total mass: the profile has unit integral."""
    G = ms.random_gaussians(4, 12, box=(-2, 2), sigma=(1.0, 1.6), aniso=1.3, alpha=(0.2, 1.0))
    for frame in (ms.AXIAL, ms.CORONAL, ms.SAGITTAL):
        st = ms.make_stack(frame, 60, 64, 64, 0.5, 0.5, 2.0, 0.5)
        S = orc.render(_g64(G), [st], K=6.0)
        assert abs(S.sum() * 0.5 * 0.5 * 0.5 / _mass(G) - 1.0) < 1e-7


def _quat_mul(a, b):
    w1, x1, y1, z1 = a
    w2, x2, y2, z2 = b
    return np.array([w1 * w2 - x1 * x2 - y1 * y2 - z1 * z2, w1 * x2 + x1 * w2 + y1 * z2 - z1 * y2,
                     w1 * y2 - x1 * z2 + y1 * w2 + z1 * x2, w1 * z2 + x1 * y2 - y1 * x2 + z1 * w2])


@pytest.mark.parametrize("seed", [0, 1])
def test_rigid_equivariance(seed):
    """Moving every Gaussian and every slice by one rigid motion leaves S unchanged."""
    G = ms.random_gaussians(12, 20 + seed, box=(-6, 6), sigma=(0.8, 2.0), aniso=3.0)
    st = _oblique_stack(seed + 5, n=4, H=12, W=10)
    rng = np.random.default_rng(seed)
    qm = rng.normal(size=4)
    qm /= np.linalg.norm(qm)
    Qm = Rotation.from_quat([qm[1], qm[2], qm[3], qm[0]]).as_matrix()
    b = rng.uniform(-10, 10, 3)
    G64 = _g64(G)
    G2 = types.SimpleNamespace(mean=G64.mean @ Qm.T + b, quat=np.array([_quat_mul(qm, q) for q in G64.quat]),
                               scale=G64.scale, alpha=G64.alpha)
    xf = np.asarray(st.xform, np.float64).copy()
    for k in range(st.n_slices):
        R = xf[k, :9].reshape(3, 3)
        xf[k, :9] = (Qm @ R).reshape(-1)
        xf[k, 9:] = Qm @ xf[k, 9:] + b
    st2 = types.SimpleNamespace(n_slices=st.n_slices, H=st.H, W=st.W, dx=st.dx, dy=st.dy,
                                thickness=st.thickness, xform=xf, n_vox=st.n_vox)
    S1 = orc.render(G64, [st], exact=True)
    S2 = orc.render(G2, [st2], exact=True)
    assert np.max(np.abs(S1 - S2)) <= 1e-12 * max(1.0, np.abs(S1).max())
    # binned at K = 6 agrees up to bin changes (terms below exp(-18))
    S1b = orc.render(G, [st], K=6.0)
    assert np.max(np.abs(S1b - S1)) <= 1e-6


def test_binned_truncation_bound():
    """|S - S^bin| <= sum_i |alpha_i| c_i exp(-K^2/2): everything dropped lies outside the K-ellipsoid."""
    G = ms.random_gaussians(60, 31, box=(-12, 12), sigma=(0.8, 2.5), aniso=3.0, alpha=(-1.0, 1.0))
    st = [ms.make_stack(ms.AXIAL, 6, 30, 28, 1.0, 1.0, 3.0, 3.0), _oblique_stack(4, n=5, H=20, W=26)]
    for K in (2.0, 3.0):
        S = orc.render(G, st, exact=True)
        Sb = orc.render(G, st, K=K)
        bound = np.abs(G.alpha.astype(np.float64)).sum() * np.exp(-K * K / 2)
        assert np.max(np.abs(S - Sb)) <= bound
    # at K = 6 the binned sum equals the full sum to 1e-6 (pins bins + evaluation together)
    Sb6 = orc.render(G, st, K=6.0)
    assert np.max(np.abs(S - Sb6)) <= 1e-6


def test_sampler_is_e7_on_grid():
    G = ms.random_gaussians(3, 41, box=(-2, 2), sigma=(0.8, 1.5), aniso=2.0)
    Gd, h = 10, 0.75
    V = orc.sample_volume(_g64(G), Gd, h, centre=(0.25, -0.125, 0.375), exact=True)
    rng = np.random.default_rng(0)
    for _ in range(20):
        c, j, i = rng.integers(Gd, size=3)
        x = np.array([0.25, -0.125, 0.375]) + h * (np.array([i, j, c]) - (Gd - 1) / 2.0)
        ref = sum(_e7(x, G.mean[g], G.quat[g], G.scale[g], float(G.alpha[g])) for g in range(G.n))
        assert abs(V[c, j, i] - ref) <= 1e-12 * (1 + abs(ref))
