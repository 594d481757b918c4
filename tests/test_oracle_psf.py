"""Pins of the oracle with a full 3-D PSF (slice profile plus an in-plane
Gaussian PSF, Sigma' = Sigma + R_k diag(pu^2, pv^2, ps^2) R_k^T): a textbook
separable convolution, an explicit 2-D convolution of the PSF-free slice on
a fine grid, and central finite differences of the analytic gradient."""
import types

import numpy as np

import mg_synth as ms
import oracle as orc

F2V = 1.0 / (8.0 * np.log(2.0))


def _g64(G):
    q = np.asarray(G.quat, np.float64)
    q = q / np.linalg.norm(q, axis=1, keepdims=True)
    return types.SimpleNamespace(mean=np.asarray(G.mean, np.float64).copy(), quat=q.copy(),
                                 scale=np.asarray(G.scale, np.float64).copy(),
                                 alpha=np.asarray(G.alpha, np.float64).copy())


def _one(st, R, t, H=1, W=1, dx=None, dy=None, psf=True):
    xf = np.concatenate([np.asarray(R, np.float64).reshape(-1), np.asarray(t, np.float64)])[None, :]
    return types.SimpleNamespace(n_slices=1, H=H, W=W, dx=dx or st.dx, dy=dy or st.dy, thickness=st.thickness,
                                 psf_u=st.psf_u if psf else 0.0, psf_v=st.psf_v if psf else 0.0, xform=xf,
                                 n_vox=H * W)


def test_isotropic_textbook_separable_convolution():
    s, a = 1.4, 0.9
    G = ms.Gaussians(np.array([[0.4, -0.3, 0.7]]), np.array([[1.0, 0, 0, 0]]), np.full((1, 3), s), np.array([a]))
    st = ms.make_stack(ms.AXIAL, 3, 9, 8, 0.7, 0.8, 2.0, 1.3, psf_u=1.2, psf_v=0.7)
    S = orc.render(G, [st], exact=True).reshape(st.n_slices, st.H, st.W)
    s, a = float(G.scale[0, 0]), float(G.alpha[0])
    vu, vv, vs = (st.psf_u ** 2) * F2V, (st.psf_v ** 2) * F2V, (st.thickness ** 2) * F2V
    mu = G.mean[0].astype(np.float64)
    for k in range(st.n_slices):
        xf = st.xform[k].astype(np.float64)
        for j in range(st.H):
            for i in range(st.W):
                x = xf[:9].reshape(3, 3) @ [(i - (st.W - 1) / 2) * st.dx, (j - (st.H - 1) / 2) * st.dy, 0] + xf[9:]
                d = x - mu
                ref = a * s ** 3 / np.sqrt((s * s + vu) * (s * s + vv) * (s * s + vs)) * np.exp(
                    -d[0] ** 2 / (2 * (s * s + vu)) - d[1] ** 2 / (2 * (s * s + vv)) - d[2] ** 2 / (2 * (s * s + vs)))
                assert abs(S[k, j, i] - ref) <= 1e-14 + 1e-12 * abs(ref)


def test_in_plane_psf_is_a_2d_convolution_of_the_slice():
    """S_psf(p) = integral of phi_u(a) phi_v(b) S(p - (a, b)) da db, the
    PSF-free thick-slice value S sampled on a fine grid in the slice plane
    (trapezoid rule: spectrally accurate for these smooth integrands)."""
    rng = np.random.default_rng(5)
    G = _g64(ms.random_gaussians(6, 31, box=(-2, 2), sigma=(0.7, 2.0), aniso=3.0, negative_frac=0.3))
    R = ms.random_rotations(1, rng)[0].astype(np.float64)
    st = ms.make_stack(ms.AXIAL, 1, 1, 1, 1.0, 1.0, 1.8, 1.0, psf_u=1.1, psf_v=0.8)
    su, sv = st.psf_u * np.sqrt(F2V), st.psf_v * np.sqrt(F2V)
    h = 0.04
    N = 2 * int(np.ceil(7 * max(su, sv) / h)) + 1
    off = (np.arange(N) - (N - 1) / 2) * h
    wu = np.exp(-off ** 2 / (2 * su * su)) / (np.sqrt(2 * np.pi) * su)
    wv = np.exp(-off ** 2 / (2 * sv * sv)) / (np.sqrt(2 * np.pi) * sv)
    for _ in range(3):
        t = rng.uniform(-1.5, 1.5, 3)
        got = orc.render(G, [_one(st, R, t)], exact=True)[0]
        fine = orc.render(G, [_one(st, R, t, H=N, W=N, dx=h, dy=h, psf=False)], exact=True).reshape(N, N)
        ref = float(wv @ fine @ wu) * h * h
        assert abs(got - ref) <= 1e-9 * max(1.0, abs(ref)), (got, ref)


def test_gradient_with_psf_vs_central_fd():
    rng = np.random.default_rng(8)
    G = ms.random_gaussians(20, 91, box=(-8, 8), sigma=(0.8, 2.5), aniso=3.0, alpha=(-1.0, 1.0))
    stacks = [ms.make_stack(ms.random_rotations(1, rng)[0], 3, 18, 20, 0.9, 1.0, 2.0, 2.5, psf_u=1.3, psf_v=0.6),
              ms.make_stack(ms.CORONAL, 2, 16, 16, 1.0, 1.0, 0.0, 3.0, psf_u=0.9, psf_v=0.0)]
    rec = orc.records(G, stacks, 3.0)
    gout = rng.normal(size=sum(s.n_vox for s in stacks))
    gr = orc.grad(G, stacks, rec, gout)

    def loss(Gx):
        return float(np.dot(gout, orc.render(Gx, stacks, rec)))

    for name, width in (("mean", 3), ("quat", 4), ("scale", 3), ("alpha", 1)):
        for _ in range(5):
            g, c = int(rng.integers(G.n)), int(rng.integers(width))
            idx = (g, c) if width > 1 else (g,)
            Gp, Gm = _g64(G), _g64(G)
            Gp.quat, Gm.quat = np.asarray(G.quat, np.float64).copy(), np.asarray(G.quat, np.float64).copy()
            base = float(getattr(Gp, name)[idx])
            hh = 1e-6 * max(1.0, abs(base))
            getattr(Gp, name)[idx] = base + hh
            getattr(Gm, name)[idx] = base - hh
            fd = (loss(Gp) - loss(Gm)) / (2 * hh)
            an = float(gr[name][idx])
            scale = max(abs(fd), 1e-3 * float(np.abs(gr[name]).max()))
            assert abs(fd - an) <= 1e-6 * scale, (name, idx, fd, an)
