"""GPU parity of the slice-pose gradient (mg_render_pose_grad, dL/dT_k)
against the FP64 oracle (itself pinned by finite differences)."""
import numpy as np
import pytest
import torch

import mg_synth as ms
import oracle as orc
from gpu_util import TOL_GRAD_REL, rel_l2, render_gpu

pytestmark = pytest.mark.gpu


def _unit32(G):
    q = np.asarray(G.quat, np.float64)
    q = (q / np.linalg.norm(q, axis=1, keepdims=True)).astype(np.float32)
    return ms.Gaussians(G.mean, q, G.scale, G.alpha)


def _check(G, stacks, seed):
    R, out, dev = render_gpu(G, stacks)
    rec = orc.records(G, stacks)
    gout = np.random.default_rng(seed).normal(size=R.dev.n_vox).astype(np.float32)
    R.backward(*dev, torch.from_numpy(gout).cuda())
    got = R.pose_grad(*dev).cpu().numpy().astype(np.float64)
    want = orc.pose_grad(G, stacks, rec, gout.astype(np.float64))
    for name, sl in (("dL/dt", slice(0, 3)), ("dL/domega", slice(3, 6))):
        r = rel_l2(got[:, sl], want[:, sl])
        assert r <= TOL_GRAD_REL, f"{name}: rel-L2 {r:.3e}"
    return got, want


@pytest.mark.parametrize("seed", [0, 1])
def test_pose_gradient_mixed_stacks(seed):
    rng = np.random.default_rng(seed)
    G = _unit32(ms.random_gaussians(250, 300 + seed, box=(-20, 20), sigma=(0.6, 3.0), aniso=3.0,
                                    negative_frac=0.1))
    stacks = [ms.make_stack(ms.AXIAL, 6, 37, 50, 1.0, 1.1, 3.0, 3.0),
              ms.make_stack(ms.random_rotations(1, rng)[0], 5, 48, 40, 0.9, 0.9, 2.0, 2.5, rng=rng,
                            max_rot_deg=5.0, max_trans_mm=1.0),
              ms.make_stack(ms.SAGITTAL, 4, 33, 17, 1.3, 1.2, 0.0, 4.0)]
    _check(G, stacks, seed)


def test_pose_gradient_with_in_plane_psf():
    rng = np.random.default_rng(6)
    G = _unit32(ms.random_gaussians(200, 320, box=(-18, 18), sigma=(0.6, 3.0), aniso=3.0))
    stacks = [ms.make_stack(ms.random_rotations(1, rng)[0], 5, 40, 36, 0.9, 0.9, 2.0, 2.5, psf_u=1.4, psf_v=0.7),
              ms.make_stack(ms.AXIAL, 4, 30, 30, 1.0, 1.0, 3.0, 3.0, psf_u=0.0, psf_v=1.2)]
    _check(G, stacks, 8)


def test_pose_gradient_degenerate_gaussians():
    """Needles and pancakes take the FP64 record geometry in the chain too."""
    rng = np.random.default_rng(4)
    G = ms.random_gaussians(100, 78, box=(-14, 14), sigma=(0.5, 2.0), aniso=1.5)
    sc = G.scale.copy()
    for i in range(0, G.n, 2):
        ax = rng.integers(3)
        sc[i, ax] *= rng.uniform(20, 60)
        sc[i, (ax + 1) % 3] /= rng.uniform(3, 8)
    G = _unit32(ms.Gaussians(G.mean, G.quat, sc, G.alpha))
    stacks = [ms.make_stack(ms.random_rotations(1, rng)[0], 6, 36, 44, 0.9, 0.9, 2.0, 3.0)]
    _check(G, stacks, 5)


def test_pose_gradient_needs_a_backward():
    from paper_2603_00145_b300 import _lib as L

    G = _unit32(ms.random_gaussians(40, 9, box=(-10, 10)))
    stacks = [ms.make_stack(ms.AXIAL, 3, 20, 20, 1.0, 1.0, 2.0, 2.0)]
    R, out, dev = render_gpu(G, stacks)
    with pytest.raises(L.MgError) as e:
        R.pose_grad(*dev)
    assert e.value.status == L.MG_ERR_STALE_WORKSPACE


def test_registration_recovers_known_slice_motion():
    """Joint motion estimation with the pose gradient: slices rendered from
    known Gaussians at their true poses, then every slice moved by up to
    0.6 mm and 1.5 degrees; Adam on the pose gradient brings them back."""
    from scipy.spatial.transform import Rotation

    from paper_2603_00145_b300 import SliceRenderer, recon
    from gpu_util import to_dev

    rng = np.random.default_rng(7)
    G = _unit32(ms.random_gaussians(400, 21, box=(-18, 18), sigma=(1.0, 3.0), aniso=2.5, alpha=(0.2, 1.0)))
    true = [ms.make_stack(ms.AXIAL, 6, 40, 40, 1.0, 1.0, 2.0, 3.0),
            ms.make_stack(ms.CORONAL, 6, 40, 40, 1.0, 1.0, 2.0, 3.0)]
    m, q, s, a = to_dev(G)
    R = SliceRenderer(true)
    target = R.forward(m, q, s, a).clone()
    x_true = R.dev.poses().double().cpu().numpy()
    S = x_true.shape[0]
    x_bad = x_true.copy()
    dt = rng.uniform(-0.6, 0.6, (S, 3))
    dw = rng.normal(size=(S, 3))
    dw *= np.radians(rng.uniform(0.3, 1.5, (S, 1))) / np.linalg.norm(dw, axis=1, keepdims=True)
    for k in range(S):
        x_bad[k, :9] = (x_true[k, :9].reshape(3, 3) @ Rotation.from_rotvec(dw[k]).as_matrix()).reshape(-1)
        x_bad[k, 9:] += dt[k]
    R.dev.set_poses(torch.from_numpy(x_bad).float().cuda())
    hist = recon.register_slices(R, m, q, s, a, target, iterations=150, lr_t=0.03, lr_r=0.005)
    x_fit = R.dev.poses().double().cpu().numpy()
    t_err = np.linalg.norm(x_fit[:, 9:] - x_true[:, 9:], axis=1)
    r_err = [np.degrees(np.linalg.norm(Rotation.from_matrix(x_fit[k, :9].reshape(3, 3).T @
                                                           x_true[k, :9].reshape(3, 3)).as_rotvec()))
             for k in range(S)]
    assert hist[-1] < 0.05 * hist[0], (hist[0], hist[-1])
    assert t_err.max() < 0.1, t_err
    assert max(r_err) < 0.25, r_err
