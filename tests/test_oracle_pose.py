"""Pin of the oracle's slice-pose gradient (dL/dT_k, Sec. 3.3.2 transforms)
against central finite differences of the FP64 render in the transforms."""
import types

import numpy as np
from scipy.spatial.transform import Rotation

import mg_synth as ms
import oracle as orc


def _unit(G):
    q = np.asarray(G.quat, np.float64)
    return ms.Gaussians(np.asarray(G.mean, np.float64), q / np.linalg.norm(q, axis=1, keepdims=True),
                        np.asarray(G.scale, np.float64), np.asarray(G.alpha, np.float64))


def _stack64(s, xf):
    return types.SimpleNamespace(n_slices=s.n_slices, H=s.H, W=s.W, dx=s.dx, dy=s.dy, thickness=s.thickness,
                                 xform=xf, n_vox=s.n_slices * s.H * s.W)


def test_pose_gradient_matches_finite_differences():
    rng = np.random.default_rng(3)
    G = _unit(ms.random_gaussians(60, 11, box=(-12, 12), sigma=(0.8, 3.0), aniso=3.0, negative_frac=0.2))
    stacks = [ms.make_stack(ms.random_rotations(1, rng)[0], 3, 24, 28, 1.0, 1.1, 2.5, 3.0, rng=rng,
                            max_rot_deg=4.0, max_trans_mm=1.0),
              ms.make_stack(ms.AXIAL, 2, 20, 17, 1.2, 1.2, 0.0, 4.0)]
    rec = orc.records(G, stacks)
    n_vox = sum(s.n_vox for s in stacks)
    gout = rng.normal(size=n_vox)
    pg = orc.pose_grad(G, stacks, rec, gout)
    base = [np.asarray(s.xform, np.float64).reshape(-1, 12).copy() for s in stacks]

    def loss(xfs):
        st = [_stack64(s, x) for s, x in zip(stacks, xfs)]
        return float(gout @ orc.render(G, st, rec))

    h = 1e-5
    k = 0
    for si, s in enumerate(stacks):
        for j in range(s.n_slices):
            for c in range(6):
                xp = [x.copy() for x in base]
                xm = [x.copy() for x in base]
                if c < 3:
                    xp[si][j, 9 + c] += h
                    xm[si][j, 9 + c] -= h
                else:
                    e = np.zeros(3)
                    e[c - 3] = h
                    R = base[si][j, :9].reshape(3, 3)
                    xp[si][j, :9] = (R @ Rotation.from_rotvec(e).as_matrix()).reshape(-1)
                    xm[si][j, :9] = (R @ Rotation.from_rotvec(-e).as_matrix()).reshape(-1)
                fd = (loss(xp) - loss(xm)) / (2 * h)
                scale = max(1.0, np.abs(pg[k]).max())
                assert abs(fd - pg[k, c]) <= 2e-6 * scale, (si, j, c, fd, pg[k, c])
            k += 1
